"""Pins against values the paper prints (tests/golden/paper_values.txt, each line cited): the
octree degree of Eq. 3, the grid and SH sizes and image sizes of the workloads, and the learning
rates used as RMSProp defaults.  No GPU."""
import os

import numpy as np
import pytest

import oracle
import seeded_inputs as si

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    vals = {}
    for line in open(os.path.join(HERE, "golden", "paper_values.txt")):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        kv, cite = line.split(";", 1)
        k, v = (x.strip() for x in kv.split("="))
        assert cite.strip().startswith("Sec."), line
        vals[k] = float(v)
    return vals


G = _golden()


def test_merge_divides_by_the_octree_degree():
    """Eq. 3: a merged parent holds (1/M) times the sum of its M children's values."""
    prims = np.array([[si.PRIM_SPHERE, si.Q // 4, si.Q // 4, si.Q // 4, si.Q // 10, 0, 0, 0]], np.int64)
    t = oracle.build_tree(prims, 1)
    kids = np.array([1.0, 2.0, 4.0, 8.0, 16.0, 32.0, 64.0, 128.0])
    # a depth-2 tree whose one level-1 node has 8 leaf children, all prune-marked
    s = np.zeros(8)
    sm = np.zeros(8, np.uint8)
    sm[0] = 1
    t2, _, s2, _, _ = oracle.refine(t, s, np.zeros((8, 3, 1)), np.zeros(8, np.uint8), sm, 8)
    child_leaves = -1 - t2["child"][1]
    s2[child_leaves] = kids
    t3, lm, s3, _, cnt = oracle.refine(t2, s2, np.zeros((15, 3, 1)), np.ones(15, np.uint8),
                                       np.zeros(15, np.uint8), 8)
    assert cnt["n_pruned_groups"] == 1
    merged = s3[lm < 0][0]
    assert merged == kids.sum() / G["octree_degree_M"]


def test_workload_shapes_follow_the_paper():
    sc, cams = si.config_nerf_synthetic(100)
    assert 2 ** sc.max_depth == G["grid_resolution"]
    assert sc.n_coeffs == G["sh_components_synthetic"]
    assert len(cams) == G["train_views_synthetic"]
    assert (cams[0].width, cams[0].height) == (G["image_width_synthetic"], G["image_height_synthetic"])
    _, tcams = si.config_tanks_temples(3)
    assert (tcams[0].width, tcams[0].height) == (G["image_width_tanks"], G["image_height_tanks"])
    # the degree-1 basis has the 4 components of the paper's Tanks & Temples models
    assert len(oracle.sh_basis(1, [0.0, 0.0, 1.0])) == G["sh_components_tanks"]


def test_rmsprop_defaults_are_the_paper_learning_rates():
    from paper_2307_15333_gb300 import dot
    o = dot.rmsprop_opts()
    assert o.lr_sigma == pytest.approx(G["lr_sigma"]) and o.lr_sh == pytest.approx(G["lr_color"])
