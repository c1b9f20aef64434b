"""The host-side camera schedule (dot_camera_order) -- no GPU: a permutation that starts at
camera 0 and always moves to the nearest camera not yet visited."""
import numpy as np

import seeded_inputs as si


def test_camera_order_is_a_greedy_nearest_neighbour_chain():
    from paper_2307_15333_gb300 import dot
    _, cams = si.config_nerf_synthetic(100)
    recs = np.stack([c.packed() for c in cams])
    order = dot.dot_camera_order(recs)
    assert sorted(order.tolist()) == list(range(100)) and order[0] == 0
    pos = recs[:, [3, 7, 11]].astype(np.float64)
    left = set(range(100)) - {0}
    for a, b in zip(order[:-1], order[1:]):
        d = ((pos[list(left)] - pos[a]) ** 2).sum(axis=1)
        assert ((pos[b] - pos[a]) ** 2).sum() == d.min()
        left.remove(b)


def test_camera_order_small_cases():
    from paper_2307_15333_gb300 import dot
    assert dot.dot_camera_order(np.zeros((0, 18), np.float32)).tolist() == []
    one = np.stack([si.pinhole((0, 0, 3), 8, 8, 10.0).packed()])
    assert dot.dot_camera_order(one).tolist() == [0]
    line = np.stack([si.pinhole((x, 0.5, 3), 8, 8, 10.0).packed() for x in (0.0, 5.0, 1.0, 4.0, 2.0)])
    assert dot.dot_camera_order(line).tolist() == [0, 2, 4, 3, 1]
