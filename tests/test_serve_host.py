"""Host-side logic of the serving loop (no GPU): output pool, slot-table packing, traces."""
import numpy as np

from paper_2307_15333_gb300 import serve


def test_pool_first_fit_and_coalescing():
    p = serve.OutputPool(1024, align=64)
    a = p.alloc(100)          # rounds to 128
    b = p.alloc(64)
    c = p.alloc(800)          # does not fit (1024 - 192 = 832, 800 rounds to 832): fits exactly
    assert (a, b, c) == (0, 128, 192)
    assert p.alloc(1) == -1
    p.release(b, 64)
    assert p.alloc(64) == 128
    p.release(a, 100)
    p.release(128, 64)
    p.release(c, 800)
    assert p.free == [(0, 1024)] and p.free_floats == 1024


def test_pack_table_layout():
    cams = [np.arange(18, dtype=np.float32) + i for i in range(3)]
    for i, c in enumerate(cams):
        c[16:18] = np.array([100 + 16 * i, 50], np.int32).view(np.float32)
    reqs = [serve.Request(i, i % 2, 100 + 16 * i, 50, cams[i], 0.0, offset=1000 * i) for i in range(3)]
    buf = serve.pack_table(reqs, pool_base_ptr=1 << 20, max_slots=4)
    assert buf.size == 16 + 96 * 4
    assert buf[0:4].view(np.int32)[0] == 3
    tiles = [r.tiles for r in reqs]
    assert buf[8:16].view(np.int64)[0] == sum(tiles)
    begin = 0
    for i, r in enumerate(reqs):
        rec = buf[16 + 96 * i: 16 + 96 * (i + 1)]
        np.testing.assert_array_equal(rec[0:72].view(np.float32), cams[i])
        assert rec[72:76].view(np.int32)[0] == r.tree
        assert rec[80:88].view(np.int64)[0] == begin
        assert rec[88:96].view(np.uint64)[0] == (1 << 20) + 4 * r.offset
        begin += tiles[i]
    assert reqs[0].tiles == 7 * 7          # ceil(100 / 16) x ceil(50 / 8)


def test_poisson_trace_is_seeded_and_has_the_rate():
    def poses(rng, tree, w, h):
        return np.zeros(18, np.float32)
    res = [(256, 256), (512, 512)]
    a = serve.poisson_trace(4000, 200.0, 3, res, poses, seed=1)
    b = serve.poisson_trace(4000, 200.0, 3, res, poses, seed=1)
    assert [r.arrival for r in a] == [r.arrival for r in b]
    rate = len(a) / a[-1].arrival
    assert 190 < rate < 210
    assert {r.tree for r in a} == {0, 1, 2}


def test_slot_groups_and_per_group_tree_index():
    """Trees that differ in storage, SH degree or compression go to different slot launches; a
    request's slot records its tree's index within its own group."""
    class T:
        def __init__(self, storage, deg, bits=0):
            self.storage, self.sh_degree, self.palette_bits = storage, deg, bits
    trees = [T(0, 1), T(1, 3), T(0, 1), T(1, 3), T(1, 3, 16), T(2, 3)]
    groups = serve.slot_groups(trees)
    assert groups == [[0, 2], [1, 3], [4], [5]]
    index = {t: j for g in groups for j, t in enumerate(g)}
    cam = np.zeros(18, np.float32)
    cam[16:18] = np.array([32, 16], np.int32).view(np.float32)
    reqs = [serve.Request(i, t, 32, 16, cam, 0.0, offset=0) for i, t in enumerate([2, 0])]
    buf = serve.pack_table(reqs, 0, 2, index)
    assert [buf[16 + 96 * i + 72: 16 + 96 * i + 76].view(np.int32)[0] for i in range(2)] == [1, 0]
