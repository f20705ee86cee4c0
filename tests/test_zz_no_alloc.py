"""pbdr_neighbors_noalloc: the neighbour stage for callers that may not
allocate device memory themselves (a host framework that owns all device
memory through its own pool, or a control loop whose latency budget an
allocation could break).  Called through the C ABI on caller-owned device
buffers, it must give exactly what the regular entry points
(pbdr_build_neighbors + pbdr_read_neighbors) and the oracle give:
bit-identical sorted keys, sorted ids and neighbour lists.  Calls run back to
back, because every call shares one static scratch array that keeps the
previous call's contents; the largest case fills that array to its stated
limit of 65536 particles.
"""
import numpy as np
import pytest

from paper_2603_14634_gb300 import scenes

pytestmark = pytest.mark.gpu

LIMIT = 65536   # particles per call, as include/pbdr.h states


def _scene(seed, num_bodies, squeeze):
    sc = scenes.random_bodies_scene(seed=seed, num_bodies=num_bodies)
    sc.pos = (sc.pos * np.float32(squeeze)).astype(np.float32)
    return sc


def _body(sc):
    return np.repeat(np.arange(sc.num_bodies, dtype=np.int32), np.diff(sc.body_off))


def _regular(pbdr_lib, sc):
    with pbdr_lib.Context(0) as c:
        sid = c.create_scene(sc)
        c.build_neighbors(sid)
        return c.read_neighbors(sid)


def _oracle(orc, pos, body, radius, method):
    sk, si = orc.sorted_keys(pos, radius)
    off, idx = orc.neighbors(pos, body, radius, method)
    return sk, si, off, idx


def _noalloc_raw(pbdr_lib, pos, body, radius, cap):
    """(sorted keys, sorted ids, full counts, [cap, n] slots) of one call."""
    torch = pytest.importorskip("torch")
    n = pos.shape[0]
    dev = torch.device("cuda", 0)
    pos_d = torch.from_numpy(np.ascontiguousarray(pos, np.float32)).to(dev)
    body_d = torch.from_numpy(np.ascontiguousarray(body, np.int32)).to(dev)
    sk = torch.empty(n, dtype=torch.int32, device=dev)
    si = torch.empty(n, dtype=torch.int32, device=dev)
    cnt = torch.empty(n, dtype=torch.int32, device=dev)
    nbr = torch.full((cap, n), -1, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    pbdr_lib.pbdr_neighbors_noalloc(pos_d.data_ptr(), body_d.data_ptr(), n, radius,
                                    sk.data_ptr(), si.data_ptr(), cnt.data_ptr(),
                                    nbr.data_ptr(), cap, None)
    torch.cuda.synchronize()
    return (sk.cpu().numpy().view(np.uint32), si.cpu().numpy().view(np.uint32),
            cnt.cpu().numpy(), nbr.cpu().numpy())


def _noalloc(pbdr_lib, pos, body, radius, cap=32):
    sk, si, cnt_h, nbr_h = _noalloc_raw(pbdr_lib, pos, body, radius, cap)
    n = pos.shape[0]
    assert (cnt_h <= cap).all()
    off = np.zeros(n + 1, np.int32)
    off[1:] = np.cumsum(cnt_h)
    idx = np.concatenate([nbr_h[:cnt_h[p], p] for p in range(n)]) if n else np.zeros(0, np.int32)
    return sk, si, off, idx.astype(np.int32)


def _assert_same(got, want, label):
    for w, g, name in zip(want, got, ("sorted_key", "sorted_id", "off", "idx")):
        np.testing.assert_array_equal(g, w, err_msg=f"{label}: {name}")


def test_noalloc_matches_regular_entry_points_and_oracle_twice(pbdr_lib, orc):
    first = _scene(seed=1, num_bodies=40, squeeze=0.55)     # 5000 particles
    second = _scene(seed=2, num_bodies=9, squeeze=0.5)      # smaller: stale scratch beyond n
    for sc in (first, second):
        pos, body = np.ascontiguousarray(sc.pos, np.float32), _body(sc)
        got = _noalloc(pbdr_lib, pos, body, sc.radius)
        want = _regular(pbdr_lib, sc)
        assert want[3].size > 50
        _assert_same(got, want, "regular entry points")
        _assert_same(got, _oracle(orc, pos, body, sc.radius, "brute"), "oracle, O(N^2)")


def _blocks_at_limit(seed=5):
    """65536 particles: 1024 bodies of 4^3 (spacing 0.1 m) on a 16 x 8 x 8
    grid of 0.4 m pitch, each shifted by up to 1 cm, so that the faces of
    neighbouring bodies come within the neighbour radius of each other."""
    rng = np.random.default_rng(seed)
    g = np.arange(4) * 0.1
    cube = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    cells = np.stack(np.meshgrid(np.arange(16), np.arange(8), np.arange(8), indexing="ij"), -1).reshape(-1, 3)
    shift = rng.uniform(-0.01, 0.01, size=(cells.shape[0], 3))
    pos = (cells[:, None, :] * 0.4 + shift[:, None, :] + cube[None, :, :] + 0.05).reshape(-1, 3)
    body = np.repeat(np.arange(cells.shape[0], dtype=np.int32), cube.shape[0])
    return pos.astype(np.float32), body


def test_noalloc_at_its_particle_limit_matches_oracle(pbdr_lib, orc):
    pos, body = _blocks_at_limit()
    assert pos.shape[0] == LIMIT
    got = _noalloc(pbdr_lib, pos, body, 0.05)
    want = _oracle(orc, pos, body, 0.05, "grid")
    assert want[3].size > 10_000
    _assert_same(got, want, f"n = {LIMIT}")


def test_noalloc_cut_lists_keep_full_counts(pbdr_lib, orc):
    """With cap = 2 on a dense scene, nbr_cnt holds the full count and the
    two slots hold the two lowest neighbour indices."""
    sc = _scene(seed=3, num_bodies=30, squeeze=0.5)
    pos, body = np.ascontiguousarray(sc.pos, np.float32), _body(sc)
    cap = 2
    sk, si, cnt, nbr = _noalloc_raw(pbdr_lib, pos, body, sc.radius, cap)
    osk, osi, off, idx = _oracle(orc, pos, body, sc.radius, "brute")
    np.testing.assert_array_equal(sk, osk)
    np.testing.assert_array_equal(si, osi)
    full = np.diff(off)
    np.testing.assert_array_equal(cnt, full)
    assert (cnt > cap).sum() > 20
    for p in range(pos.shape[0]):
        k = min(full[p], cap)
        np.testing.assert_array_equal(nbr[:k, p], idx[off[p]:off[p] + k], err_msg=f"particle {p}")


def test_noalloc_rejects_oversize(pbdr_lib):
    with pytest.raises(pbdr_lib.PbdrError) as e:
        pbdr_lib.pbdr_neighbors_noalloc(0, 0, LIMIT + 1, 0.05, 0, 0, 0, 0, 32, None)
    assert e.value.code == -1
    assert str(LIMIT) in str(e.value)
