"""pbdr_neighbors_noalloc: the neighbour stage for callers that may not
allocate device memory themselves (a host framework that owns all device
memory through its own pool, or a control loop whose latency budget an
allocation could break).  Called through the C ABI on caller-owned device
buffers, it must give exactly what the regular entry points
(pbdr_build_neighbors + pbdr_read_neighbors) give: bit-identical sorted keys,
sorted ids and neighbour lists.  Two calls run back to back, because every
call shares one static scratch array that keeps the previous call's contents.
"""
import numpy as np
import pytest

from paper_2603_14634_gb300 import scenes

pytestmark = pytest.mark.gpu


def _scene(seed, num_bodies, squeeze):
    sc = scenes.random_bodies_scene(seed=seed, num_bodies=num_bodies)
    sc.pos = (sc.pos * np.float32(squeeze)).astype(np.float32)
    return sc


def _regular(pbdr_lib, sc):
    with pbdr_lib.Context(0) as c:
        sid = c.create_scene(sc)
        c.build_neighbors(sid)
        return c.read_neighbors(sid)


def _noalloc(pbdr_lib, sc, cap=32):
    torch = pytest.importorskip("torch")
    n = sc.num_particles
    body = np.repeat(np.arange(sc.num_bodies, dtype=np.int32), np.diff(sc.body_off))
    dev = torch.device("cuda", 0)
    pos_d = torch.from_numpy(np.ascontiguousarray(sc.pos, np.float32)).to(dev)
    body_d = torch.from_numpy(body).to(dev)
    sk = torch.empty(n, dtype=torch.int32, device=dev)
    si = torch.empty(n, dtype=torch.int32, device=dev)
    cnt = torch.empty(n, dtype=torch.int32, device=dev)
    nbr = torch.full((cap, n), -1, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    pbdr_lib.pbdr_neighbors_noalloc(pos_d.data_ptr(), body_d.data_ptr(), n, sc.radius,
                                    sk.data_ptr(), si.data_ptr(), cnt.data_ptr(),
                                    nbr.data_ptr(), cap, None)
    torch.cuda.synchronize()
    cnt_h = cnt.cpu().numpy()
    nbr_h = nbr.cpu().numpy()
    assert (cnt_h <= cap).all()
    off = np.zeros(n + 1, np.int32)
    off[1:] = np.cumsum(cnt_h)
    idx = np.concatenate([nbr_h[:cnt_h[p], p] for p in range(n)]) if n else np.zeros(0, np.int32)
    return (sk.cpu().numpy().view(np.uint32), si.cpu().numpy().view(np.uint32), off,
            idx.astype(np.int32))


def test_noalloc_matches_regular_entry_points_twice(pbdr_lib):
    first = _scene(seed=1, num_bodies=40, squeeze=0.55)     # 5000 particles
    second = _scene(seed=2, num_bodies=9, squeeze=0.5)      # smaller: stale scratch beyond n
    for sc in (first, second):
        want = _regular(pbdr_lib, sc)
        got = _noalloc(pbdr_lib, sc)
        assert want[3].size > 50
        for w, g, name in zip(want, got, ("sorted_key", "sorted_id", "off", "idx")):
            np.testing.assert_array_equal(g, w, err_msg=name)


def test_noalloc_rejects_oversize(pbdr_lib):
    with pytest.raises(pbdr_lib.PbdrError) as e:
        pbdr_lib.pbdr_neighbors_noalloc(0, 0, 65537, 0.05, 0, 0, 0, 0, 32, None)
    assert e.value.code == -1
    assert "65536" in str(e.value)
