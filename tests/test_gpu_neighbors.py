"""GPU neighbour stage vs the oracle: sorted cell keys, sorted particle ids
and neighbour lists must be bit-identical on identical FP32 positions."""
import numpy as np
import pytest

from paper_2603_14634_gb300 import scenes

pytestmark = pytest.mark.gpu


def _scene_from(pos, body_sizes):
    pos = np.ascontiguousarray(pos, np.float32)
    off = np.zeros(len(body_sizes) + 1, np.int32)
    off[1:] = np.cumsum(body_sizes)
    assert off[-1] == pos.shape[0]
    return scenes.Scene(pos=pos, vel=np.zeros_like(pos), inv_mass=np.ones(pos.shape[0], np.float32),
                        body_off=off)


def _check_scene(ctx, orc, sid, sc):
    sk, si, off, idx = ctx.read_neighbors(sid)
    ok_k, ok_i = orc.sorted_keys(sc.pos, sc.radius)
    np.testing.assert_array_equal(sk, ok_k)
    np.testing.assert_array_equal(si, ok_i)
    o_off, o_idx = orc.neighbors(sc.pos, orc.body_index(sc.body_off), sc.radius, "brute")
    np.testing.assert_array_equal(off, o_off)
    np.testing.assert_array_equal(idx, o_idx)
    return o_idx.size


@pytest.mark.parametrize("n_bodies,per_body", [(1, 1), (2, 1), (31, 1), (33, 1), (40, 50),
                                               (97, 43), (3, 1366)])
def test_random_positions_bit_exact(ctx, orc, n_bodies, per_body):
    rng = np.random.default_rng(n_bodies * 1000 + per_body)
    n = n_bodies * per_body
    box = 0.08 * max(n, 8) ** (1 / 3)
    sc = _scene_from(rng.random((n, 3)) * box, [per_body] * n_bodies)
    sid = ctx.create_scene(sc)
    ctx.build_neighbors(sid)
    _check_scene(ctx, orc, sid, sc)


def test_lattice_bodies_bit_exact(ctx, orc):
    sc = scenes.random_bodies_scene(seed=1, num_bodies=20)
    sc.pos = (sc.pos * np.float32(0.55)).astype(np.float32)   # push bodies into each other
    sid = ctx.create_scene(sc)
    ctx.build_neighbors(sid)
    assert _check_scene(ctx, orc, sid, sc) > 100


def test_boundary_pairs_bit_exact(ctx, orc):
    Rn, Rn2, h, inv_h = orc.nbr_constants(0.05)
    pts = []
    for k, base in enumerate((0.0, float(h), 3 * float(h), -2 * float(h), 7.5 * float(h))):
        for j, gap in enumerate((np.nextafter(Rn, np.float32(0)), Rn, np.nextafter(Rn, np.float32(1)))):
            p = np.array([base, 0.37 + 1.0 * (3 * k + j), 0.11], np.float32)
            q = p.copy()
            q[0] = np.float32(p[0] + gap)
            pts += [p, q]
    sc = _scene_from(np.stack(pts), [1] * len(pts))
    sid = ctx.create_scene(sc)
    ctx.build_neighbors(sid)
    _check_scene(ctx, orc, sid, sc)


def test_batched_scenes_local_numbering(ctx, orc):
    rng = np.random.default_rng(7)
    scs = [scenes.batch_scene(rng) for _ in range(6)]
    for sc in scs:   # squeeze to create contacts
        sc.pos = (sc.pos * np.float32(0.6)).astype(np.float32)
    ids = [ctx.create_scene(sc) for sc in scs]
    ctx.build_neighbors(ids)
    for sid, sc in zip(ids, scs):
        _check_scene(ctx, orc, sid, sc)
    # a subset in another order gives the same per-scene result
    ctx.build_neighbors([ids[4], ids[1]])
    _check_scene(ctx, orc, ids[4], scs[4])
    _check_scene(ctx, orc, ids[1], scs[1])


def test_predicted_positions_feed_the_lists(ctx, orc):
    """After a substep the lists are those of x~ = x + dt (v + dt g)."""
    sc = scenes.random_bodies_scene(seed=2, num_bodies=10)
    sc.pos = (sc.pos * np.float32(0.5)).astype(np.float32)
    sid = ctx.create_scene(sc)
    ctx.step(sid, 1)
    resident = ctx.path_name == "resident"
    sk, si, off, idx = ctx.read_neighbors(sid, lists_only=resident)
    if not resident:
        # sorted ids are a permutation, keys ascending
        assert sorted(si.tolist()) == list(range(sc.num_particles))
        assert np.all(np.diff(sk.astype(np.int64)) >= 0)
    body = orc.body_index(sc.body_off)
    for p in range(sc.num_particles):
        lst = idx[off[p]:off[p + 1]]
        assert np.all(np.diff(lst) > 0)
        assert np.all(body[lst] != body[p])


def test_resident_lists_equal_oracle_on_exact_prediction(ctx, orc):
    """With zero velocity and zero gravity x~ = x exactly, so the lists the
    substep builds (either form) are the oracle's lists of the given
    positions, bit for bit."""
    rng = np.random.default_rng(3)
    scs = [scenes.batch_scene(rng) for _ in range(5)]
    for sc in scs:
        sc.pos = (sc.pos * np.float32(0.6)).astype(np.float32)
        sc.vel[:] = 0
        sc.gravity = (0.0, 0.0, 0.0)
        sc.plane = (0.0, 0.0, 1.0, -100.0)
    ids = [ctx.create_scene(s) for s in scs]
    ctx.step(ids, 1)
    for sid, sc in zip(ids, scs):
        _, _, off, idx = ctx.read_neighbors(sid, lists_only=True)
        o_off, o_idx = orc.neighbors(sc.pos, orc.body_index(sc.body_off), sc.radius, "brute")
        np.testing.assert_array_equal(off, o_off)
        np.testing.assert_array_equal(idx, o_idx)


def test_overflow_sets_error_bit(ctx, pbdr_lib):
    """40 one-particle bodies inside one small ball: 39 neighbours each,
    more than the 32-slot lists hold."""
    rng = np.random.default_rng(0)
    pos = (rng.random((40, 3)) * 0.01 + [0, 0, 1.0]).astype(np.float32)
    sc = _scene_from(pos, [1] * 40)
    sid = ctx.create_scene(sc)
    ctx.step(sid, 1)
    _, _, err = ctx.read_state(sid)
    assert err & pbdr_lib.EBIT_NBR_OVERFLOW
    _, _, err = ctx.read_state(sid)      # bits clear on read
    assert err == 0



def test_lists_exact_with_rotated_bodies(ctx, orc):
    """The scene-resident kernel bounds bodies by boxes in the frame of their
    last shape-matching rotation.  Spin the bodies first so those frames are
    not the rest frame, then zero the velocities (x~ = x exactly) and compare
    the lists of the next substep with the O(N^2) definition."""
    rng = np.random.default_rng(21)
    scs = [scenes.batch_scene(rng) for _ in range(4)]
    ids = []
    for sc in scs:
        sc.pos = (sc.pos * np.float32(0.7)).astype(np.float32)
        sc.gravity = (0.0, 0.0, 0.0)
        sc.plane = (0.0, 0.0, 1.0, -100.0)
        ids.append(ctx.create_scene(sc))
    ctx.step(ids, 40)
    written = {}
    for sid in ids:
        pos, _, _ = ctx.read_state(sid)
        ctx.write_state(sid, pos, np.zeros_like(pos))
        written[sid] = pos
    ctx.step(ids, 1)
    total = 0
    for sid, sc in zip(ids, scs):
        _, _, off, idx = ctx.read_neighbors(sid, lists_only=True)
        o_off, o_idx = orc.neighbors(written[sid], orc.body_index(sc.body_off), sc.radius, "brute")
        np.testing.assert_array_equal(off, o_off)
        np.testing.assert_array_equal(idx, o_idx)
        total += idx.size
    assert total > 0
