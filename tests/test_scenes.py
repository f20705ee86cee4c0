"""The seeded input recipes (CPU): the batched workload's size draws and
totals, the placement guarantee (no two particles of different bodies closer
than 2r), rigid lattices with rigid velocity fields in the stated ranges, and
the cube-drop start.  These pin the inputs every parity test and the bench
use, so a change of a generator cannot pass unnoticed."""
import math

import numpy as np
import pytest

from paper_2603_14634_gb300 import scenes


def _size_draws(child):
    """n_b and the lattice sizes a batch scene draws first from its stream."""
    rng = np.random.default_rng(child)
    nb = int(math.floor(math.exp(rng.random() * math.log(33))))
    nb = min(max(nb, 1), 32)
    return [scenes.BATCH_LATTICE_SIZES[i] for i in rng.integers(0, 4, nb)]


def test_batched_workload_totals():
    """4096 scenes from seed 0: 5 033 654 particles in 36 076 bodies (the
    figures the benchmark reports); body counts log-uniform in [1, 32] with
    mean (32 ln 33 - ln 32!)/ln 33 = 8.675."""
    kids = np.random.SeedSequence(0).spawn(4096)
    draws = [_size_draws(k) for k in kids]
    assert sum(len(d) for d in draws) == 36076
    assert sum(sum(n ** 3 for n in d) for d in draws) == 5033654
    counts = np.array([len(d) for d in draws])
    assert counts.min() == 1 and counts.max() == 32
    mean = (32 * math.log(33) - math.lgamma(33)) / math.log(33)
    assert abs(mean - 8.675) < 1e-3
    assert abs(counts.mean() - mean) < 4 * counts.std() / math.sqrt(counts.size)


def test_batch_scene_matches_its_size_draws():
    kids = np.random.SeedSequence(0).spawn(4096)
    for k in (0, 1, 2, 1000, 4095):
        sc = scenes.batch_scene(np.random.default_rng(kids[k]))
        sizes = np.diff(sc.body_off)
        assert list(sizes) == [n ** 3 for n in _size_draws(kids[k])]
        assert sc.iterations == 10 and sc.friction == 0.5 and abs(sc.dt - 1 / 240) < 1e-12


def _rigid_checks(sc, vmax=1.0, wmax=2.0):
    r = sc.radius
    pos = sc.pos.astype(np.float64)
    vel = sc.vel.astype(np.float64)
    body = np.repeat(np.arange(sc.num_bodies), np.diff(sc.body_off))
    # no two particles of different bodies closer than 2r (brute force)
    d2 = ((pos[:, None, :] - pos[None, :, :]) ** 2).sum(-1)
    other = body[:, None] != body[None, :]
    assert d2[other].min() >= (2 * r) ** 2 * (1 - 1e-5)
    for b in range(sc.num_bodies):
        s = slice(sc.body_off[b], sc.body_off[b + 1])
        p, v = pos[s], vel[s]
        n = round(p.shape[0] ** (1 / 3))
        assert n ** 3 == p.shape[0]
        # a rigid n^3 lattice of spacing 2r: pairwise distances of the lattice
        ref = scenes.lattice_cube(n, 2 * r)
        dp = np.sort(np.linalg.norm(p[:, None] - p[None], axis=-1).ravel())
        dr = np.sort(np.linalg.norm(ref[:, None] - ref[None], axis=-1).ravel())
        assert np.abs(dp - dr).max() < 1e-5
        # rigid velocity field v + w x (x - c) with |v_i| <= vmax, |w_i| <= wmax
        c = p.mean(0)
        A = np.zeros((3 * p.shape[0], 6))
        for i, e in enumerate(p - c):
            A[3 * i:3 * i + 3, :3] = np.eye(3)
            A[3 * i:3 * i + 3, 3:] = -np.array([[0, -e[2], e[1]], [e[2], 0, -e[0]], [-e[1], e[0], 0]])
        sol, *_ = np.linalg.lstsq(A, v.ravel(), rcond=None)
        assert np.abs(A @ sol - v.ravel()).max() < 1e-5
        assert np.all(np.abs(sol[:3]) <= vmax + 1e-5) and np.all(np.abs(sol[3:]) <= wmax + 1e-5)
        # above the ground plane
        assert p[:, 2].min() >= r - 1e-6


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_bodies_placement_and_rigid_velocities(seed):
    sc = scenes.random_bodies_scene(seed=seed, num_bodies=24)
    assert sc.num_particles == 24 * 125
    _rigid_checks(sc)


def test_batch_scenes_placement():
    kids = np.random.SeedSequence(7).spawn(6)
    for k in kids:
        _rigid_checks(scenes.batch_scene(np.random.default_rng(k)))


def test_cube_drop_start():
    sc = scenes.cube_drop()
    assert sc.num_particles == 64 and sc.num_bodies == 1
    assert abs(float(sc.pos[:, 2].min()) - sc.radius - 1.0) < 1e-6   # bottom surface 1 m up
    assert np.all(sc.vel == 0) and sc.iterations == 10 and sc.friction == 0.5
    assert np.allclose(sc.inv_mass, 1.0)
