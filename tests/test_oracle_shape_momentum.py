"""Pins of the oracle's shape-matching rotation, inertia tensor and momentum
enforcement (CPU only).

Shape matching pulls each particle to the goal of the least-squares optimal
rigid transformation from the rest pose (Sec. III-C, Mueller et al. 2005):
the rotation is the proper rotation maximising tr(R^T A).  The momentum
constraint (Sec. III-C, Eqs. lin_momentum and ang_momentum) solves
sum m (v_asm + dv) = P_bsm and L_asm - L_bsm = I w with
I = sum m (|r|^2 I3 - r r^T).
"""
import numpy as np
import pytest


def _rand_rot(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def _kabsch_numpy(A):
    """textbook SVD solution of max tr(R^T A) over SO(3) with numpy's SVD"""
    U, S, Vt = np.linalg.svd(A)
    d = np.sign(np.linalg.det(U @ Vt))
    return U @ np.diag([1.0, 1.0, d]) @ Vt


@pytest.mark.parametrize("seed", range(20))
def test_polar_matches_library_svd(orc, seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(3, 3))
    R = orc.polar_rotation(A)
    np.testing.assert_allclose(R, _kabsch_numpy(A), atol=1e-10)
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-12)
    assert abs(np.linalg.det(R) - 1) < 1e-12


@pytest.mark.parametrize("seed", range(10))
def test_polar_optimality_condition(orc, seed):
    """R^T A is symmetric, and positive semi-definite when det A > 0"""
    rng = np.random.default_rng(100 + seed)
    A = rng.normal(size=(3, 3))
    if np.linalg.det(A) < 0:
        A[:, 0] *= -1
    S = orc.polar_rotation(A).T @ A
    np.testing.assert_allclose(S, S.T, atol=1e-10)
    assert np.linalg.eigvalsh(0.5 * (S + S.T)).min() > -1e-10


def test_polar_recovers_rigid_rotation(orc):
    rng = np.random.default_rng(7)
    for _ in range(10):
        R0 = _rand_rot(rng)
        M = rng.normal(size=(3, 3))
        S = M @ M.T + 0.5 * np.eye(3)          # SPD stretch
        np.testing.assert_allclose(orc.polar_rotation(R0 @ S), R0, atol=1e-10)


def test_polar_rank_deficient_keeps_previous(orc):
    rng = np.random.default_rng(9)
    Rprev = _rand_rot(rng)
    A = np.outer(rng.normal(size=3), rng.normal(size=3))     # rank 1
    np.testing.assert_array_equal(orc.polar_rotation(A, Rprev), Rprev)
    np.testing.assert_array_equal(orc.polar_rotation(np.zeros((3, 3)), Rprev), Rprev)
    # rank 2 (coplanar body) is still unique
    A2 = _rand_rot(rng) @ np.diag([2.0, 1.0, 0.0]) @ _rand_rot(rng)
    np.testing.assert_allclose(orc.polar_rotation(A2), _kabsch_numpy(A2), atol=1e-10)


@pytest.mark.parametrize("n", [3, 4, 5, 7])
def test_cube_inertia_closed_form(orc, n):
    """n^3 lattice, spacing s, particle mass m: sum over one axis of the
    squared offsets is n^2 * s^2 * n (n^2 - 1)/12 (Faulhaber), so
    I = 2 m n^3 s^2 (n^2 - 1)/12 * I3."""
    from paper_2603_14634_gb300.scenes import lattice_cube
    s, m = 0.1, 0.25
    x = lattice_cube(n, s) + np.array([0.3, -1.2, 2.0])
    I = orc.body_inertia(x, np.full(n ** 3, m), x.mean(0))
    expect = 2 * m * n ** 3 * s * s * (n * n - 1) / 12.0
    np.testing.assert_allclose(I, expect * np.eye(3), atol=1e-13)


def _momenta(m, x, v):
    c = (m[:, None] * x).sum(0) / m.sum()
    P = (m[:, None] * v).sum(0)
    L = np.cross(x - c, m[:, None] * v).sum(0)
    return c, P, L


@pytest.mark.parametrize("seed", range(8))
def test_momentum_correction_restores_pre_shape_matching_momenta(orc, seed):
    rng = np.random.default_rng(seed)
    n = 40
    m = rng.uniform(0.5, 2.0, n)
    xb = rng.normal(size=(n, 3))
    vb = rng.normal(size=(n, 3))
    xa = xb + 0.05 * rng.normal(size=(n, 3))
    va = vb + 0.3 * rng.normal(size=(n, 3))
    dt = 1 / 240
    x, v = orc.enforce_momentum(m, xb, vb, xa, va, dt)
    _, Pb, Lb = _momenta(m, xb, vb)
    ca, _, _ = _momenta(m, xa, va)
    # the corrected velocities carry P_bsm and, about c_asm with the
    # post-shape-matching positions, L_bsm
    np.testing.assert_allclose((m[:, None] * v).sum(0), Pb, atol=1e-12)
    np.testing.assert_allclose(np.cross(xa - ca, m[:, None] * v).sum(0), Lb, atol=1e-11)
    # the correction is a rigid velocity field and positions move by corr*dt
    corr = v - va
    np.testing.assert_allclose(x - xa, corr * dt, atol=1e-14)
    # rigid: corr_p = dv - w x r_p  ->  differences are w x (r_q - r_p)
    A = np.zeros((3 * n, 6))
    r = xa - ca
    for p in range(n):
        A[3 * p:3 * p + 3, :3] = np.eye(3)
        A[3 * p:3 * p + 3, 3:] = np.array([[0, r[p, 2], -r[p, 1]],
                                           [-r[p, 2], 0, r[p, 0]],
                                           [r[p, 1], -r[p, 0], 0]])
    sol, res, *_ = np.linalg.lstsq(A, corr.ravel(), rcond=None)
    assert np.abs(A @ sol - corr.ravel()).max() < 1e-12


def test_momentum_flags(orc):
    rng = np.random.default_rng(1)
    n = 20
    m = np.ones(n)
    xb = rng.normal(size=(n, 3))
    vb = rng.normal(size=(n, 3))
    xa = xb + 0.1 * rng.normal(size=(n, 3))
    va = vb + 0.5 * rng.normal(size=(n, 3))
    _, Pb, Lb = _momenta(m, xb, vb)
    ca, Pa, La = _momenta(m, xa, va)
    x, v = orc.enforce_momentum(m, xb, vb, xa, va, 0.01, orc.NO_LINMOM)
    np.testing.assert_allclose(v.sum(0), Pa, atol=1e-12)      # P untouched
    np.testing.assert_allclose(np.cross(xa - ca, v).sum(0), Lb, atol=1e-11)
    x, v = orc.enforce_momentum(m, xb, vb, xa, va, 0.01, orc.NO_ANGMOM)
    np.testing.assert_allclose(v.sum(0), Pb, atol=1e-12)
    np.testing.assert_allclose(v - va, np.broadcast_to((Pb - Pa) / n, v.shape), atol=1e-13)
    x, v = orc.enforce_momentum(m, xb, vb, xa, va, 0.01, orc.NO_ANGMOM | orc.NO_LINMOM)
    np.testing.assert_array_equal(v, va)
    np.testing.assert_array_equal(x, xa)


def test_single_particle_body(orc):
    m = np.array([2.0])
    x, v = orc.enforce_momentum(m, [[0, 0, 1.0]], [[1.0, 0, 0]], [[0, 0, 1.0]],
                                [[0.5, 0, 0]], 0.1)
    np.testing.assert_allclose(v, [[1.0, 0, 0]])
    np.testing.assert_allclose(x, [[0.05, 0, 1.0]])
