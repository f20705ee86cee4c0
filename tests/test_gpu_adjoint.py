"""Reverse-mode adjoint of the substep on the GPU (pbdr_adjoint): the
dot-product identity against the forward-mode tangents on random
per-particle directions (contacts between bodies included), the oracle's
central differences, free-flight closed forms, checkpoint invariance and the
primal it leaves behind."""
import numpy as np
import pytest

from fd_oracle import mu_fd, rigid_fd_jacobian, sliding_grid
from paper_2603_14634_gb300 import diff, scenes

pytestmark = pytest.mark.gpu


def _contact_scene(seed):
    """Bodies pushed into each other: pair contacts with friction active."""
    sc = scenes.random_bodies_scene(seed=seed, num_bodies=8)
    sc.pos = (sc.pos * np.float32(0.75)).astype(np.float32)
    return sc


@pytest.mark.parametrize("which", ["sliding", "contacts"])
def test_dot_product_identity_with_tangents(pbdr_lib, which):
    """<xbar_T, dX_T> + <vbar_T, dV_T> = <xbar_0, dX_0> + <vbar_0, dV_0> for
    random directions (dX_0, dV_0) and random final adjoints: the adjoint
    kernels are the transpose of the tangent kernels."""
    sc = sliding_grid(seed=2)[0] if which == "sliding" else _contact_scene(5)
    rng = np.random.default_rng(0)
    n, steps = sc.num_particles, 12
    dx0 = rng.standard_normal((n, 3)).astype(np.float32) * 1e-2
    dv0 = rng.standard_normal((n, 3)).astype(np.float32)
    xbT = rng.standard_normal((n, 3)).astype(np.float32)
    vbT = rng.standard_normal((n, 3)).astype(np.float32)
    with pbdr_lib.Context(0) as c:
        a = c.create_scene(sc)
        c.write_tangent(a, dx0, dv0)
        c.step_tangent(a, steps)
        dxT, dvT = c.read_tangent(a)
        pa, va, err_a = c.read_state(a)
        b = c.create_scene(sc)
        c.write_adjoint(b, xbT, vbT)
        c.adjoint(b, steps, 5)
        xb0, vb0 = c.read_adjoint(b)
        pb, vb, err_b = c.read_state(b)
    assert err_a == err_b == 0
    lhs = float((xbT.astype(np.float64) * dxT).sum() + (vbT.astype(np.float64) * dvT).sum())
    rhs = float((xb0.astype(np.float64) * dx0).sum() + (vb0.astype(np.float64) * dv0).sum())
    assert abs(lhs - rhs) <= 2e-4 * max(abs(lhs), abs(rhs)), (lhs, rhs)
    assert np.array_equal(pa, pb) and np.array_equal(va, vb)   # same primal trajectory


def test_rigid_gradient_matches_oracle(pbdr_lib, orc):
    sc, v, w = sliding_grid(seed=1)
    steps = 48
    wts = np.random.default_rng(1).standard_normal((sc.num_bodies, 3))
    with pbdr_lib.Context(0) as c:
        final, g = diff.com_gradient_reverse(c, sc, v, w, steps, wts, checkpoint_every=16)
    J_ref = rigid_fd_jacobian(orc, sc, v, w, steps)
    g_ref = (J_ref.T @ wts.reshape(-1)).reshape(sc.num_bodies, 6)
    assert np.abs(g - g_ref).max() <= 5e-3 * np.abs(g_ref).max()


def test_free_flight_gradient_closed_form(pbdr_lib):
    p = scenes.lattice_cube(4, 0.1)
    sc = scenes._assemble([p, p + np.array([1.0, 0.0, 0.0])], [np.zeros_like(p)] * 2, 1.0,
                          friction=0.3, dt=1 / 240, iterations=10, radius=0.05)
    sc.plane = (0.0, 0.0, 1.0, -100.0)
    v = np.array([[0.3, 0.1, 0.2], [-0.4, 0.0, 0.5]])
    w = np.array([[1.0, 0.0, 2.0], [0.0, -1.0, 0.5]])
    wts = np.array([[1.0, -2.0, 0.5], [0.3, 0.7, -1.1]])
    n = 40
    with pbdr_lib.Context(0) as c:
        _, g = diff.com_gradient_reverse(c, sc, v, w, n, wts, checkpoint_every=7)
    assert np.allclose(g[:, :3], n / 240 * wts, rtol=1e-5, atol=1e-6)
    assert np.abs(g[:, 3:]).max() < 1e-5


def test_checkpoint_interval_does_not_change_the_result(pbdr_lib):
    sc, v, w = sliding_grid(seed=7)
    wts = np.ones((sc.num_bodies, 3))
    res = []
    with pbdr_lib.Context(0) as c:
        for every in (1, 6, 25, 100):
            res.append(diff.com_gradient_reverse(c, sc, v, w, 25, wts, checkpoint_every=every))
    for f, g in res[1:]:
        assert np.array_equal(f, res[0][0]) and np.array_equal(g, res[0][1])


def test_autograd_reverse_mode(pbdr_lib, orc):
    torch = pytest.importorskip("torch")
    sc, v, w = sliding_grid(seed=6)
    steps = 36
    vt = torch.tensor(v, dtype=torch.float64, requires_grad=True)
    wt = torch.tensor(w, dtype=torch.float64, requires_grad=True)
    weights = torch.tensor(np.random.default_rng(0).standard_normal((sc.num_bodies, 3)))
    with pbdr_lib.Context(0) as c:
        out = diff.FinalCoM.apply(vt, wt, c, sc, steps, "reverse")
        (out * weights).sum().backward()
    J_ref = rigid_fd_jacobian(orc, sc, v, w, steps)
    g_ref = (J_ref.T @ weights.numpy().reshape(-1)).reshape(sc.num_bodies, 6)
    got = np.concatenate([vt.grad.numpy(), wt.grad.numpy()], 1)
    assert np.abs(got - g_ref).max() <= 5e-3 * np.abs(g_ref).max()


@pytest.mark.parametrize("flags", [scenes.CONTACT_AVG, scenes.NO_LINMOM, scenes.NO_ANGMOM,
                                   scenes.NO_LINMOM | scenes.NO_ANGMOM])
def test_dot_product_identity_with_flags(pbdr_lib, flags):
    """The transpose relation holds for the averaged-contact reading and the
    momentum ablations too."""
    sc = _contact_scene(9)
    sc.flags = flags
    rng = np.random.default_rng(3)
    n, steps = sc.num_particles, 8
    dx0 = rng.standard_normal((n, 3)).astype(np.float32) * 1e-2
    dv0 = rng.standard_normal((n, 3)).astype(np.float32)
    xbT = rng.standard_normal((n, 3)).astype(np.float32)
    vbT = rng.standard_normal((n, 3)).astype(np.float32)
    with pbdr_lib.Context(0) as c:
        a = c.create_scene(sc)
        c.write_tangent(a, dx0, dv0)
        c.step_tangent(a, steps)
        dxT, dvT = c.read_tangent(a)
        b = c.create_scene(sc)
        c.write_adjoint(b, xbT, vbT)
        c.adjoint(b, steps, 3)
        xb0, vb0 = c.read_adjoint(b)
    lhs = float((xbT.astype(np.float64) * dxT).sum() + (vbT.astype(np.float64) * dvT).sum())
    rhs = float((xb0.astype(np.float64) * dx0).sum() + (vb0.astype(np.float64) * dv0).sum())
    assert abs(lhs - rhs) <= 2e-4 * max(abs(lhs), abs(rhs)), (lhs, rhs)


def test_batched_adjoint_equals_separate_runs(pbdr_lib):
    """Scenes in one pbdr_adjoint call get the adjoints they get alone."""
    scs = [sliding_grid(seed=s)[0] for s in (11, 12, 13)]
    rng = np.random.default_rng(5)
    bars = [rng.standard_normal((s.num_particles, 3)).astype(np.float32) for s in scs]
    with pbdr_lib.Context(0) as c:
        ids = [c.create_scene(s) for s in scs]
        for sid, xb in zip(ids, bars):
            c.write_adjoint(sid, xb, None)
        c.adjoint(ids, 15, 4)
        together = [c.read_adjoint(sid) for sid in ids]
    for sc, xb, (x0, v0) in zip(scs, bars, together):
        with pbdr_lib.Context(0) as c:
            sid = c.create_scene(sc)
            c.write_adjoint(sid, xb, None)
            c.adjoint(sid, 15, 4)
            ax, av = c.read_adjoint(sid)
        assert np.array_equal(ax, x0) and np.array_equal(av, v0)


def test_friction_derivative_forward_reverse_and_oracle(pbdr_lib, orc):
    """d(final CoMs)/d(mu): forward tangent (seed dmu = 1) against the
    oracle's central differences; dL/dmu of the adjoint against the tangent
    column (L = weights . CoMs)."""
    sc, v, w = sliding_grid(seed=1)
    steps = 48
    wts = np.random.default_rng(2).standard_normal((sc.num_bodies, 3))
    with pbdr_lib.Context(0) as c:
        _, J = diff.final_com_and_jacobian(c, sc, v, w, steps, with_mu=True)
        _, g, mubar = diff.com_gradient_reverse(c, sc, v, w, steps, wts, checkpoint_every=16,
                                                with_mu=True)
    dmu = J[:, -1]
    ref = mu_fd(orc, scenes.Scene(**{**sc.__dict__}), steps)
    assert np.abs(dmu - ref).max() <= 5e-3 * np.abs(ref).max()
    want = float(wts.reshape(-1) @ dmu)
    assert abs(mubar - want) <= 1e-4 * max(abs(want), 1e-6), (mubar, want)
    assert np.abs(g - (J[:, :-1].T @ wts.reshape(-1)).reshape(sc.num_bodies, 6)).max() <= \
        1e-4 * np.abs(g).max()


def test_c5_gradient_matches_oracle_fd(pbdr_lib, orc):
    """The differentiation workload itself: 16 bodies of 5^3 sliding on the
    plane (mu = 0.5, K = 10), 200 substeps, checkpoints every 20.  The
    reverse-mode gradient of L = sum_b w_b . c_b(final) with respect to the
    initial rigid velocities (v_b, omega_b) and mu matches the oracle's FP64
    central differences (all 97 columns) within 0.5 % of the largest entry."""
    from fd_oracle import rigid_mu_fd_jacobian_parallel
    sc = diff.c5_scene(seed=0)
    B, steps = sc.num_bodies, 200
    v = np.stack([sc.vel[s].astype(np.float64).mean(0) for s in diff.body_slices(sc)])
    w = np.zeros_like(v)
    sc.vel = diff.rigid_velocity(sc, v, w).astype(np.float32)
    wts = np.random.default_rng(3).standard_normal((B, 3))
    J_ref = rigid_mu_fd_jacobian_parallel(sc, v, w, steps)
    with pbdr_lib.Context(0) as c:
        final, g, mubar = diff.com_gradient_reverse(c, sc, v, w, steps, wts, checkpoint_every=20,
                                                    with_mu=True)
    g_ref = (J_ref.T @ wts.reshape(-1))
    got = np.concatenate([g.reshape(-1), [mubar]])
    scale = np.abs(g_ref).max()
    assert np.abs(got - g_ref).max() <= 5e-3 * scale, (np.abs(got - g_ref).max(), scale)
    final_ref = diff.body_coms(sc, orc.OracleScene(sc).substep(steps).x)
    assert np.abs(final - final_ref).max() <= 1e-4
