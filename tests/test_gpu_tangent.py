"""Forward-mode tangents of the substep on the GPU (pbdr_step_tangent)
against the FP64 oracle's central differences, closed forms and algebraic
properties; the autograd wrapper's backward against the same reference."""
import numpy as np
import pytest

from fd_oracle import rigid_fd_jacobian, sliding_grid
from paper_2603_14634_gb300 import diff, scenes

pytestmark = pytest.mark.gpu


def _box(v, w, plane_d=-100.0, n=4, mu=0.3):
    p = scenes.lattice_cube(n, 0.1)
    p[:, 2] += 0.05 - p[:, 2].min()
    sc = scenes._assemble([p], [np.zeros_like(p)], 1.0, friction=mu, dt=1 / 240, iterations=10,
                          radius=0.05)
    sc.plane = (0.0, 0.0, 1.0, plane_d)
    sc.vel = diff.rigid_velocity(sc, np.array([v]), np.array([w])).astype(np.float32)
    return sc


def test_free_flight_tangent_is_n_dt(pbdr_lib):
    n = 30
    sc = _box((0.3, -0.2, 0.5), (1.0, 2.0, -1.0))
    with pbdr_lib.Context(0) as c:
        _, J = diff.com_jacobian(c, sc, n, diff.rigid_seeds(sc))
    assert np.allclose(J[:, :3], n / 240 * np.eye(3), rtol=1e-5, atol=1e-6)
    assert np.abs(J[:, 3:]).max() < 1e-5


def test_sliding_grid_matches_oracle_differences(pbdr_lib, orc):
    """4 spinning boxes sliding on the ground with kinetic friction, 48
    substeps: d(final CoM)/d(v, omega) of the FP32 tangents against FP64
    central differences of the oracle."""
    sc, v, w = sliding_grid(seed=1)
    steps = 48
    with pbdr_lib.Context(0) as c:
        final, J = diff.final_com_and_jacobian(c, sc, v, w, steps)
    J_ref = rigid_fd_jacobian(orc, sc, v, w, steps)
    scale = np.abs(J_ref).max()
    assert np.abs(J - J_ref).max() <= 5e-3 * scale, np.abs(J - J_ref).max() / scale
    ref_final = diff.body_coms(sc, orc.OracleScene(sc).substep(steps).x)
    assert np.abs(final - ref_final).max() < 1e-4


def test_tangent_is_linear_in_the_seed(pbdr_lib):
    sc, v, w = sliding_grid(seed=2)
    s = diff.rigid_seeds(sc)
    a, b = 0.7, -1.9
    with pbdr_lib.Context(0) as c:
        _, J = diff.com_jacobian(c, sc, 20, [s[0], s[7], a * s[0] + b * s[7]])
    lhs, rhs = J[:, 2], a * J[:, 0] + b * J[:, 1]
    assert np.abs(lhs - rhs).max() <= 1e-5 * max(1.0, np.abs(rhs).max())


def test_primal_equals_the_streaming_step(pbdr_lib):
    """The tangent step advances the state with the streaming form's
    arithmetic."""
    sc, _, _ = sliding_grid(seed=4)
    with pbdr_lib.Context(0) as c:
        c.set_path(streaming=True)
        a = c.create_scene(sc)
        b = c.create_scene(sc)
        c.write_tangent(b, None, np.ones((sc.num_particles, 3), np.float32))
        c.step(a, 15)
        c.step_tangent(b, 15)
        pa, va, _ = c.read_state(a)
        pb, vb, _ = c.read_state(b)
    assert np.abs(pa - pb).max() <= 1e-6 and np.abs(va - vb).max() <= 1e-5


def test_new_scenes_start_with_zero_tangent(pbdr_lib):
    sc, _, _ = sliding_grid(seed=5)
    with pbdr_lib.Context(0) as c:
        a = c.create_scene(sc)
        c.write_tangent(a, np.ones((sc.num_particles, 3)), np.ones((sc.num_particles, 3)))
        c.step_tangent(a, 3)
        c.destroy_scene(a)
        b = c.create_scene(sc)             # reuses a's range
        dp, dv = c.read_tangent(b)
        assert not dp.any() and not dv.any()
        c.step_tangent(b, 5)
        dp, dv = c.read_tangent(b)
        assert not dp.any() and not dv.any()


def test_unsupported_scenes_are_refused(pbdr_lib):
    sc = scenes.analytic_box(1)            # carries a body force
    with pbdr_lib.Context(0) as c:
        sid = c.create_scene(sc)
        with pytest.raises(pbdr_lib.PbdrError) as e:
            c.step_tangent(sid, 1)
        assert e.value.code == -8


def test_autograd_backward_matches_oracle(pbdr_lib, orc):
    torch = pytest.importorskip("torch")
    sc, v, w = sliding_grid(seed=6)
    steps = 36
    vt = torch.tensor(v, dtype=torch.float64, requires_grad=True)
    wt = torch.tensor(w, dtype=torch.float64, requires_grad=True)
    weights = torch.tensor(np.random.default_rng(0).standard_normal((sc.num_bodies, 3)))
    with pbdr_lib.Context(0) as c:
        out = diff.FinalCoM.apply(vt, wt, c, sc, steps)
        (out * weights).sum().backward()
    J_ref = rigid_fd_jacobian(orc, sc, v, w, steps)
    g_ref = (J_ref.T @ weights.numpy().reshape(-1)).reshape(sc.num_bodies, 6)
    got = np.concatenate([vt.grad.numpy(), wt.grad.numpy()], 1)
    assert np.abs(got - g_ref).max() <= 5e-3 * np.abs(g_ref).max()
