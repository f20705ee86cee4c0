"""Pins of the reference derivatives (FP64 oracle, central differences) that
the GPU tangents are checked against: closed forms of free flight and of a
box sliding with kinetic friction (Table I, Test 1 kinematics)."""
import numpy as np
import pytest

from fd_oracle import final_coms, mu_fd, rigid_fd_jacobian, sliding_grid
from paper_2603_14634_gb300 import diff, scenes


def _box(v, w=(0.0, 0.0, 0.0), mu=0.3, n=4, plane_d=0.0):
    p = scenes.lattice_cube(n, 0.1)
    p[:, 2] += 0.05 - p[:, 2].min()
    sc = scenes._assemble([p], [np.zeros_like(p)], 1.0, friction=mu, dt=1 / 240, iterations=10,
                          radius=0.05)
    sc.plane = (0.0, 0.0, 1.0, plane_d)
    sc.vel = diff.rigid_velocity(sc, np.array([v]), np.array([w])).astype(np.float32)
    return sc


def test_free_flight_derivative_is_n_dt(orc):
    """No contact: the final centre of mass is c0 + n dt v + const, so
    d c / d v = n dt I and d c / d omega = 0."""
    n = 30
    sc = _box((0.3, -0.2, 0.5), (1.0, 2.0, -1.0), plane_d=-100.0)
    v = np.array([[0.3, -0.2, 0.5]])
    w = np.array([[1.0, 2.0, -1.0]])
    J = rigid_fd_jacobian(orc, sc, v, w, n)
    assert np.allclose(J[:, :3], n / 240 * np.eye(3), atol=1e-9)
    assert np.allclose(J[:, 3:], 0.0, atol=1e-9)


def test_sliding_box_derivative_closed_form(orc):
    """A box sliding at speed s along x with kinetic friction loses mu g dt
    of speed per substep, so after n substeps it has moved
    x_n = n s dt - mu g dt^2 n (n + 1) / 2 along its velocity (the discrete
    form of x = s T - mu g T^2 / 2): d x / d v_x = n dt, and a sideways
    perturbation turns the path, d y / d v_y = n dt - mu g dt^2 n (n + 1) / (2 s)."""
    n, mu, speed, dt = 48, 0.3, 1.5, 1 / 240
    sc = _box((speed, 0.0, 0.0), mu=mu)
    J = rigid_fd_jacobian(orc, sc, np.array([[speed, 0.0, 0.0]]), np.zeros((1, 3)), n)
    assert J[0, 0] == pytest.approx(n * dt, rel=5e-4)
    assert J[1, 1] == pytest.approx(n * dt - mu * scenes.GRAVITY * dt * dt * n * (n + 1) / (2 * speed), rel=5e-4)
    assert abs(J[1, 0]) < 1e-8 and abs(J[0, 1]) < 1e-8


def test_fd_step_size_is_converged(orc):
    """The central differences agree between h = 1e-4 and 1e-5 on the
    sliding grid (no friction branch change inside the step)."""
    sc, v, w = sliding_grid(seed=3)
    steps = 24
    J1 = rigid_fd_jacobian(orc, sc, v, w, steps, h=1e-4)
    J2 = rigid_fd_jacobian(orc, sc, v, w, steps, h=1e-5)
    assert np.abs(J1 - J2).max() < 1e-5 * max(1.0, np.abs(J1).max())


def test_sliding_box_friction_derivative_closed_form(orc):
    """With x_n = n s dt - mu g dt^2 n (n + 1) / 2 (see above),
    d x / d mu = -g dt^2 n (n + 1) / 2."""
    n, mu, speed, dt = 48, 0.3, 1.5, 1 / 240
    sc = _box((speed, 0.0, 0.0), mu=mu)
    d = mu_fd(orc, sc, n)
    assert d[0] == pytest.approx(-0.5 * scenes.GRAVITY * dt * dt * n * (n + 1), rel=5e-4)
    assert abs(d[1]) < 1e-8
