"""Pins of the oracle's whole PBD-R substep (Algorithm 1) against closed
forms, conservation laws and the paper's analytic physics tests (CPU only).
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2603_14634_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
G = 9.81


def _free_space(sc):
    sc.gravity = (0.0, 0.0, 0.0)
    sc.plane = (0.0, 0.0, 1.0, -100.0)
    return sc


def test_free_fall_discrete_closed_form(orc):
    """No contact: the integration step of Algorithm 1 alone, so v_n = v_0 + n g dt and
    x_n = x_0 + n dt v_0 + g dt^2 n(n+1)/2 (symplectic Euler)."""
    sc = scenes.cube_drop(clearance=50.0)
    sc.vel[:] = np.array([0.3, -0.2, 1.5], np.float32)
    o = orc.OracleScene(sc)
    n, dt = 120, sc.dt
    o.substep(n)
    g = np.array(sc.gravity)
    v0 = sc.vel.astype(np.float64)
    x0 = sc.pos.astype(np.float64)
    # FP64 rounding of the shape-matching correction is ~ulp(|x|)/dt per step
    np.testing.assert_allclose(o.v, v0 + n * dt * g, rtol=0, atol=1e-9)
    np.testing.assert_allclose(o.x, x0 + n * dt * v0 + g * dt * dt * n * (n + 1) / 2,
                               rtol=0, atol=1e-11)


def test_standard_velocity_equals_incremental_without_corrections(orc):
    """With dX = 0 the standard update (X - X_init)/dt and the incremental
    V~ + dX/dt coincide (Sec. III-B)."""
    a = scenes.cube_drop(clearance=50.0)
    b = a.copy()
    b.flags = scenes.STD_VELOCITY
    oa, ob = orc.OracleScene(a), orc.OracleScene(b)
    oa.substep(50)
    ob.substep(50)
    np.testing.assert_allclose(oa.x, ob.x, atol=1e-12)
    np.testing.assert_allclose(oa.v, ob.v, atol=1e-9)


def test_rest_height_closed_form(orc):
    """Cube of n_z layers resting on the plane.  Per iteration the ground
    pushes the bottom layer out by its penetration, and shape matching
    spreads that over the body, so the penetration shrinks by
    beta = 1 - 1/n_z; a steady substep (zero velocity at its start) needs the
    K iterations to undo one step of gravity, g dt^2 = pen_0 (1 - beta^K),
    leaving pen_K = g dt^2 beta^K / (1 - beta^K): bottom layer centre at
    z = r - pen_K.  4^3 cube dropped from 1 m, dt = 1/240, K = 10."""
    sc = scenes.cube_drop()
    o = orc.OracleScene(sc)
    o.substep(240)
    beta, K, dt = 1 - 1 / 4, sc.iterations, sc.dt
    pen = G * dt * dt * beta ** K / (1 - beta ** K)
    np.testing.assert_allclose(o.x[:16, 2], sc.radius - pen, rtol=0, atol=1e-12)
    assert abs(o.x[:, 2].mean() - (0.2 - pen)) < 1e-7     # FP32 lattice rounding
    assert np.abs(o.v).max() < 1e-12
    # the 5^3 version of the same closed form
    sc5 = scenes.cube_drop(n=5, clearance=0.2)
    o5 = orc.OracleScene(sc5)
    o5.substep(240)
    beta = 1 - 1 / 5
    pen5 = G * dt * dt * beta ** K / (1 - beta ** K)
    np.testing.assert_allclose(o5.x[:25, 2], sc5.radius - pen5, rtol=0, atol=1e-12)


def test_free_spin_conserves_momenta_and_shape(orc):
    sc = _free_space(scenes.cube_drop(n=4))
    w = np.array([0.3, -0.5, 2.0])
    c0 = sc.pos.astype(np.float64).mean(0)
    sc.vel = np.cross(w[None, :], sc.pos - c0).astype(np.float32)
    o = orc.OracleScene(sc)
    _, P0, L0 = o.body_momenta()
    o.substep(1000)
    _, P, L = o.body_momenta()
    assert np.abs(P - P0).max() < 1e-11
    assert np.abs(L - L0).max() / np.abs(L0).max() < 1e-5
    d0 = np.linalg.norm(sc.pos[:, None].astype(np.float64) - sc.pos[None], axis=-1)
    d1 = np.linalg.norm(o.x[:, None] - o.x[None], axis=-1)
    assert np.abs(d1 - d0).max() < 1e-12
    # rotation angle about the spin axis: |w| t within the per-step
    # extrapolation error (atan(|w| dt) vs |w| dt per substep)
    ang = np.linalg.norm(w) * sc.dt * 1000
    R = orc.polar_rotation(((o.x - o.x.mean(0)).T @ (sc.pos - c0)))
    got = math.acos(max(-1.0, min(1.0, (np.trace(R) - 1) / 2)))
    assert abs(got - (ang % (2 * math.pi))) < 1e-3


def test_without_angular_correction_spin_decays(orc):
    """The mutation NO_ANGMOM (drop Eq. ang_momentum) must visibly lose L,
    which is what the conservation pin above guards against."""
    sc = _free_space(scenes.cube_drop(n=4))
    w = np.array([0.3, -0.5, 2.0])
    c0 = sc.pos.astype(np.float64).mean(0)
    sc.vel = np.cross(w[None, :], sc.pos - c0).astype(np.float32)
    sc.flags = scenes.NO_ANGMOM
    o = orc.OracleScene(sc)
    _, _, L0 = o.body_momenta()
    o.substep(1000)
    _, _, L = o.body_momenta()
    assert np.abs(L - L0).max() / np.abs(L0).max() > 1e-2


def test_symmetric_collision(orc):
    """Two equal cubes flying at each other: total momentum is conserved
    (pairwise antisymmetric contacts) and the outcome is mirror symmetric."""
    a = scenes.lattice_cube(3, 0.1)
    pos = np.concatenate([a + [-0.16, 0, 1.0], a + [0.16, 0, 1.0]]).astype(np.float32)
    vel = np.concatenate([np.tile([1.0, 0, 0], (27, 1)), np.tile([-1.0, 0, 0], (27, 1))]).astype(np.float32)
    sc = scenes.Scene(pos=pos, vel=vel, inv_mass=np.ones(54, np.float32),
                      body_off=np.array([0, 27, 54], np.int32), friction=0.5)
    _free_space(sc)
    o = orc.OracleScene(sc)
    o.substep(40)
    _, P, _ = o.body_momenta()
    assert np.abs(P.sum(0)).max() < 1e-11
    assert abs(P[0, 0]) < 27 * 1.0        # the contact slowed them down
    # lattice index i + 3j + 9k mirrors to (2 - i) + 3j + 9k
    perm = np.array([(2 - i) + 3 * j + 9 * k for k in range(3) for j in range(3) for i in range(3)])
    mirror = o.x[27:][perm].copy()
    mirror[:, 0] *= -1
    np.testing.assert_allclose(o.x[:27], mirror, atol=1e-12)
    assert o.x[:27, 0].max() < o.x[27:, 0].min()


def test_wrench_gives_force_and_torque(orc):
    """A constant CoM force F and torque tau on a body at rest in free space:
    after one substep P = F dt and L = tau dt (rigid bodies)."""
    sc = _free_space(scenes.cube_drop(n=4))
    sc.force = np.array([[1.0, -2.0, 0.5]], np.float32)
    sc.torque = np.array([[0.01, 0.02, -0.03]], np.float32)
    o = orc.OracleScene(sc)
    o.substep(1)
    _, P, L = o.body_momenta()
    np.testing.assert_allclose(P[0], sc.force[0] * sc.dt, atol=1e-12)
    np.testing.assert_allclose(L[0], sc.torque[0] * sc.dt, rtol=1e-6, atol=1e-12)


def test_grid_and_brute_force_substeps_identical(orc):
    sc = scenes.random_bodies_scene(seed=0)
    a, b = orc.OracleScene(sc), orc.OracleScene(sc)
    a.substep(2)
    b.substep(2, brute=True)
    np.testing.assert_array_equal(a.x, b.x)
    np.testing.assert_array_equal(a.v, b.v)


def _analytic_run(orc, test, T):
    sc = scenes.analytic_box(test)
    o = orc.OracleScene(sc)
    c0 = o.x.mean(0).copy()
    o.substep(int(round(T / sc.dt)))
    return sc, o, c0


def test_analytic_physics_tests(orc):
    """Table I tests 1-3 with Table II parameters (box 4 kg, 4^3 spheres,
    dt = 1 ms, 10 iterations; Sec. IV-B): the oracle tracks the closed forms
    x(t) = 1/2 (F - mu M g)/M t^2, theta(t) = 1/2 tau/lambda t^2 and
    x(t) = 1/2 (g sin th - mu g cos th) t^2 at t = 2 s."""
    with open(os.path.join(GOLDEN, "table2_parameters.json")) as f:
        P = json.load(f)
    T = 2.0
    M, mu = P["box_mass_kg"], P["friction_tests_1_3"]
    # test 1
    sc, o, c0 = _analytic_run(orc, 1, T)
    exp = 0.5 * (P["force_test_1_N"] - mu * M * G) / M * T * T
    got = o.x.mean(0)[0] - c0[0]
    assert abs(got - exp) / exp < 0.02
    # test 2: lambda of the discrete 4^3 box (spacing 0.1, 1/16 kg each) = 0.1
    sc, o, c0 = _analytic_run(orc, 2, T)
    lam = orc.body_inertia(sc.pos, 1 / sc.inv_mass.astype(np.float64), sc.pos.mean(0))[2, 2]
    assert abs(lam - 0.1) < 1e-6
    exp = 0.5 * P["torque_test_2_Nm"] / lam * T * T
    r0 = sc.pos[0, :2] - sc.pos[:, :2].mean(0)
    r1 = o.x[0, :2] - o.x[:, :2].mean(0)
    got = math.atan2(r0[0] * r1[1] - r0[1] * r1[0], r0 @ r1)
    assert abs(got - exp) / exp < 0.005
    # test 3
    sc, o, c0 = _analytic_run(orc, 3, T)
    th = P["slope_angle_test_3_rad"]
    exp = 0.5 * (G * math.sin(th) - mu * G * math.cos(th)) * T * T
    got = o.x.mean(0)[0] - c0[0]
    assert abs(got - exp) / exp < 0.03


def test_friction_mutation_detected(orc):
    """Dropping friction (mu = 0) in test 1 moves the box 13x too far: the
    analytic pin above catches a missing or sign-flipped friction term."""
    sc = scenes.analytic_box(1)
    sc.friction = 0.0
    o = orc.OracleScene(sc)
    c0 = o.x.mean(0).copy()
    o.substep(2000)
    exp = 0.5 * (17 - 0.4 * 4 * G) / 4 * 4.0
    assert abs((o.x.mean(0)[0] - c0[0]) - exp) / exp > 1.0


def test_empty_and_single_particle_scenes(orc):
    sc = scenes.Scene(pos=np.array([[0, 0, 0.5]], np.float32), vel=np.zeros((1, 3), np.float32),
                      inv_mass=np.ones(1, np.float32), body_off=np.array([0, 1], np.int32))
    o = orc.OracleScene(sc)
    o.substep(1)
    assert abs(o.v[0, 2] + G * sc.dt) < 1e-12
    sc0 = scenes.Scene(pos=np.zeros((0, 3), np.float32), vel=np.zeros((0, 3), np.float32),
                       inv_mass=np.zeros(0, np.float32), body_off=np.array([0], np.int32))
    orc.OracleScene(sc0).substep(1)
