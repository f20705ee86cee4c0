"""Host-side metrics of the ablation / analytic benchmark: the closed forms
of Table I and the error measures must read zero on exact analytic states
and recover known rotations."""
import math

import numpy as np
import pytest

from paper_2603_14634_gb300 import ablation, scenes


def _rot_z(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def test_reference_accelerations_table1():
    sc1 = scenes.analytic_box(1)
    r = ablation.reference(1, sc1, 2.0)
    a = (17.0 - 0.4 * 4.0 * scenes.GRAVITY) / 4.0            # Table I, Test 1
    assert r["d"][0] == pytest.approx(0.5 * a * 4.0) and r["v"][0] == pytest.approx(2 * a)
    sc3 = scenes.analytic_box(3)
    th = math.pi / 8
    a3 = scenes.GRAVITY * (math.sin(th) - 0.4 * math.cos(th))   # Table I, Test 3
    assert ablation.reference(3, sc3, 1.0)["d"][0] == pytest.approx(0.5 * a3)
    sc2 = scenes.analytic_box(2)
    lam = ablation.inertia_zz(sc2.pos.astype(np.float64), 1.0 / sc2.inv_mass.astype(np.float64))
    assert lam == pytest.approx(0.1, rel=1e-6)                # discrete 4 kg 4^3 box, s = 0.1
    assert ablation.reference(2, sc2, 3.0)["theta"] == pytest.approx(0.5 * 0.01 / lam * 9.0)


def test_best_rotation_recovers_rotation():
    rng = np.random.default_rng(0)
    p0 = scenes.lattice_cube(4, 0.1).astype(np.float64)
    m = np.ones(len(p0))
    for R in scenes.random_rotations(rng, 5):
        p = p0 @ np.asarray(R, np.float64).T + rng.random(3)
        Rf = ablation.best_rotation(p0, p, m)
        assert np.allclose(Rf, R, atol=1e-12)
        ang = math.degrees(math.acos((np.trace(R) - 1) / 2))
        assert ablation.rotation_angle_deg(Rf) == pytest.approx(ang, abs=1e-6)


@pytest.mark.parametrize("test", [1, 2, 3])
def test_metrics_vanish_on_the_analytic_state(test):
    sc = scenes.analytic_box(test)
    p0 = sc.pos.astype(np.float64)
    m = 1.0 / sc.inv_mass.astype(np.float64)
    c0 = (m[:, None] * p0).sum(0) / m.sum()
    t = 3.0
    ref = ablation.reference(test, sc, t)
    R = _rot_z(ref["theta"])
    p = (p0 - c0) @ R.T + c0 + ref["d"]
    w = np.array([0.0, 0.0, ref["omega"]])
    v = ref["v"][None, :] + np.cross(w[None, :], p - (c0 + ref["d"]))
    met = ablation.body_metrics(test, sc, p0, p, v, t, ref["theta"])
    for key in ("pos", "vel", "lin", "rot"):
        assert met[key] < 1e-9, (key, met)
    assert met["ang"] < 1e-9


def test_metrics_see_a_displacement_and_a_spin():
    sc = scenes.analytic_box(1)
    p0 = sc.pos.astype(np.float64)
    ref = ablation.reference(1, sc, 1.0)
    p = p0 + ref["d"] + np.array([0.0, 0.03, 0.0])
    met = ablation.body_metrics(1, sc, p0, p, np.zeros_like(p), 1.0, 0.0)
    assert met["pos"] == pytest.approx(0.03)
    assert met["vel"] == pytest.approx(np.linalg.norm(ref["v"]))
    c0 = p0.mean(0)
    p = (p0 - c0) @ _rot_z(math.radians(10.0)).T + c0 + ref["d"]
    met = ablation.body_metrics(1, sc, p0, p, np.zeros_like(p), 1.0, 0.0)
    assert met["rot"] == pytest.approx(10.0, abs=1e-9)
