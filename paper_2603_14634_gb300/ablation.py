"""Ablation and analytic benchmark on the GPU path (Sec. V-C / Table III,
Sec. V-A / Table I).

Every variant of a study is one scene of ONE batched pbdr_step call, so a
whole study (all ablations, or a whole friction x force sweep) advances
together on the device; states are read back every ``sample_dt`` seconds and
the errors are computed on the host against the closed forms of Table I.

* ``table3``: Test 1 (pushed box, F = 17 N, mu = 0.4, 4 kg 4^3 box, dt = 1 ms,
  K = 10, Table II) — the paper's ablation test — and Test 2 (box with
  torque) with PBD-R and with each of its two modifications removed (the
  velocity update of Sec. III-B, the linear and the angular part of the
  momentum constraint of Sec. III-C), and standard PBD (all three removed).
  Errors at t = 2 s, at the end, their mean over the samples and the ratio
  of the mean to PBD-R's, as in Table III.
* ``tests123``: Tests 1-3 for PBD-R and PBD, position / rotation errors at
  t = 2 s and at the end.
* ``sweep``: Test 1 over a grid of friction coefficients and forces, PBD-R
  vs PBD (the friction x force sweep of Sec. V-A).

Metrics of a body state (positions p, velocities v, masses m):
  position error  |(c(t) - c(0)) - d_ref(t)|, c = centre of mass
  velocity error  |v_c(t) - v_ref(t)|
  linear momentum |P(t) - M v_ref(t)|
  rotation error  angle of the best-fit rotation of p(t) onto p(0) (Test 1, 3)
                  or |theta_z(t) - theta_ref(t)| (Test 2), in degrees
  angular momentum |L(t) - L_ref(t)| about the centre of mass.
"""
from __future__ import annotations

import argparse
import json
import math
from typing import Dict, List, Sequence

import numpy as np

from . import scenes

VARIANTS = {
    "PBD-R": 0,
    "no velocity update": scenes.STD_VELOCITY,
    "no linear momentum": scenes.NO_LINMOM,
    "no angular momentum": scenes.NO_ANGMOM,
    "PBD": scenes.STD_VELOCITY | scenes.NO_LINMOM | scenes.NO_ANGMOM,
}


# ---- closed forms of Table I ------------------------------------------------
def reference(test: int, sc, t: float) -> dict:
    """Analytic CoM displacement, CoM velocity (both 3-vectors), rotation
    angle about z and its rate for the box of ``scenes.analytic_box``."""
    g = scenes.GRAVITY
    m = 1.0 / sc.inv_mass.astype(np.float64)
    M = float(m.sum())
    zero = np.zeros(3)
    if test == 1:
        F = float(np.asarray(sc.force, np.float64).reshape(-1, 3)[0, 0])
        a = max(F - sc.friction * M * g, 0.0) / M
        return {"d": np.array([0.5 * a * t * t, 0.0, 0.0]), "v": np.array([a * t, 0.0, 0.0]),
                "theta": 0.0, "omega": 0.0}
    if test == 2:
        tau = float(np.asarray(sc.torque, np.float64).reshape(-1, 3)[0, 2])
        lam = inertia_zz(sc.pos.astype(np.float64), m)
        return {"d": zero, "v": zero, "theta": 0.5 * tau / lam * t * t, "omega": tau / lam * t}
    if test == 3:
        th = math.pi / 8
        a = max(g * math.sin(th) - sc.friction * g * math.cos(th), 0.0)
        return {"d": np.array([0.5 * a * t * t, 0.0, 0.0]), "v": np.array([a * t, 0.0, 0.0]),
                "theta": 0.0, "omega": 0.0}
    raise ValueError("test must be 1, 2 or 3")


def inertia_zz(p: np.ndarray, m: np.ndarray) -> float:
    c = (m[:, None] * p).sum(0) / m.sum()
    r = p - c
    return float((m * (r[:, 0] ** 2 + r[:, 1] ** 2)).sum())


def best_rotation(p0: np.ndarray, p: np.ndarray, m: np.ndarray) -> np.ndarray:
    """Proper rotation R minimising sum m |R (p0 - c0) - (p - c)|^2 (Kabsch)."""
    c0 = (m[:, None] * p0).sum(0) / m.sum()
    c = (m[:, None] * p).sum(0) / m.sum()
    H = ((p - c) * m[:, None]).T @ (p0 - c0)
    U, _, Vt = np.linalg.svd(H)
    D = np.diag([1.0, 1.0, np.sign(np.linalg.det(U @ Vt))])
    return U @ D @ Vt


def rotation_angle_deg(R: np.ndarray) -> float:
    return math.degrees(math.acos(max(-1.0, min(1.0, (np.trace(R) - 1.0) / 2.0))))


def body_metrics(test: int, sc, p0: np.ndarray, p: np.ndarray, v: np.ndarray, t: float,
                 theta_z: float) -> dict:
    """Errors of one state against the closed form (see the module doc)."""
    m = 1.0 / sc.inv_mass.astype(np.float64)
    M = float(m.sum())
    ref = reference(test, sc, t)
    c0 = (m[:, None] * p0).sum(0) / M
    c = (m[:, None] * p).sum(0) / M
    P = (m[:, None] * v).sum(0)
    r = p - c
    L = (m[:, None] * np.cross(r, v)).sum(0)
    if test == 2:
        rot = abs(math.degrees(theta_z - ref["theta"]))
        L_ref = np.array([0.0, 0.0, inertia_zz(p0, m) * ref["omega"]])
    else:
        rot = rotation_angle_deg(best_rotation(p0, p, m))
        L_ref = np.zeros(3)
    return {
        "pos": float(np.linalg.norm((c - c0) - ref["d"])),
        "vel": float(np.linalg.norm(P / M - ref["v"])),
        "lin": float(np.linalg.norm(P - M * ref["v"])),
        "rot": rot,
        "ang": float(np.linalg.norm(L - L_ref)),
    }


# ---- running a study ----------------------------------------------------------
def run_study(ctx, cases: Sequence[tuple], T: float, sample_dt: float = 0.1, stream=None) -> List[dict]:
    """cases: (test, scene) pairs, all stepped together.  Returns, per case,
    the sample times and the metric series."""
    ids = [ctx.create_scene(sc) for _, sc in cases]
    dt = float(cases[0][1].dt)
    per = max(1, int(round(sample_dt / dt)))
    n_samples = int(round(T / (per * dt)))
    p0 = [sc.pos.astype(np.float64) for _, sc in cases]
    series = [{"t": [], "pos": [], "vel": [], "lin": [], "rot": [], "ang": []} for _ in cases]
    theta_prev = [0.0] * len(cases)
    for k in range(1, n_samples + 1):
        ctx.step(ids, per, stream)
        t = k * per * dt
        for j, ((test, sc), sid) in enumerate(zip(cases, ids)):
            pos, vel, err = ctx.read_state(sid, stream)
            if err:
                raise RuntimeError(f"device error bits {err} in case {j}")
            p = pos.astype(np.float64)
            m = 1.0 / sc.inv_mass.astype(np.float64)
            R = best_rotation(p0[j], p, m)
            # unwrap the z angle across samples (far below pi per sample)
            th = math.atan2(R[1, 0], R[0, 0])
            th += 2 * math.pi * round((theta_prev[j] - th) / (2 * math.pi))
            theta_prev[j] = th
            met = body_metrics(test, sc, p0[j], p, vel.astype(np.float64), t, th)
            series[j]["t"].append(t)
            for key in ("pos", "vel", "lin", "rot", "ang"):
                series[j][key].append(met[key])
    for sid in ids:
        ctx.destroy_scene(sid)
    return series


def _at(series: dict, key: str, t: float) -> float:
    ts = np.asarray(series["t"])
    return float(np.asarray(series[key])[int(np.argmin(np.abs(ts - t)))])


def table3(ctx, T: float = 10.0, sample_dt: float = 0.1, dt: float = 1e-3, iterations: int = 10,
           stream=None, tests: Sequence[int] = (1, 2)) -> Dict[str, dict]:
    """Table III: PBD-R, each ablation and PBD on Test 1 (the paper's
    ablation test) and on Test 2 (where rotation is driven, so the angular
    part of the constraint has something to conserve).  Per test and
    variant: each metric at t = 2 s, at the end, its mean over the samples
    and the ratio of that mean to PBD-R's."""
    cases, keys = [], []
    for test in tests:
        for name, flags in VARIANTS.items():
            sc = scenes.analytic_box(test, dt=dt, iterations=iterations)
            sc.flags = flags
            cases.append((test, sc))
            keys.append((f"test{test}", name))
    series = run_study(ctx, cases, T, sample_dt, stream)
    out: Dict[str, dict] = {}
    for (tk, name), s in zip(keys, series):
        out.setdefault(tk, {})[name] = {
            key: {"t2": _at(s, key, 2.0), "end": _at(s, key, T), "mean": float(np.mean(s[key]))}
            for key in ("pos", "vel", "lin", "rot", "ang")}
    for tk, variants in out.items():
        base = variants["PBD-R"]
        for name in variants:
            for key in variants[name]:
                m0 = base[key]["mean"]
                variants[name][key]["x"] = variants[name][key]["mean"] / m0 if m0 > 0 else float("inf")
    return out


def tests123(ctx, T: float = 10.0, sample_dt: float = 0.1, dt: float = 1e-3, iterations: int = 10,
             stream=None) -> Dict[str, dict]:
    """Tests 1-3 of Table I, PBD-R vs PBD."""
    cases, names = [], []
    for test in (1, 2, 3):
        for name in ("PBD-R", "PBD"):
            sc = scenes.analytic_box(test, dt=dt, iterations=iterations)
            sc.flags = VARIANTS[name]
            cases.append((test, sc))
            names.append(f"test{test} {name}")
    series = run_study(ctx, cases, T, sample_dt, stream)
    return {n: {key: {"t2": _at(s, key, 2.0), "end": _at(s, key, T)} for key in ("pos", "rot")}
            for n, s in zip(names, series)}


def sweep(ctx, mus: Sequence[float] = (0.1, 0.2, 0.3, 0.4), forces: Sequence[float] = (20.0, 25.0, 30.0, 40.0),
          T: float = 5.0, sample_dt: float = 0.5, dt: float = 1e-3, iterations: int = 10,
          stream=None) -> List[dict]:
    """Test 1 over mu x F, PBD-R vs PBD: errors at T."""
    cases, keys = [], []
    for mu in mus:
        for F in forces:
            for name in ("PBD-R", "PBD"):
                sc = scenes.analytic_box(1, dt=dt, iterations=iterations)
                sc.friction = float(mu)
                sc.force = np.array([[F, 0.0, 0.0]], np.float32)
                sc.flags = VARIANTS[name]
                cases.append((1, sc))
                keys.append((mu, F, name))
    series = run_study(ctx, cases, T, sample_dt, stream)
    rows = {}
    for (mu, F, name), s in zip(keys, series):
        r = rows.setdefault((mu, F), {"mu": mu, "F": F})
        r[f"{name} pos"] = _at(s, "pos", T)
        r[f"{name} rot"] = _at(s, "rot", T)
    return list(rows.values())


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--study", choices=["table3", "tests123", "sweep", "all"], default="all")
    ap.add_argument("--T", type=float, default=10.0)
    ap.add_argument("--device", type=int, default=0)
    a = ap.parse_args(argv)
    from .binding import Context
    out = {}
    with Context(a.device) as ctx:
        if a.study in ("table3", "all"):
            out["table3"] = table3(ctx, T=a.T)
        if a.study in ("tests123", "all"):
            out["tests123"] = tests123(ctx, T=a.T)
        if a.study in ("sweep", "all"):
            out["sweep"] = sweep(ctx, T=min(a.T, 5.0))
    print(json.dumps(out, indent=1))
    return out


if __name__ == "__main__":
    main()
