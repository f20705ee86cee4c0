"""Per-body momentum checks of a GPU substep against the oracle (test
infrastructure: uses only the oracle and numpy).

The momentum constraint (Sec. III-C, Eqs. lin_momentum / ang_momentum)
restores each body's linear momentum P = sum m v and angular momentum
L = sum m (x - c) x v.  After one substep from the same FP32 state:

* free bodies (no particle within the contact band of another body or of
  the ground in the start, GPU or oracle state): |dP| <= 1e-6 sum m |v| and
  |dL| <= 1e-6 sum m |r| |v|, the relative target as stated;
* bodies in contact: a contact correction is a function of positions, so
  the momentum a body leaves a substep with depends on its particles'
  positions with a gain of about m / dt.  FP32 positions are known to one
  unit in the last place, and the oracle's own per-body momentum moves by
  `resp` when the predicted positions of the FP32 input move by one ulp
  (through x, or through v by ulp(x) / dt).  That response is measured here
  on the same state, per body, and the GPU may differ by 1e-6 s + K resp:
  each of its K iterations stores the state in FP32 (half an ulp) and forms
  the contact corrections from it (about another half ulp), so the solve
  perturbs the positions by at most about one ulp per iteration, each moving
  the impulse by at most the measured response.  (Measured: up to 1.6 resp
  at K = 10 and 7.4 resp at K = 20 on the colliding and resting scenes of
  the GPU tests.)
"""
import numpy as np

MOM_TOL = 1e-6
TRIALS = 3


def body_moments(sc, x, v):
    """P [B, 3], L about the CoM [B, 3], sum m|v| [B], sum m|r||v| [B]."""
    m = 1.0 / np.asarray(sc.inv_mass, np.float64)
    B = sc.num_bodies
    P, L = np.zeros((B, 3)), np.zeros((B, 3))
    sP, sL = np.zeros(B), np.zeros(B)
    for b in range(B):
        s0, s1 = sc.body_off[b], sc.body_off[b + 1]
        mb = m[s0:s1, None]
        xb = np.asarray(x[s0:s1], np.float64)
        vb = np.asarray(v[s0:s1], np.float64)
        r = xb - (mb * xb).sum(0) / mb.sum()
        P[b] = (mb * vb).sum(0)
        L[b] = np.cross(r, mb * vb).sum(0)
        sP[b] = (mb[:, 0] * np.linalg.norm(vb, axis=1)).sum()
        sL[b] = (mb[:, 0] * np.linalg.norm(r, axis=1) * np.linalg.norm(vb, axis=1)).sum()
    return P, L, sP, sL


def contact_bodies(orc, sc, *states):
    """Bodies with a particle within 2.2 r of another body or 1.5 r of the
    ground in any of the given states."""
    bid = orc.body_index(sc.body_off)
    n = np.array(sc.plane[:3], np.float64)
    hit = np.zeros(sc.num_particles, bool)
    for x in states:
        off, _ = orc.neighbors(np.asarray(x, np.float32), bid, sc.radius)
        hit |= np.diff(off) > 0
        hit |= (np.asarray(x, np.float64) @ n - sc.plane[3]) < 1.5 * sc.radius
    return np.array([hit[sc.body_off[b]:sc.body_off[b + 1]].any() for b in range(sc.num_bodies)])


def _oracle_step(orc, sc, x32, v32):
    o = orc.OracleScene(sc)
    o.set_state(x32, v32)
    o.substep(1)
    return o.x, o.v


def _impulse(orc, sc, x32, v32):
    """Change of each body's P and L over one oracle substep."""
    Pi, Li, _, _ = body_moments(sc, x32, v32)
    Po, Lo, _, _ = body_moments(sc, *_oracle_step(orc, sc, x32, v32))
    return Po - Pi, Lo - Li


def ulp_response(orc, sc, x32, v32, trials=TRIALS, seed=0):
    """Per body, the largest change of the momentum the oracle's substep
    gives the body (output minus input P and L) when every predicted
    position x~ = x + dt v~ of the FP32 input moves by one ulp of x in each
    coordinate (random signs): once through x, once through v (by
    ulp(x) / dt), `trials` times each.  Both sides of a comparison start from
    the same input, so only the substep's own response counts."""
    x32 = np.ascontiguousarray(x32, np.float32)
    v32 = np.ascontiguousarray(v32, np.float32)
    P0, L0 = _impulse(orc, sc, x32, v32)
    rP = np.zeros(sc.num_bodies)
    rL = np.zeros(sc.num_bodies)
    rng = np.random.default_rng(seed)
    for _ in range(trials):
        for through in ("x", "v"):
            up = rng.random(x32.shape) < 0.5
            nxt = np.nextafter(x32, np.where(up, np.float32(np.inf), np.float32(-np.inf))).astype(np.float32)
            if through == "x":
                xp, vp = nxt, v32
            else:
                xp = x32
                vp = (v32.astype(np.float64) + (nxt.astype(np.float64) - x32) / sc.dt).astype(np.float32)
            P1, L1 = _impulse(orc, sc, xp, vp)
            rP = np.maximum(rP, np.linalg.norm(P1 - P0, axis=1))
            rL = np.maximum(rL, np.linalg.norm(L1 - L0, axis=1))
    return rP, rL


def check_momenta(orc, sc, x_start, pos, vel, o, label, state32, check_P=True, check_L=True):
    """Asserts the bounds above for every body of one compared substep;
    returns the largest relative |dP|, |dL| over the free bodies."""
    hit = contact_bodies(orc, sc, x_start, pos, o.x)
    Pg, Lg, _, _ = body_moments(sc, pos, vel)
    Po, Lo, sP, sL = body_moments(sc, o.x, o.v)
    dP = np.linalg.norm(Pg - Po, axis=1)
    dL = np.linalg.norm(Lg - Lo, axis=1)
    rP = rL = np.zeros(sc.num_bodies)
    if hit.any():
        rP, rL = ulp_response(orc, sc, *state32)
    worst = [0.0, 0.0]
    gain = float(sc.iterations)
    for b in range(sc.num_bodies):
        bP = MOM_TOL * sP[b] + (gain * rP[b] if hit[b] else 0.0)
        bL = MOM_TOL * sL[b] + (gain * rL[b] if hit[b] else 0.0)
        kind = "contact" if hit[b] else "free"
        if check_P:
            assert dP[b] <= bP, f"{label}: {kind} body {b} |dP| {dP[b]:.3e} > {bP:.3e} (s {sP[b]:.2e}, resp {rP[b]:.2e})"
        if check_L:
            assert dL[b] <= bL, f"{label}: {kind} body {b} |dL| {dL[b]:.3e} > {bL:.3e} (s {sL[b]:.2e}, resp {rL[b]:.2e})"
        if not hit[b]:
            worst[0] = max(worst[0], dP[b] / max(sP[b], 1e-30))
            worst[1] = max(worst[1], dL[b] / max(sL[b], 1e-30))
    return worst
