"""How well an FP32 state determines the momentum the oracle's substep gives
each body (Sec. III-C, Eqs. lin_momentum / ang_momentum), measured by moving
every predicted position of the FP32 input by one ulp (tests/momentum_bounds).

The GPU tests compare per-body momentum with a relative bound of 1e-6 for
free bodies and, for bodies in contact, with a multiple of exactly this
measured response.  These CPU tests pin what that rests on:

* for bodies in free flight the substep's impulse does not depend on the
  positions at all (P) or only through r x v at rounding level (L), so FP32
  inputs resolve it far below 1e-6 and the relative bound is meaningful;
* for a body resting on the ground the impulse is whatever cancels gravity
  and the input velocity, so a one-ulp change of the input moves it by a
  large fraction of the body's whole momentum scale - no FP32
  implementation can meet 1e-6 relative there - and the response scales
  with ulp/dt as the contact model predicts.
"""
import numpy as np
import pytest

from momentum_bounds import body_moments, contact_bodies, ulp_response
from paper_2603_14634_gb300 import scenes


def _out(orc, sc, x32, v32):
    o = orc.OracleScene(sc)
    o.set_state(x32, v32)
    o.substep(1)
    return o


@pytest.mark.parametrize("seed", [0, 2])
def test_free_bodies_are_resolved_far_below_the_target(orc, seed):
    sc = scenes.random_bodies_scene(seed=seed)   # 64 bodies of 5^3 in flight, K = 20
    x32, v32 = sc.pos.astype(np.float32), sc.vel.astype(np.float32)
    o = _out(orc, sc, x32, v32)
    assert not contact_bodies(orc, sc, x32, o.x).any()
    _, _, sP, sL = body_moments(sc, o.x, o.v)
    rP, rL = ulp_response(orc, sc, x32, v32)
    assert (rP <= 1e-12 * sP).all(), (rP / sP).max()
    assert (rL <= 1e-7 * sL).all(), (rL / sL).max()


def test_resting_body_is_not_resolved_to_the_target(orc):
    sc = scenes.cube_drop()                      # the 4^3 cube, at rest by substep 232
    o = orc.OracleScene(sc)
    o.substep(232)
    x32, v32 = o.x.astype(np.float32), o.v.astype(np.float32)
    out = _out(orc, sc, x32, v32)
    assert contact_bodies(orc, sc, x32).all()
    _, _, sP, sL = body_moments(sc, out.x, out.v)
    rP, rL = ulp_response(orc, sc, x32, v32)
    # a one-ulp change of the FP32 input moves the resting body's momentum by
    # more than 1e4 times the relative target
    assert rP[0] > 1e-2 * sP[0] and rL[0] > 1e-2 * sL[0], (rP / sP, rL / sL)
    # and by about sqrt(n) m ulp(x)/dt: the impulse absorbs any velocity the
    # input carries, particle by particle
    m = 1.0 / sc.inv_mass.astype(np.float64)
    ulp = np.abs(np.nextafter(x32, np.float32(np.inf)) - x32).max(1)
    scale = np.sqrt(((m * ulp / sc.dt) ** 2).sum())
    assert 0.2 * scale <= rP[0] <= 5.0 * scale, (rP[0], scale)


def test_response_grows_with_the_contact_set(orc):
    """16 bodies colliding: bodies in contact respond by orders of magnitude
    more than bodies in flight in the same scene."""
    sc = scenes.random_bodies_scene(seed=0, num_bodies=16)
    sc.pos = (sc.pos * np.float32(0.8)).astype(np.float32)
    o = orc.OracleScene(sc)
    o.substep(120)
    x32, v32 = o.x.astype(np.float32), o.v.astype(np.float32)
    out = _out(orc, sc, x32, v32)
    hit = contact_bodies(orc, sc, x32, out.x)
    assert hit.any() and (~hit).any()
    _, _, sP, _ = body_moments(sc, out.x, out.v)
    rP, _ = ulp_response(orc, sc, x32, v32)
    rel = rP / sP
    assert rel[~hit].max() <= 1e-12
    assert np.median(rel[hit]) > 1e-8
