"""Closed forms of the contact and friction terms (Sec. III-A constraints
(1) and (2) in the standard PBD reading: push-out by the penetration, pair
corrections split by inverse mass, Coulomb friction removing the tangential
displacement of the substep up to mu times the penetration), checked on the
FP64 oracle with single-particle bodies, for which shape matching and the
momentum constraint are identities, gravity zero and one solver iteration.

Ground (plane z = 0): a particle at height z0 moving down with v0 ends on the
surface, z1 = r, v1_z = (r - z0)/dt.  Its tangential displacement dt v_t is
removed when dt |v_t| <= mu pen (static) and shortened by mu pen otherwise
(kinetic: v1_t = v_t - mu pen/dt along v_t).

Pair (far from the ground): particles at distance d < 2r move apart along
their normal, particle p by pen w_p/(w_p + w_q) (pen = 2r - d), so their
distance becomes 2r and their momentum is unchanged; their relative
tangential displacement is removed (static) or shortened by mu pen
(kinetic), again split by inverse mass.  A mistake in any of these - the
sign of the normal, the weight split, the friction branch, the friction
scale - fails one of the tests below."""
import numpy as np
import pytest

from paper_2603_14634_gb300.scenes import Scene

R, DT, MU = 0.05, 1.0 / 240.0, 0.5


def _scene(pos, vel, inv_mass, plane=(0.0, 0.0, 1.0, 0.0), dt=DT):
    pos = np.asarray(pos, np.float32)
    n = pos.shape[0]
    return Scene(pos=pos, vel=np.asarray(vel, np.float32), inv_mass=np.asarray(inv_mass, np.float32),
                 body_off=np.arange(n + 1, dtype=np.int32), radius=R, friction=MU,
                 gravity=(0.0, 0.0, 0.0), plane=plane, dt=dt, iterations=1)


def _f(x):   # the FP32 input as the oracle sees it
    return float(np.float32(x))


def _step(orc, sc):
    return orc.OracleScene(sc).substep(1)


def test_ground_push_out_without_friction(orc):
    z0, vz = 0.06, -6.0
    o = _step(orc, _scene([[0.3, -0.2, z0]], [[0.0, 0.0, vz]], [1.0]))
    assert abs(o.x[0, 2] - R) < 1e-12
    assert abs(o.v[0, 2] - (R - _f(z0)) / DT) < 1e-9
    assert abs(o.x[0, 0] - _f(0.3)) < 1e-15 and abs(o.x[0, 1] - _f(-0.2)) < 1e-15
    assert abs(o.v[0, 0]) < 1e-15 and abs(o.v[0, 1]) < 1e-15


@pytest.mark.parametrize("vx", [1.0, 4.0])
def test_ground_friction_static_and_kinetic(orc, vx):
    z0, vz = 0.06, -6.0
    o = _step(orc, _scene([[0.0, 0.0, z0]], [[vx, 0.0, vz]], [1.0]))
    pen = R - (_f(z0) + DT * _f(vz))
    assert pen > 0
    slide = DT * _f(vx)
    if slide <= MU * pen:      # static: the tangential step is undone
        assert vx == 1.0
        want_x, want_v = 0.0, 0.0
    else:                      # kinetic: shortened by mu pen
        assert vx == 4.0
        want_x, want_v = slide - MU * pen, _f(vx) - MU * pen / DT
    assert abs(o.x[0, 0] - want_x) < 1e-12
    assert abs(o.v[0, 0] - want_v) < 1e-9
    assert abs(o.x[0, 2] - R) < 1e-12


@pytest.mark.parametrize("w2", [1.0, 1.0 / 3.0])
def test_pair_push_out_split_by_inverse_mass(orc, w2):
    a = 0.045                  # distance 0.09 < 2r
    far = (0.0, 0.0, 1.0, -100.0)
    o = _step(orc, _scene([[-a, 0.0, 5.0], [a, 0.0, 5.0]], [[0, 0, 0], [0, 0, 0]], [1.0, w2], far))
    d0 = _f(a) - _f(-a)
    pen = 2 * R - d0
    wf = _f(w2)
    s1, s2 = 1.0 / (1.0 + wf), wf / (1.0 + wf)
    assert abs(o.x[0, 0] - (_f(-a) - s1 * pen)) < 1e-12
    assert abs(o.x[1, 0] - (_f(a) + s2 * pen)) < 1e-12
    assert abs((o.x[1, 0] - o.x[0, 0]) - 2 * R) < 1e-12
    m1, m2 = 1.0, 1.0 / _f(w2)
    assert abs(m1 * o.v[0, 0] + m2 * o.v[1, 0]) < 1e-9          # momentum unchanged
    assert abs(o.v[0, 0] + s1 * pen / DT) < 1e-9


@pytest.mark.parametrize("s", [0.25, 1.5])
def test_pair_friction_static_and_kinetic(orc, s):
    a = 0.045
    far = (0.0, 0.0, 1.0, -100.0)
    dt = 1.0 / 256.0           # s dt exact: the predicted positions lie exactly on the x axis
    y0 = s * dt
    o = _step(orc, _scene([[-a, -y0, 5.0], [a, y0, 5.0]], [[0, s, 0], [0, -s, 0]], [1.0, 1.0], far, dt))
    # the normal is x; the relative displacement of the substep, dt (v1 - v2), is along y
    pen = 2 * R - (_f(a) - _f(-a))
    rel = 2 * dt * s
    if rel <= MU * pen:        # static: removed, half by each particle
        assert s == 0.25
        want_y, want_v = 0.0, 0.0
    else:                      # kinetic: shortened by mu pen, half each
        assert s == 1.5
        want_y, want_v = dt * s - 0.5 * MU * pen, s - 0.5 * MU * pen / dt
    # displacement of the substep along y: particle 1 by want_y, particle 2 by -want_y
    assert abs((o.x[0, 1] + y0) - want_y) < 1e-12 and abs((o.x[1, 1] - y0) + want_y) < 1e-12
    assert abs(o.v[0, 1] - want_v) < 1e-9 and abs(o.v[1, 1] + want_v) < 1e-9
    assert abs((o.x[1, 0] - o.x[0, 0]) - 2 * R) < 1e-12          # normal part unchanged by friction


def test_pair_beyond_contact_distance_is_untouched(orc):
    far = (0.0, 0.0, 1.0, -100.0)
    # within the neighbour radius 2.2 r but farther apart than 2r: no correction
    o = _step(orc, _scene([[-0.052, 0.0, 5.0], [0.052, 0.0, 5.0]], [[0, 1, 0], [0, -1, 0]], [1.0, 1.0], far))
    assert abs(o.x[0, 0] - _f(-0.052)) < 1e-15 and abs(o.v[0, 1] - 1.0) < 1e-15


@pytest.mark.parametrize("avg", [False, True])
def test_pair_sum_and_contact_averaging(orc, avg):
    """A particle pressed by two neighbours on opposite sides takes the plain
    sum of its two pair corrections (the summation of the contact
    corrections in Algorithm 1), or their mean with the CONTACT_AVG flag (the
    averaging of Macklin et al. 2014)."""
    far = (0.0, 0.0, 1.0, -100.0)
    xs = [0.0, 0.09, -0.095]       # overlaps 0.01 with the right and 0.005 with the left neighbour
    sc = _scene([[x, 0.0, 5.0] for x in xs], [[0, 0, 0]] * 3, [1.0] * 3, far)
    sc.flags = orc.CONTACT_AVG if avg else 0
    o = _step(orc, sc)
    pen_r = 2 * R - (_f(0.09) - _f(0.0))
    pen_l = 2 * R - (_f(0.0) - _f(-0.095))
    terms = [-0.5 * pen_r, 0.5 * pen_l]          # pushed left by the right one, right by the left one
    want = sum(terms) / (2 if avg else 1)
    assert abs(o.x[0, 0] - want) < 1e-12
    # each outer particle has one contact: the same either way
    assert abs(o.x[1, 0] - (_f(0.09) + 0.5 * pen_r)) < 1e-12
    assert abs(o.x[2, 0] - (_f(-0.095) - 0.5 * pen_l)) < 1e-12
