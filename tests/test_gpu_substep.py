"""GPU PBD-R substep vs the FP64 oracle from identical FP32 states.

Tolerances (one substep):
- positions within 1e-5 m;
- per-body momentum (tests/momentum_bounds.py): free bodies within 1e-6 of
  sum m|v| (P) and of sum m|r||v| (L); bodies in contact within that plus a
  multiple of the oracle's own response, on the same state, to a one-ulp
  change of the FP32 predicted positions.
Trajectories: errors against the closed forms of the analytic tests within
1.05x the oracle's own error + 1e-4.
"""
import math
import os
import sys

import numpy as np
import pytest

from paper_2603_14634_gb300 import scenes

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from momentum_bounds import check_momenta  # noqa: E402

pytestmark = pytest.mark.gpu

POS_TOL = 1e-5
G = 9.81


def _check_momenta(orc, sc, x0, pos, vel, o, label, state32, check_P=True, check_L=True):
    """x0: the oracle's start state (FP64); state32: the FP32 (x, v) both
    sides started from."""
    return check_momenta(orc, sc, x0, pos, vel, o, label, state32, check_P, check_L)


def _compare_one_substep(ctx, orc, sc, state=None, label="", check_P=True, check_L=True):
    """Both sides start from the same FP32 state (the scene's or `state`)."""
    sid = ctx.create_scene(sc)
    o = orc.OracleScene(sc)
    if state is not None:
        pos32, vel32 = (np.ascontiguousarray(a, np.float32) for a in state)
        ctx.write_state(sid, pos32, vel32)
        o.set_state(pos32, vel32)
    else:
        pos32, vel32 = (np.ascontiguousarray(a, np.float32) for a in (sc.pos, sc.vel))
    x_start = o.x.copy()
    ctx.step(sid, 1)
    pos, vel, err = ctx.read_state(sid)
    o.substep(1)
    assert err == 0, f"{label}: error bits {err}"
    dx = np.abs(pos - o.x).max()
    assert dx <= POS_TOL, f"{label}: max |dx| {dx}"
    rel = _check_momenta(orc, sc, x_start, pos, vel, o, label, (pos32, vel32), check_P, check_L)
    return dx, rel


def test_cube_free_fall(ctx, orc):
    _compare_one_substep(ctx, orc, scenes.cube_drop(), label="cube drop")


def test_cube_impact_and_rest(ctx, orc):
    sc = scenes.cube_drop()
    o = orc.OracleScene(sc)
    for n in (107, 2, 3, 20, 100):   # impact, bounce, settling, rest
        o.substep(n)
        _compare_one_substep(ctx, orc, sc, (o.x, o.v), label=f"cube after {n}")


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_bodies_scene(ctx, orc, seed):
    sc = scenes.random_bodies_scene(seed=seed)
    _compare_one_substep(ctx, orc, sc, label=f"64 bodies seed {seed}")


@pytest.mark.parametrize("seed", [0, 1])
def test_random_bodies_colliding(ctx, orc, seed):
    """States evolved by the oracle until bodies touch each other and the
    ground, then one substep on both sides."""
    sc = scenes.random_bodies_scene(seed=seed, num_bodies=16)
    sc.pos = (sc.pos * np.float32(0.8)).astype(np.float32)   # denser: collisions early
    o = orc.OracleScene(sc)
    o.substep(120)
    _compare_one_substep(ctx, orc, sc, (o.x, o.v), label=f"16 bodies colliding seed {seed}")


def test_large_scene_set_up_on_host_threads(ctx, orc):
    """A scene of 22 500 particles (above the size from which scene set-up
    splits its rest-shape pass over the context's host threads) with uneven
    particle masses: its state reads back exactly as given, and one substep
    agrees with the oracle."""
    sc = scenes.random_bodies_scene(seed=5, num_bodies=180)
    rng = np.random.default_rng(5)
    sc.inv_mass = rng.uniform(0.5, 2.0, sc.num_particles).astype(np.float32)
    assert sc.num_particles >= 16384
    sid = ctx.create_scene(sc)
    pos, vel, err = ctx.read_state(sid)
    assert err == 0 and np.array_equal(pos, sc.pos) and np.array_equal(vel, sc.vel)
    ctx.destroy_scene(sid)
    _compare_one_substep(ctx, orc, sc, label="22500 particles, uneven masses")


def test_batched_scenes_one_substep(ctx, orc):
    rng = np.random.default_rng(11)
    scs = [scenes.batch_scene(rng) for _ in range(8)]
    states = []
    for sc in scs:
        o = orc.OracleScene(sc)
        o.substep(60)
        states.append((o.x.astype(np.float32), o.v.astype(np.float32)))
    ids = [ctx.create_scene(sc) for sc in scs]
    for sid, (x, v) in zip(ids, states):
        ctx.write_state(sid, x, v)
    ctx.step(ids, 1)
    for sid, sc, (x, v) in zip(ids, scs, states):
        o = orc.OracleScene(sc)
        o.set_state(x, v)
        o.substep(1)
        pos, vel, err = ctx.read_state(sid)
        assert err == 0
        assert np.abs(pos - o.x).max() <= POS_TOL
        _check_momenta(orc, sc, x, pos, vel, o, f"batched scene {sid}", (x, v))


def test_wrench_one_substep(ctx, orc):
    for t in (1, 2, 3):
        sc = scenes.analytic_box(t)
        o = orc.OracleScene(sc)
        o.substep(30)
        _compare_one_substep(ctx, orc, sc, (o.x, o.v), label=f"analytic box {t}")


def test_flags_one_substep(ctx, orc):
    """Ablation flags: positions agree; a momentum is only compared where its
    correction is kept and the velocity is the incremental one (without them
    FP32 drifts, which is the paper's point, Sec. III-B and III-C)."""
    for flags in (scenes.NO_LINMOM, scenes.NO_ANGMOM, scenes.CONTACT_AVG, scenes.STD_VELOCITY):
        sc = scenes.random_bodies_scene(seed=4, num_bodies=12)
        sc.pos = (sc.pos * np.float32(0.8)).astype(np.float32)
        sc.flags = flags
        o = orc.OracleScene(sc)
        o.substep(100)
        _compare_one_substep(ctx, orc, sc, (o.x, o.v), label=f"flags {flags}",
                             check_P=not (flags & (scenes.NO_LINMOM | scenes.STD_VELOCITY)),
                             check_L=not (flags & (scenes.NO_ANGMOM | scenes.STD_VELOCITY)))


def test_momentum_correction_removes_fp32_drift(ctx, orc):
    """Sec. III-C: without Eq. lin_momentum the FP32 shape matching leaks
    linear momentum; with it a free body keeps P to ~1e-6."""
    errs = {}
    for flags in (0, scenes.NO_LINMOM):
        sc = scenes.cube_drop(n=7, clearance=5.0)
        sc.gravity = (0.0, 0.0, 0.0)
        c0 = sc.pos.astype(np.float64).mean(0)
        w = np.array([1.5, -2.0, 1.0])
        sc.vel = (np.array([0.7, -0.4, 0.2]) + np.cross(w, sc.pos - c0)).astype(np.float32)
        sc.flags = flags
        sid = ctx.create_scene(sc)
        ctx.step(sid, 50)
        pos, vel, _ = ctx.read_state(sid)
        P0 = sc.vel.astype(np.float64).sum(0)
        P1 = vel.astype(np.float64).sum(0)
        S = np.linalg.norm(sc.vel.astype(np.float64), axis=1).sum()
        errs[flags] = np.linalg.norm(P1 - P0) / S
    assert errs[0] < 1e-6 * 50 ** 0.5, errs
    assert errs[scenes.NO_LINMOM] > 10 * errs[0], errs


def test_rest_height_closed_form_on_gpu(ctx):
    """Bottom layer of the resting 4^3 cube at r - g dt^2 b^K/(1 - b^K),
    b = 3/4 (the oracle meets this to 1e-12)."""
    sc = scenes.cube_drop()
    sid = ctx.create_scene(sc)
    ctx.step(sid, 240)
    pos, vel, err = ctx.read_state(sid)
    beta, K, dt = 0.75, sc.iterations, sc.dt
    pen = G * dt * dt * beta ** K / (1 - beta ** K)
    assert err == 0
    assert np.abs(pos[:16, 2] - (sc.radius - pen)).max() < 1e-4
    assert np.abs(vel).max() < 1e-3


def test_cube_drop_trajectory(ctx, orc):
    sc = scenes.cube_drop()
    sid = ctx.create_scene(sc)
    o = orc.OracleScene(sc)
    for chunk in range(8):
        ctx.step(sid, 30)
        o.substep(30)
        pos, vel, _ = ctx.read_state(sid)
        assert np.abs(pos - o.x).max() < 1e-4, f"after {30 * (chunk + 1)} steps"


def _analytic(test, x_or_theta, t):
    if test == 1:
        return 0.5 * (17.0 - 0.4 * 4.0 * G) / 4.0 * t * t
    if test == 2:
        return 0.5 * 0.01 / 0.1 * t * t
    th = math.pi / 8
    return 0.5 * (G * math.sin(th) - 0.4 * G * math.cos(th)) * t * t


def _measure(test, sc, x):
    c = x.mean(0)
    if test == 2:
        r0 = sc.pos[0, :2] - sc.pos[:, :2].mean(0)
        r1 = x[0, :2] - c[:2]
        return math.atan2(r0[0] * r1[1] - r0[1] * r1[0], r0 @ r1)
    return c[0] - sc.pos.astype(np.float64).mean(0)[0]


@pytest.mark.parametrize("test", [1, 2, 3])
def test_analytic_tests_within_oracle_error(ctx, orc, test):
    """Table I tests at t = 2 s with Table II parameters: |GPU - analytic| <=
    1.05 |oracle - analytic| + 1e-4."""
    T = 2.0
    sc = scenes.analytic_box(test)
    n = int(round(T / sc.dt))
    sid = ctx.create_scene(sc)
    ctx.step(sid, n)
    pos, _, err = ctx.read_state(sid)
    o = orc.OracleScene(sc).substep(n)
    exp = _analytic(test, None, T)
    e_gpu = abs(_measure(test, sc, pos.astype(np.float64)) - exp)
    e_orc = abs(_measure(test, sc, o.x) - exp)
    assert err == 0
    assert e_gpu <= 1.05 * e_orc + 1e-4, (e_gpu, e_orc)


def test_rigidity_and_momentum_long_run(ctx, orc):
    """1000 substeps of 64 bodies: every body stays rigid (pairwise
    distances of its particles within 1e-4 m of the rest shape)."""
    sc = scenes.random_bodies_scene(seed=0)
    sid = ctx.create_scene(sc)
    ctx.step(sid, 1000)
    pos, vel, err = ctx.read_state(sid)
    assert err == 0 and np.isfinite(pos).all()
    for b in range(0, sc.num_bodies, 7):
        s0, s1 = sc.body_off[b], sc.body_off[b + 1]
        d0 = np.linalg.norm(sc.pos[s0:s1, None].astype(np.float64) - sc.pos[None, s0:s1], axis=-1)
        d1 = np.linalg.norm(pos[s0:s1, None].astype(np.float64) - pos[None, s0:s1], axis=-1)
        assert np.abs(d1 - d0).max() < 1e-4
    assert pos[:, 2].min() > 0.0          # nothing fell through the ground


@pytest.mark.parametrize("streaming", [False, True])
def test_determinism_and_batch_invariance(pbdr_lib, streaming):
    """Two runs repeat bit for bit, and a scene stepped alone equals the same
    scene stepped inside a batch of others."""
    rng = np.random.default_rng(5)
    scs = [scenes.batch_scene(rng) for _ in range(12)]
    outs = []
    for trial in range(2):
        with pbdr_lib.Context(0) as c:
            c.set_path(streaming)
            ids = [c.create_scene(s) for s in scs]
            c.step(ids, 40)
            outs.append([c.read_state(i)[:2] for i in ids])
    for a, b in zip(*outs):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    with pbdr_lib.Context(0) as c:
        c.set_path(streaming)
        sid = c.create_scene(scs[5])
        c.step(sid, 40)
        alone = c.read_state(sid)[:2]
    assert np.array_equal(alone[0], outs[0][5][0]) and np.array_equal(alone[1], outs[0][5][1])


def test_mixed_sizes_every_class_and_streaming_rest(ctx, orc):
    """One batch holding scenes of every size class of the scene-resident
    kernel (<= 1024, 2048, 4096, 8192 particles; the smallest class with
    scenes of 250 to 750 particles) and one larger scene that the streaming
    kernels take, one substep from oracle-evolved states."""
    scs = [scenes.random_bodies_scene(seed=s, num_bodies=nb) for s, nb in
           ((8, 2), (9, 4), (10, 6), (11, 14), (12, 30), (13, 60), (14, 80))]   # 250 .. 10000 particles
    states = []
    for sc in scs:
        sc.pos = (sc.pos * np.float32(0.85)).astype(np.float32)
        o = orc.OracleScene(sc)
        o.substep(90)
        states.append((o.x.astype(np.float32), o.v.astype(np.float32)))
    ids = [ctx.create_scene(sc) for sc in scs]
    for sid, (x, v) in zip(ids, states):
        ctx.write_state(sid, x, v)
    ctx.step(ids, 1)
    for sid, sc, (x, v) in zip(ids, scs, states):
        o = orc.OracleScene(sc)
        o.set_state(x, v)
        o.substep(1)
        pos, vel, err = ctx.read_state(sid)
        assert err == 0
        assert np.abs(pos - o.x).max() <= POS_TOL, f"scene of {sc.num_particles}"
        _check_momenta(orc, sc, x, pos, vel, o, f"scene of {sc.num_particles}", (x, v))


def test_nonfinite_state_is_reported(ctx, pbdr_lib):
    sc = scenes.cube_drop()
    sid = ctx.create_scene(sc)
    vel = sc.vel.copy()
    vel[3, 0] = np.nan
    ctx.write_state(sid, sc.pos, vel)
    ctx.step(sid, 1)
    _, _, err = ctx.read_state(sid)
    assert err & pbdr_lib.EBIT_NONFINITE


def test_invalid_arguments(ctx, pbdr_lib):
    E = pbdr_lib.PbdrError
    base = scenes.cube_drop()
    bad = base.copy()
    bad.body_off = np.array([0, 40, 30, 64], np.int32)
    with pytest.raises(E) as e:
        ctx.create_scene(bad)
    assert e.value.code == -1
    for field, val in (("radius", -1.0), ("dt", 0.0), ("iterations", 0), ("plane", (0, 0, 2.0, 0))):
        b = base.copy()
        setattr(b, field, val)
        with pytest.raises(E):
            ctx.create_scene(b)
    b = base.copy()
    b.pos = b.pos.copy()
    b.pos[0, 0] = np.inf
    with pytest.raises(E):
        ctx.create_scene(b)
    b = base.copy()
    b.flags = scenes.SM_FROM_XI
    with pytest.raises(E) as e:
        ctx.create_scene(b)
    assert e.value.code == -8
    sid = ctx.create_scene(base)
    with pytest.raises(E):
        ctx.step([sid, sid], 1)
    with pytest.raises(E):
        ctx.step([sid + 100], 1)
    ctx.destroy_scene(sid)
    with pytest.raises(E):
        ctx.read_state(sid)


def test_budget_exceeded(pbdr_lib):
    with pbdr_lib.Context(0, hbm_budget_bytes=1 << 20) as c:
        sc = scenes.random_bodies_scene(seed=0)
        with pytest.raises(pbdr_lib.PbdrError) as e:
            c.create_scene(sc)
        assert e.value.code == -3


def test_empty_and_single_particle_scene(ctx, orc):
    empty = scenes.Scene(pos=np.zeros((0, 3), np.float32), vel=np.zeros((0, 3), np.float32),
                         inv_mass=np.zeros(0, np.float32), body_off=np.array([0], np.int32))
    e = ctx.create_scene(empty)
    one = scenes.Scene(pos=np.array([[0, 0, 0.5]], np.float32), vel=np.zeros((1, 3), np.float32),
                       inv_mass=np.ones(1, np.float32), body_off=np.array([0, 1], np.int32))
    s = ctx.create_scene(one)
    ctx.step([e, s], 3)
    pos, vel, err = ctx.read_state(s)
    o = orc.OracleScene(one).substep(3)
    assert err == 0 and np.abs(pos - o.x).max() < 1e-6


@pytest.mark.parametrize("streaming", [False, True])
def test_graph_replay_and_autotune_are_bit_identical(pbdr_lib, streaming):
    """A captured CUDA graph per substep and the launch-shape autotuner change
    nothing in the results: plain launches, graph replay and graph replay
    with tuning give identical bytes.  340 scenes fill the small size
    classes past the SM count (so they are tuned) and one larger scene takes
    the streaming kernels; the tuning starts inside the second call, after
    128 substeps, and the graph is captured again after it."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    scs = [scenes.batch_scene(rng) for _ in range(340)]
    scs.append(scenes.random_bodies_scene(seed=3, num_bodies=75))   # 9375 particles
    outs, cfgs = [], []
    for graphs, tune in ((0, 0), (1, 0), (1, 1)):
        with pbdr_lib.Context(0) as c:
            c.set_path(streaming)
            c.set_option(pbdr_lib.OPT_GRAPHS, graphs)
            c.set_option(pbdr_lib.OPT_AUTOTUNE, tune)
            ids = [c.create_scene(s) for s in scs]
            st = torch.cuda.Stream()
            c.step(ids, 7, st.cuda_stream)
            c.step(ids, 130, st.cuda_stream)
            outs.append([c.read_state(i, st.cuda_stream)[:2] for i in ids])
            cfgs.append(c.plan_config(ids))
    if not streaming:
        assert any(k["scenes"] >= 152 for k in cfgs[2])   # a class was large enough to tune
    for other in outs[1:]:
        for (p0, v0), (p1, v1) in zip(outs[0], other):
            assert np.array_equal(p0, p1) and np.array_equal(v0, v1)


@pytest.mark.gpu
def test_tune_after_option(pbdr_lib):
    """PBDR_OPT_TUNE_AFTER takes a substep count >= 1; a scene set tuned
    after 5 substeps ends bit-identical to the same set never tuned."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(9)
    scs = [scenes.batch_scene(rng) for _ in range(400)]
    outs, cfgs = [], []
    for tune in (0, 1):
        with pbdr_lib.Context(0) as c:
            with pytest.raises(RuntimeError):
                c.set_option(pbdr_lib.OPT_TUNE_AFTER, 0)
            c.set_option(pbdr_lib.OPT_AUTOTUNE, tune)
            c.set_option(pbdr_lib.OPT_TUNE_AFTER, 5)
            ids = [c.create_scene(s) for s in scs]
            st = torch.cuda.Stream()
            c.step(ids, 4, st.cuda_stream)
            c.step(ids, 6, st.cuda_stream)   # tuned at its second substep when tune == 1
            outs.append([c.read_state(i, st.cuda_stream)[:2] for i in ids])
            cfgs.append(c.plan_config(ids))
    assert any(k["scenes"] >= 152 for k in cfgs[1])   # a class was large enough to tune
    for (p0, v0), (p1, v1) in zip(outs[0], outs[1]):
        assert np.array_equal(p0, p1) and np.array_equal(v0, v1)


def _two_particle_scene(pos, vel, inv_mass, plane, dt):
    pos = np.asarray(pos, np.float32)
    return scenes.Scene(pos=pos, vel=np.asarray(vel, np.float32), inv_mass=np.asarray(inv_mass, np.float32),
                        body_off=np.arange(pos.shape[0] + 1, dtype=np.int32), radius=0.05, friction=0.5,
                        gravity=(0.0, 0.0, 0.0), plane=plane, dt=dt, iterations=1)


def test_contact_and_friction_closed_form_cases(ctx, orc):
    """The configurations whose oracle results are pinned by closed forms
    (ground push-out, static and kinetic ground friction, pair push-out split
    by inverse mass, static and kinetic pair friction; single-particle
    bodies, one iteration) give the oracle's result on the GPU."""
    far = (0.0, 0.0, 1.0, -100.0)
    ground = (0.0, 0.0, 1.0, 0.0)
    dt = 1.0 / 256.0
    cases = [
        _two_particle_scene([[0.3, -0.2, 0.06]], [[0.0, 0.0, -6.0]], [1.0], ground, 1 / 240),
        _two_particle_scene([[0.0, 0.0, 0.06]], [[1.0, 0.0, -6.0]], [1.0], ground, 1 / 240),
        _two_particle_scene([[0.0, 0.0, 0.06]], [[4.0, 0.0, -6.0]], [1.0], ground, 1 / 240),
        _two_particle_scene([[-0.045, 0, 0.5], [0.045, 0, 0.5]], [[0, 0, 0], [0, 0, 0]], [1.0, 1.0], far, dt),
        _two_particle_scene([[-0.045, 0, 0.5], [0.045, 0, 0.5]], [[0, 0, 0], [0, 0, 0]], [1.0, 1 / 3], far, dt),
        _two_particle_scene([[-0.045, -0.25 * dt, 0.5], [0.045, 0.25 * dt, 0.5]], [[0, 0.25, 0], [0, -0.25, 0]],
                            [1.0, 1.0], far, dt),
        _two_particle_scene([[-0.045, -1.5 * dt, 0.5], [0.045, 1.5 * dt, 0.5]], [[0, 1.5, 0], [0, -1.5, 0]],
                            [1.0, 1.0], far, dt),
    ]
    ids = [ctx.create_scene(sc) for sc in cases]
    ctx.step(ids, 1)
    for sid, sc in zip(ids, cases):
        pos, vel, err = ctx.read_state(sid)
        o = orc.OracleScene(sc).substep(1)
        assert err == 0
        assert np.abs(pos - o.x).max() < 1e-6, (sid, pos, o.x)
        assert np.abs(vel - o.v).max() < 1e-3 * max(1.0, np.abs(o.v).max()), (sid, vel, o.v)
