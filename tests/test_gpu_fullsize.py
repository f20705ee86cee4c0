"""The full batched workload (4096 scenes, ~5M particles) in the launch
configuration the benchmark times: one batched pbdr_step over all scenes,
after the 240 settling substeps the benchmark runs before its timed region
(bodies resting on the ground and on each other, launch shapes tuned).
Sampled scenes - 16 at random and the 8 with the most neighbour entries -
are compared with the oracle one by one: one substep from the settled state,
and the neighbour lists the substep builds."""
import os
import sys

import numpy as np
import pytest

from paper_2603_14634_gb300 import scenes

pytestmark = pytest.mark.gpu

SETTLE = 240     # substeps the benchmark runs before timing


@pytest.fixture(scope="module")
def full_batch():
    return scenes.batched_scenes(4096, seed=0, workers=min(os.cpu_count() or 1, 32))


@pytest.fixture(scope="module")
def settled(pbdr_lib, full_batch):
    """A context holding the batch after SETTLE batched substeps, the sampled
    scene indices and their FP32 states at that point."""
    scs = full_batch
    c = pbdr_lib.Context(0)
    ids = [c.create_scene(s) for s in scs]
    c.step(ids, SETTLE)
    pos_all, vel_all, err = c.read_states(ids)
    assert not err.any()
    assert np.isfinite(pos_all).all() and np.isfinite(vel_all).all()
    totals = np.array([c.neighbor_total([i]) for i in ids])
    rng = np.random.default_rng(0)
    sample = sorted(set(rng.choice(len(scs), 16, replace=False).tolist()) |
                    set(np.argsort(-totals)[:8].tolist()))
    states = {k: c.read_state(ids[k])[:2] for k in sample}
    yield c, ids, sample, states, totals
    c.close()


def test_full_batch_settled_parity(orc, full_batch, settled):
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from test_gpu_substep import POS_TOL, _check_momenta
    scs = full_batch
    n = sum(s.num_particles for s in scs)
    assert 4.0e6 < n < 6.5e6
    c, ids, sample, states, totals = settled
    assert totals[sample].max() > 0          # contacts between bodies are in the sample
    c.step(ids, 1)                           # the whole batch, as the benchmark steps it
    for k in sample:
        x32, v32 = states[k]
        pos, vel, e = c.read_state(ids[k])
        assert e == 0, f"scene {k}: error bits {e}"
        o = orc.OracleScene(scs[k])
        o.set_state(x32, v32)
        x_start = o.x.copy()
        o.substep(1)
        dx = np.abs(pos - o.x).max()
        assert dx <= POS_TOL, f"scene {k}: max |dx| {dx:.2e}"
        _check_momenta(orc, scs[k], x_start, pos, vel, o, f"scene {k}", state32=(x32, v32))


def test_full_batch_settled_lists_exact(orc, full_batch, settled):
    """The lists the scene-resident kernel builds at the settled state equal
    the O(N^2) definition.  Each sampled scene is given the velocity
    v = -dt g (FP32), so that v~ = v + dt g vanishes and x~ = x exactly:
    the lists of x~ are then the oracle's lists of the known positions."""
    scs = full_batch
    c, ids, sample, states, totals = settled
    entries = 0
    for k in sample:
        sc = scs[k]
        x32 = states[k][0]
        v = np.zeros_like(x32)
        v[:] = -(np.float32(sc.dt) * np.asarray(sc.gravity, np.float32))
        c.write_state(ids[k], x32, v)
    c.step([ids[k] for k in sample], 1)
    for k in sample:
        sc = scs[k]
        _, _, off, idx = c.read_neighbors(ids[k], lists_only=True)
        o_off, o_idx = orc.neighbors(states[k][0], orc.body_index(sc.body_off), sc.radius, "brute")
        np.testing.assert_array_equal(off, o_off, err_msg=f"scene {k}")
        np.testing.assert_array_equal(idx, o_idx, err_msg=f"scene {k}")
        entries += idx.size
    assert entries > 0


def test_batched_equals_alone(pbdr_lib, full_batch):
    """A scene's result in the 4096-scene batch equals the scene stepped alone."""
    scs = full_batch
    with pbdr_lib.Context(0) as c:
        ids = [c.create_scene(s) for s in scs]
        c.step(ids, 1)
        for k in (5, 1234, len(scs) - 1):
            with pbdr_lib.Context(0) as c2:
                sid = c2.create_scene(scs[k])
                c2.step(sid, 1)
                alone = c2.read_state(sid)
            got = c.read_state(ids[k])
            assert np.array_equal(alone[0], got[0]) and np.array_equal(alone[1], got[1]), f"scene {k}"
