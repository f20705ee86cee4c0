"""The full batched workload (4096 scenes, ~5M particles) in the launch
configuration the benchmark times: one batched pbdr_step over all scenes.
Sampled scenes are compared with the oracle one by one."""
import os
import sys

import numpy as np
import pytest

from paper_2603_14634_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full_batch():
    return scenes.batched_scenes(4096, seed=0, workers=min(os.cpu_count() or 1, 32))


def test_full_batch_sampled_parity(pbdr_lib, orc, full_batch):
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from test_gpu_substep import POS_TOL, _check_momenta
    scs = full_batch
    n = sum(s.num_particles for s in scs)
    assert 4.0e6 < n < 6.5e6
    with pbdr_lib.Context(0) as c:
        ids = [c.create_scene(s) for s in scs]
        c.step(ids, 1)
        pos_all, vel_all, err = c.read_states(ids)
        assert not err.any()
        assert np.isfinite(pos_all).all() and np.isfinite(vel_all).all()
        rng = np.random.default_rng(0)
        sample = sorted(rng.choice(len(scs), 16, replace=False).tolist()) + [len(scs) - 1]
        for k in sample:
            pos, vel, e = c.read_state(ids[k])
            o = orc.OracleScene(scs[k]).substep(1)
            assert np.abs(pos - o.x).max() <= POS_TOL, f"scene {k}"
            _check_momenta(orc, scs[k], scs[k].pos, pos, vel, o, f"scene {k}")
        # the batched result of each sampled scene equals that scene stepped alone
        k = sample[3]
        with pbdr_lib.Context(0) as c2:
            sid = c2.create_scene(scs[k])
            c2.step(sid, 1)
            alone = c2.read_state(sid)
        got = c.read_state(ids[k])
        assert np.array_equal(alone[0], got[0]) and np.array_equal(alone[1], got[1])
