"""Step plans are cached per scene list, hold no device memory of their own
and are evicted least recently used; scene slots and table ranges of
destroyed scenes are reused.  None of that may change a result: every scene
must end bit-identical to the same scene stepped alone in a fresh context."""
import numpy as np
import pytest

from paper_2603_14634_gb300 import scenes

pytestmark = pytest.mark.gpu


def _alone(pbdr_lib, sc, steps, streaming):
    with pbdr_lib.Context(0) as c:
        c.set_path(streaming)
        sid = c.create_scene(sc)
        c.step(sid, steps)
        return c.read_state(sid)


@pytest.mark.parametrize("streaming", [False, True])
@pytest.mark.parametrize("graphs", [0, 1])
def test_rotating_subsets_past_the_plan_cache(pbdr_lib, streaming, graphs):
    """24 distinct scene subsets (more than the cache keeps) stepped in
    rotation, twice over, with graph replay on a side stream or plain
    launches; the big scene (9375 particles) takes the streaming kernels."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(31)
    scs = [scenes.batch_scene(rng) for _ in range(9)]
    scs.append(scenes.random_bodies_scene(seed=4, num_bodies=75))
    steps = np.zeros(len(scs), int)
    with pbdr_lib.Context(0) as c:
        c.set_path(streaming)
        c.set_option(pbdr_lib.OPT_GRAPHS, graphs)
        c.set_option(pbdr_lib.OPT_AUTOTUNE, 0)
        ids = [c.create_scene(s) for s in scs]
        st = torch.cuda.Stream()
        subsets = []
        for k in range(24):
            m = rng.random(len(scs)) < 0.5
            m[k % len(scs)] = True
            subsets.append(np.flatnonzero(m))
        for rep in range(2):
            for sub in subsets:
                c.step([ids[i] for i in sub], 1, st.cuda_stream)
                steps[sub] += 1
        got = [c.read_state(i, st.cuda_stream) for i in ids]
    for sc, n, (pos, vel, err) in zip(scs, steps, got):
        wpos, wvel, werr = _alone(pbdr_lib, sc, int(n), streaming)
        assert err == werr == 0
        assert np.array_equal(pos, wpos) and np.array_equal(vel, wvel)


@pytest.mark.parametrize("streaming", [False, True])
def test_slot_and_range_reuse(pbdr_lib, streaming):
    """Scenes destroyed between steps hand their slots and particle, body and
    chunk ranges to new scenes of other sizes, while the survivors keep
    stepping on a side stream; every scene still matches its solo run."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(32)
    pool = [scenes.batch_scene(rng) for _ in range(14)]
    pool.append(scenes.random_bodies_scene(seed=5, num_bodies=70))
    with pbdr_lib.Context(0) as c:
        c.set_path(streaming)
        st = torch.cuda.Stream()
        live = {}                       # sid -> (pool index, steps)
        results = []
        nxt = 0
        for tick in range(12):
            while len(live) < 5 and nxt < len(pool):
                live[c.create_scene(pool[nxt])] = [nxt, 0]
                nxt += 1
            c.step(list(live), 2, st.cuda_stream)
            for v in live.values():
                v[1] += 2
            if tick % 2 == 1:            # retire the two oldest
                for sid in sorted(live, key=lambda s: live[s][0])[:2]:
                    k, n = live.pop(sid)
                    results.append((k, n, c.read_state(sid, st.cuda_stream)))
                    c.destroy_scene(sid)
        for sid, (k, n) in live.items():
            results.append((k, n, c.read_state(sid, st.cuda_stream)))
    assert len(results) == len(pool)
    for k, n, (pos, vel, err) in results:
        wpos, wvel, werr = _alone(pbdr_lib, pool[k], n, streaming)
        assert err == werr == 0
        assert np.array_equal(pos, wpos) and np.array_equal(vel, wvel)


def test_two_contexts_in_lockstep_stay_identical(pbdr_lib):
    """Two contexts step the same 340 scenes (plus one scene for the
    streaming kernels, whose launches leave other data in shared memory
    between the scene-resident launches) one substep at a time; their states
    must stay bit-identical.  A missing barrier between the integration and
    the bounding-box pass once made rare neighbour lists depend on stale
    shared memory, which this catches."""
    rng = np.random.default_rng(8)
    scs = [scenes.batch_scene(rng) for _ in range(340)]
    scs.append(scenes.random_bodies_scene(seed=3, num_bodies=75))
    ctxs = []
    try:
        for _ in range(2):
            c = pbdr_lib.Context(0)
            c.set_option(pbdr_lib.OPT_GRAPHS, 0)
            c.set_option(pbdr_lib.OPT_AUTOTUNE, 0)
            ctxs.append((c, [c.create_scene(s) for s in scs]))
        for step in range(1, 201):
            for c, ids in ctxs:
                c.step(ids, 1)
            if step % 10 == 0:
                a = ctxs[0][0].read_states(ctxs[0][1])
                b = ctxs[1][0].read_states(ctxs[1][1])
                assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), f"substep {step}"
    finally:
        for c, _ in ctxs:
            c.close()


@pytest.mark.parametrize("read_before_destroy", [False, True])
def test_reuse_of_ranges_freed_with_work_in_flight_or_done(pbdr_lib, read_before_destroy):
    """A scene is destroyed either while its substeps may still run on the
    device (the next scene that takes its ranges must wait for them) or
    after its results were read (no wait: the next scene is created while
    another scene's substeps run on the side stream).  Either way the new
    scene, which takes the destroyed one's slot and ranges, ends
    bit-identical to the same scene stepped alone."""
    torch = pytest.importorskip("torch")
    a_sc = scenes.random_bodies_scene(seed=7, num_bodies=20)
    b_sc = scenes.random_bodies_scene(seed=8, num_bodies=20)
    other = scenes.random_bodies_scene(seed=9, num_bodies=40)
    with pbdr_lib.Context(0) as c:
        c.set_option(pbdr_lib.OPT_AUTOTUNE, 0)
        st = torch.cuda.Stream()
        o = c.create_scene(other)
        a = c.create_scene(a_sc)
        c.step([o, a], 30, st.cuda_stream)
        if read_before_destroy:
            c.read_state(a, st.cuda_stream)
        c.destroy_scene(a)
        c.step(o, 30, st.cuda_stream)        # keeps the device busy
        b = c.create_scene(b_sc)
        assert b == a                         # the freed slot (and ranges) are reused
        c.step([o, b], 6, st.cuda_stream)
        pos, vel, err = c.read_state(b, st.cuda_stream)
        opos, ovel, oerr = c.read_state(o, st.cuda_stream)
    wpos, wvel, werr = _alone(pbdr_lib, b_sc, 6, False)
    assert err == werr == 0 and oerr == 0
    assert np.array_equal(pos, wpos) and np.array_equal(vel, wvel)
    upos, uvel, _ = _alone(pbdr_lib, other, 66, False)
    assert np.array_equal(opos, upos) and np.array_equal(ovel, uvel)
