"""Continuous-batching server: host logic on a fake context (CPU) and, on a
GPU, results that are identical alone and in the mix."""
import numpy as np
import pytest

from paper_2603_14634_gb300 import scenes
from paper_2603_14634_gb300.serve import Server, poisson_trace


class _Err(RuntimeError):
    def __init__(self, code):
        super().__init__(f"fake error {code}")
        self.code = code


class FakeContext:
    """Counts substeps per scene instead of simulating; enforces a particle
    capacity like the library's HBM budget."""

    def __init__(self, capacity):
        self.capacity = capacity
        self.used = 0
        self.scenes = {}
        self.next = 0
        self.step_sets = []

    def create_scene(self, sc):
        if self.used + sc.num_particles > self.capacity:
            raise _Err(-3)
        sid = self.next
        self.next += 1
        self.scenes[sid] = {"n": sc.num_particles, "steps": 0}
        self.used += sc.num_particles
        return sid

    def step(self, ids, substeps, stream=None):
        self.step_sets.append(tuple(sorted(ids)))
        for i in ids:
            self.scenes[i]["steps"] += substeps

    def read_state(self, sid, stream=None):
        n = self.scenes[sid]["n"]
        k = self.scenes[sid]["steps"]
        return np.full((n, 3), k, np.float32), np.zeros((n, 3), np.float32), 0

    def read_states(self, ids, stream=None):
        parts = [self.read_state(i) for i in ids]
        return (np.concatenate([p for p, _, _ in parts]), np.concatenate([v for _, v, _ in parts]),
                np.zeros(len(ids), np.uint32))

    def destroy_scene(self, sid):
        self.used -= self.scenes.pop(sid)["n"]


class _S:   # minimal scene stand-in
    def __init__(self, n, iterations=10):
        self.num_particles = n
        self.iterations = iterations


class VirtualClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-3
        return self.t


def test_every_request_gets_exactly_its_substeps():
    rng = np.random.default_rng(0)
    fake = FakeContext(capacity=10_000)
    srv = Server(hbm_budget_bytes=10_000, bytes_per_particle=1, ctx_factory=lambda: fake,
                 clock=VirtualClock())
    want = {}
    for k, t in enumerate(poisson_trace(200.0, 0.5, seed=1)):
        n = int(rng.integers(500, 3000))
        steps = int(rng.integers(1, 20))
        rid = srv.submit(_S(n), steps, arrival=float(t))
        want[rid] = steps
    st = srv.run(realtime=True)
    assert st["requests"] == len(want)
    for rid, steps in want.items():
        pos, _, _ = srv.results[rid]
        assert (pos == steps).all()
    assert fake.used == 0 and not fake.scenes


def test_budget_limits_residency_and_keeps_fifo():
    fake = FakeContext(capacity=5_000)
    srv = Server(hbm_budget_bytes=5_000, bytes_per_particle=1, ctx_factory=lambda: fake,
                 clock=VirtualClock())
    for k in range(8):
        srv.submit(_S(2_000), steps=3 + k % 3, arrival=0.0)
    srv.run(realtime=False)
    assert max(len(s) for s in fake.step_sets) <= 2        # 2 x 2000 <= 5000 < 3 x 2000
    order = [r.rid for r in sorted(srv.finished, key=lambda r: r.admitted)]
    assert order == sorted(order)                          # admitted first come first served


def test_late_arrivals_join_running_batches():
    fake = FakeContext(capacity=100_000)
    srv = Server(hbm_budget_bytes=100_000, bytes_per_particle=1, ctx_factory=lambda: fake,
                 clock=VirtualClock())
    a = srv.submit(_S(1000), steps=50, arrival=0.0)
    b = srv.submit(_S(1000), steps=5, arrival=0.01)
    srv.run(realtime=True)
    ra = next(r for r in srv.finished if r.rid == a)
    rb = next(r for r in srv.finished if r.rid == b)
    assert rb.admitted > ra.admitted and rb.done < ra.done
    assert any(len(s) == 2 for s in fake.step_sets)        # shared batched steps
    st = srv.stats()
    assert st["latency_ms_p50"] is not None and st["tick_ms_p99"] >= st["tick_ms_p50"]


def test_results_delivered_to_a_callback_are_not_kept():
    """With on_result, every finished request is handed over once, with its
    substep count in the fake's positions, and `results` stays empty."""
    fake = FakeContext(capacity=50_000)
    got = {}

    def on_result(rid, pos, vel, err):
        assert rid not in got
        got[rid] = (int(pos[0, 0]), pos.shape[0], err)

    srv = Server(hbm_budget_bytes=50_000, bytes_per_particle=1, ctx_factory=lambda: fake,
                 clock=VirtualClock(), on_result=on_result)
    want = {}
    for k in range(12):
        n, steps = 500 + 100 * k, 1 + k % 5
        want[srv.submit(_S(n), steps, arrival=0.001 * k)] = (steps, n, 0)
    srv.run(realtime=True)
    assert got == want and not srv.results


def test_poisson_trace_rate():
    t = poisson_trace(2000.0, 5.0, seed=0)
    assert abs(len(t) / 5.0 - 2000.0) < 100
    assert np.all(np.diff(t) > 0)


@pytest.mark.gpu
def test_results_identical_alone_and_in_the_mix(pbdr_lib):
    """Requests served with others (continuous batching, staggered
    arrivals, slots reused) end bit-identical to the same request stepped
    alone in a fresh context."""
    rng = np.random.default_rng(4)
    reqs = []
    for k in range(8):
        sc = scenes.random_bodies_scene(seed=100 + k, num_bodies=int(rng.integers(4, 20)))
        reqs.append((sc, int(rng.integers(2, 12)), 0.002 * k))
    srv = Server(hbm_budget_bytes=4 << 30)
    ids = [srv.submit(sc, steps, arrival=t) for sc, steps, t in reqs]
    st = srv.run(realtime=True)
    assert st["requests"] == len(reqs)
    assert srv._pin_err is not None   # results came through the asynchronous page-locked read
    for rid, (sc, steps, _) in zip(ids, reqs):
        with pbdr_lib.Context(0) as c:
            sid = c.create_scene(sc)
            c.step(sid, steps)
            pos, vel, err = c.read_state(sid)
        gpos, gvel, gerr = srv.results[rid]
        assert err == gerr == 0
        assert np.array_equal(pos, gpos) and np.array_equal(vel, gvel)


@pytest.mark.gpu
def test_served_results_match_oracle(pbdr_lib, orc):
    """Every request served by continuous batching (staggered arrivals,
    requests of 10^3 to 10^4 particles, so that both the scene-resident
    kernel and the streaming form run in the same ticks) ends within the
    position tolerance of the oracle stepping the same scene alone."""
    rng = np.random.default_rng(12)
    reqs = []
    for k in range(6):
        sc, _ = scenes.serving_request(rng, min_particles=1000, max_particles=12000)
        reqs.append((sc, int(rng.integers(2, 8)), 0.003 * k))
    assert max(sc.num_particles for sc, _, _ in reqs) > 8192   # one takes the streaming form
    srv = Server(hbm_budget_bytes=4 << 30)
    ids = [srv.submit(sc, steps, arrival=t) for sc, steps, t in reqs]
    st = srv.run(realtime=True)
    assert st["requests"] == len(reqs)
    assert len(srv.tick_ms) == st["ticks"] and min(srv.tick_ms) > 0
    for rid, (sc, steps, _) in zip(ids, reqs):
        gpos, gvel, gerr = srv.results[rid]
        assert gerr == 0
        o = orc.OracleScene(sc)
        o.substep(steps)
        dx = np.abs(gpos - o.x).max()
        assert dx <= 1e-5, f"request {rid} ({sc.num_particles} particles, {steps} substeps): |dx| {dx:.2e}"


@pytest.mark.gpu
def test_async_read_equals_sync_read(pbdr_lib):
    """pbdr_read_states_async into page-locked buffers, completed by an event
    on the same stream, gives the same bytes and error bits as the
    synchronous batched read; scenes read this way and destroyed after the
    event free ranges that a new scene can take."""
    import torch
    c = pbdr_lib.Context(0)
    scs = [scenes.random_bodies_scene(seed=300 + k, num_bodies=6 + k) for k in range(5)]
    ids = [c.create_scene(sc) for sc in scs]
    st = torch.cuda.Stream()
    c.step(ids, 4, st.cuda_stream)
    pick = [ids[3], ids[0], ids[4]]
    total = sum(scs[ids.index(i)].num_particles for i in pick)
    pos = torch.empty((total, 3), dtype=torch.float32, pin_memory=True).numpy()
    vel = torch.empty((total, 3), dtype=torch.float32, pin_memory=True).numpy()
    err = torch.zeros(len(pick), dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    c.read_states_async(pick, pos, vel, err, stream=st.cuda_stream)
    ev = torch.cuda.Event()
    ev.record(st)
    c.step([ids[1], ids[2]], 2, st.cuda_stream)      # other scenes keep stepping
    ev.synchronize()
    spos, svel, serr = c.read_states(pick, stream=st.cuda_stream)
    assert np.array_equal(pos, spos) and np.array_equal(vel, svel)
    assert np.array_equal(err, serr) and not err.any()
    for i in pick:
        c.destroy_scene(i)
    sid = c.create_scene(scs[0])                    # takes freed ranges
    c.step([sid], 3, st.cuda_stream)
    p2, v2, e2 = c.read_state(sid, stream=st.cuda_stream)
    with pbdr_lib.Context(0) as a:
        s0 = a.create_scene(scs[0])
        a.step(s0, 3)
        p0, v0, e0 = a.read_state(s0)
    assert e2 == e0 == 0 and np.array_equal(p2, p0) and np.array_equal(v2, v0)
    c.close()
