"""Cooperative behaviour on the GPU: forced kill/fork schedules, the host arbiter, timeouts.

Schedule invariance (Sec. 3.1: an offer_kill may always be a no-op and k = 0 forks is
always legal, so every schedule must give the same result): random seeded schedules
must leave BFS levels and SSSP distances bit-identical to the oracle, and every resize
the device logs must be a legal Fork/Kill sequence of the operational semantics
(Appendix A), replayed on oracle.semantics.
"""
import threading
import time

import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1707_01989_gb300 as coop
from gpu_util import DevGraph, assert_same, hub_graph, run_bfs, run_sssp
from oracle.semantics import replay_resize_log

pytestmark = pytest.mark.gpu


@pytest.fixture()
def ctx(cuda_device):
    c = coop.coop_init(0)
    yield c
    coop.coop_destroy(c)


def _replay(ctx, st):
    """Replay the device's resize log on the semantics model; returns (M_before, k, W, M_after) records."""
    full = coop.coop_get_resize_log(ctx)
    log = [r[2:6] for r in full]
    N = coop.coop_query(ctx)["max_ctas"]
    model = replay_resize_log(N, st.initial_active, log)
    assert sum(r[1] for r in log) == st.forks
    assert sum(r[2] for r in log) == st.kills
    assert min([st.initial_active] + [r[3] for r in log]) == st.min_active
    barriers = [r[0] for r in full]
    assert barriers == sorted(barriers) and all(1 <= b <= st.barriers for b in barriers)
    if st.barriers <= 2048:
        assert sorted(set(barriers)) == list(range(1, st.barriers + 1))  # every barrier recorded
    assert [r[1] for r in full] == sorted(r[1] for r in full)  # timestamps are monotone
    assert sum(r[6] for r in full) + st.initial_active + st.kills >= st.forks  # forks come from launches
    return log, model


@pytest.mark.parametrize("seed", range(32))
def test_random_schedules_bfs_bit_exact(ctx, seed):
    g = gg.rmat(13, 16, seed=seed % 4) if seed % 3 else gg.grid(64, 64)
    src = gg.max_out_degree_vertex(g) if seed % 3 else 0
    coop.coop_set_schedule(ctx, seed, p_kill=0.3, p_fork=0.5)
    lv, st = run_bfs(ctx, DevGraph(g), src)
    assert_same(lv, oracle.bfs(g, src), f"schedule {seed}")
    log, _ = _replay(ctx, st)
    if st.barriers > 60:  # the grid cases: the schedule really shrank and regrew the kernel
        assert st.kills > 0 and st.forks > 0


@pytest.mark.parametrize("seed", range(12))
def test_random_schedules_sssp_bit_exact(ctx, seed):
    g = gg.rmat(13, 16, seed=10 + seed % 3)
    w = gg.weights(g, seed)
    src = gg.max_out_degree_vertex(g)
    coop.coop_set_schedule(ctx, 1000 + seed, p_kill=0.4, p_fork=0.4)
    d, st = run_sssp(ctx, DevGraph(g, w), src)
    assert_same(d, oracle.dijkstra(g, w, src), f"sssp schedule {seed}")
    _replay(ctx, st)


def test_kill_at_every_barrier(ctx):
    """A schedule that accepts kills at every barrier only ever shrinks M, never below 1."""
    g = gg.rmat(12, 8, seed=2)
    src = gg.max_out_degree_vertex(g)
    coop.coop_set_schedule(ctx, 5, p_kill=1.0, p_fork=0.0)
    lv, st = run_bfs(ctx, DevGraph(g), src)
    assert_same(lv, oracle.bfs(g, src), "kill at every barrier")
    log, _ = _replay(ctx, st)
    assert all(r[1] == 0 for r in log)
    assert [r[3] for r in log] == sorted([r[3] for r in log], reverse=True)
    assert st.min_active >= 1 and st.forks == 0


def test_master_alone(ctx):
    """With N-1 CTAs lent to the host, the traversal runs on CTA 0 alone (M = 1 is legal)."""
    N = coop.coop_query(ctx)["max_ctas"]
    assert coop.coop_request_resources(ctx, N - 1) == N - 1
    g = gg.rmat(12, 8, seed=2)
    w = gg.weights(g, 3)
    src = gg.max_out_degree_vertex(g)
    dg = DevGraph(g, w)
    lv, st = run_bfs(ctx, dg, src)
    assert_same(lv, oracle.bfs(g, src), "master alone bfs")
    assert st.max_active == 1 and st.min_active == 1
    d, _ = run_sssp(ctx, dg, src)
    assert_same(d, oracle.dijkstra(g, w, src), "master alone sssp")
    coop.coop_release(ctx, N - 1)
    lv, st = run_bfs(ctx, dg, src)
    assert st.initial_active > 1


def test_host_request_and_release_during_run(ctx):
    """The scheduler takes half the CTAs from a running kernel, runs the co-runner on
    the freed SMs, and gives them back (Sec. 4.2)."""
    import torch
    N = coop.coop_query(ctx)["max_ctas"]
    half = N // 2
    # everything the co-runner needs is allocated up front: an allocation (or any other
    # device-synchronising call) made while the cooperative kernel runs waits for it
    x = torch.arange(1 << 22, dtype=torch.float32, device="cuda")
    y = torch.ones_like(x)
    ref = 2.0 * x + 1.0
    torch.testing.assert_close(ref, ref)  # loads every kernel the checks below use
    cs = torch.cuda.Stream(priority=-1)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    coop.coop_barrier_bench(ctx, 400000, stream=s, stats=False)
    time.sleep(0.02)
    t0 = time.perf_counter()
    got = coop.coop_request_resources(ctx, half, timeout_us=2_000_000)
    gather_ms = (time.perf_counter() - t0) * 1e3
    assert got == half
    assert coop.coop_query(ctx)["lent"] == half
    coop.coop_saxpy(half, 2.0, x, y, stream=cs)
    cs.synchronize()
    coop.coop_release(ctx, half)
    assert coop.coop_query(ctx)["lent"] == 0
    torch.testing.assert_close(y, ref)
    assert coop.coop_sync(ctx) == coop.COOP_OK
    st = coop.coop_get_stats(ctx)
    log, model = _replay(ctx, st)
    assert st.kills >= half and st.forks == half
    assert st.ctas_launched == N + half  # the main grid plus the forked CTAs
    assert any(r[2] == half for r in log)
    assert gather_ms < 1000


def test_request_with_no_run_in_flight_is_granted(ctx):
    N = coop.coop_query(ctx)["max_ctas"]
    assert coop.coop_request_resources(ctx, 3) == 3
    g = gg.rmat(11, 8, seed=1)
    src = gg.max_out_degree_vertex(g)
    lv, st = run_bfs(ctx, DevGraph(g), src)
    assert st.max_active <= N - 3  # the traversal ran without the lent CTAs
    assert_same(lv, oracle.bfs(g, src), "with lent ctas")
    coop.coop_release(ctx, 3)
    with pytest.raises(coop.CoopError):
        coop.coop_request_resources(ctx, N)  # CTA 0 is never surrendered


def test_concurrent_requests_from_another_thread(ctx):
    """Random request/release traffic from a host thread while traversals run."""
    import torch
    g = gg.rmat(16, 16, seed=3)
    w = gg.weights(g, 4)
    src = gg.max_out_degree_vertex(g)
    dg = DevGraph(g, w)
    exp_l, exp_d = oracle.bfs(g, src), oracle.dijkstra(g, w, src)
    stop = threading.Event()
    errors = []

    def arbiter():
        rng = np.random.default_rng(0)
        try:
            while not stop.is_set():
                n = int(rng.integers(1, 40))
                got = coop.coop_request_resources(ctx, n, timeout_us=500_000)
                time.sleep(0.0005)
                coop.coop_release(ctx, got)
        except Exception as exc:  # surfaced below
            errors.append(exc)

    t = threading.Thread(target=arbiter)
    t.start()
    try:
        for i in range(10):
            lv, _ = run_bfs(ctx, dg, src)
            assert_same(lv, exp_l, f"bfs under arbiter {i}")
            d, _ = run_sssp(ctx, dg, src)
            assert_same(d, exp_d, f"sssp under arbiter {i}")
    finally:
        stop.set()
        t.join()
    assert not errors, errors
    coop.coop_sync(ctx)


def test_barrier_wait_times_out_cleanly(ctx):
    """A barrier waiting for arrivals that never come returns COOP_ETIMEOUT (no hang, no
    fault) and the context keeps working."""
    coop.coop_set_timeout(ctx, 200_000)
    t0 = time.perf_counter()
    st = coop.coop_barrier_bench(ctx, 10, never_arrive=1, ok=(coop.COOP_ETIMEOUT,))
    assert st.status == coop.COOP_ETIMEOUT
    assert time.perf_counter() - t0 < 10
    coop.coop_set_timeout(ctx, 2_000_000)
    st = coop.coop_barrier_bench(ctx, 1000)
    assert st.status == coop.COOP_OK and st.barriers == 1000
    g = gg.grid(30, 30)
    lv, _ = run_bfs(ctx, DevGraph(g), 0)
    assert_same(lv, oracle.bfs(g, 0), "after timeout")


def test_saxpy_ragged(ctx):
    import torch
    for n in (1, 3, 1000, (1 << 20) + 3):
        x = torch.randn(n, device="cuda")
        y = torch.randn(n, device="cuda")
        ref = 3.0 * x + y
        coop.coop_saxpy(7, 3.0, x, y)
        torch.cuda.synchronize()
        torch.testing.assert_close(y, ref)


def test_barrier_bench_under_forced_schedule(ctx):
    """Empty resizing barriers with a kill or fork at about one barrier in eight: every
    barrier completes, and the resizes form a legal Fork/Kill sequence (Appendix A)."""
    coop.coop_set_schedule(ctx, 7, p_kill=1.0 / 16, p_fork=1.0 / 16)
    st = coop.coop_barrier_bench(ctx, 3000)
    coop.coop_set_schedule(ctx, 0, 0.0, 0.0)
    assert st.status == coop.COOP_OK and st.barriers == 3000
    assert st.kills > 0 and st.forks > 0
    _replay(ctx, st)
    st = coop.coop_barrier_bench(ctx, 100)
    assert st.kills == 0 and st.forks == 0  # the schedule is off again


@pytest.mark.parametrize("mode", ["chunk", "query", "simple"])
def test_kill_modes_serve_requests(ctx, mode):
    """Each place a host request can be served (Sec. 4.2: the regular barrier, the query
    barrier, and the query barrier with kill points between chunks) frees the CTAs asked
    for, logs a legal resize sequence and leaves every result unchanged."""
    import torch
    m = {"chunk": coop.COOP_KILL_CHUNK, "query": coop.COOP_KILL_QUERY, "simple": coop.COOP_KILL_SIMPLE}[mode]
    coop.coop_set_kill_mode(ctx, m)
    try:
        N = coop.coop_query(ctx)["max_ctas"]
        half = N // 2
        s = torch.cuda.Stream()
        torch.cuda.synchronize()
        coop.coop_barrier_bench(ctx, 400000, stream=s, stats=False)
        time.sleep(0.02)
        assert coop.coop_request_resources(ctx, half, timeout_us=2_000_000) == half
        coop.coop_release(ctx, half)
        assert coop.coop_sync(ctx) == coop.COOP_OK
        st = coop.coop_get_stats(ctx)
        log, _ = _replay(ctx, st)
        kill_barriers = [r for r in coop.coop_get_resize_log(ctx) if r[4] > 0]
        assert sum(r[4] for r in kill_barriers) >= half
        if mode == "simple":  # one offer_kill per CTA and barrier: the kills spread over barriers
            assert len(kill_barriers) >= 2
        g = gg.rmat(14, 16, seed=3)
        w = gg.weights(g, 4)
        src = gg.max_out_degree_vertex(g)
        dg = DevGraph(g, w)
        exp_l, exp_d = oracle.bfs(g, src), oracle.dijkstra(g, w, src)
        stop = threading.Event()
        errors = []

        def arbiter():
            rng = np.random.default_rng(1)
            try:
                while not stop.is_set():
                    got = coop.coop_request_resources(ctx, int(rng.integers(1, 60)), timeout_us=500_000)
                    time.sleep(0.0003)
                    coop.coop_release(ctx, got)
            except Exception as exc:  # surfaced below
                errors.append(exc)

        t = threading.Thread(target=arbiter)
        t.start()
        try:
            for i in range(6):
                lv, _ = run_bfs(ctx, dg, src)
                assert_same(lv, exp_l, f"bfs, kill mode {mode}, run {i}")
                d, _ = run_sssp(ctx, dg, src)
                assert_same(d, exp_d, f"sssp, kill mode {mode}, run {i}")
        finally:
            stop.set()
            t.join()
        assert not errors, errors
        coop.coop_sync(ctx)
    finally:
        coop.coop_set_kill_mode(ctx, coop.COOP_KILL_CHUNK)


def test_kill_mode_rejects_unknown(ctx):
    with pytest.raises(coop.CoopError):
        coop.coop_set_kill_mode(ctx, 3)


@pytest.mark.parametrize("seed", range(6))
def test_topology_driven_sssp_under_schedules(ctx, seed):
    """p-sssp under forced kill/fork schedules and host requests: bit-exact, legal log."""
    g = gg.rmat(12, 16, seed=40 + seed)
    w = gg.weights(g, 41 + seed)
    src = gg.max_out_degree_vertex(g)
    dg = DevGraph(g, w)
    coop.coop_set_schedule(ctx, 500 + seed, p_kill=0.3, p_fork=0.4)
    out = dg.empty()
    st = coop.coop_sssp_topo(ctx, dg.csr, dg.w, src, out, stats=True)
    coop.coop_set_schedule(ctx, 0, 0.0, 0.0)
    assert_same(out.cpu().numpy().view(np.uint32), oracle.dijkstra(g, w, src), f"p-sssp schedule {seed}")
    assert st.kills > 0 or st.forks > 0
    _replay(ctx, st)


@pytest.mark.parametrize("seed", range(3))
def test_topology_driven_sssp_heavy_rows_under_schedules(ctx, seed):
    """p-sssp whose heavy rows go through the chunk list, under forced kill/fork
    schedules: the chunks are dealt over whatever grid each relax interval has."""
    g, w, src = hub_graph(10 + seed)
    dg = DevGraph(g, w)
    coop.coop_set_schedule(ctx, 600 + seed, p_kill=0.3, p_fork=0.4)
    out = dg.empty()
    try:
        st = coop.coop_sssp_topo(ctx, dg.csr, dg.w, src, out, stats=True)
    finally:
        coop.coop_set_schedule(ctx, 0, 0.0, 0.0)
    assert_same(out.cpu().numpy().view(np.uint32), oracle.dijkstra(g, w, src), f"p-sssp hubs schedule {seed}")
    assert st.kills > 0 or st.forks > 0
    _replay(ctx, st)


@pytest.mark.slow
def test_full_size_rmat22_bfs_under_schedules(ctx):
    """R-MAT scale 22 BFS (the cooperative-multitasking workload) under the bench's forced
    random kill/fork schedules: every seed kills and forks, the levels are bit-exact and
    the resize log is legal."""
    from schedule_model import RMAT22_SCHEDULE, RMAT22_SEEDS
    g = gg.rmat(22, 16, seed=22)
    src = gg.max_out_degree_vertex(g)
    dg = DevGraph(g)
    ref = oracle.bfs(g, src)
    for seed in RMAT22_SEEDS:
        coop.coop_set_schedule(ctx, seed, *RMAT22_SCHEDULE)
        try:
            lv, st = run_bfs(ctx, dg, src)
        finally:
            coop.coop_set_schedule(ctx, 0, 0.0, 0.0)
        assert_same(lv, ref, f"rmat22 bfs under schedule {seed}")
        assert st.kills > 0 and st.forks > 0, (seed, st.kills, st.forks)
        _replay(ctx, st)


@pytest.mark.parametrize("name,period_ms,task_ms,share", [("light", 70.0, 3.0, 4), ("medium", 40.0, 3.0, 4),
                                                            ("heavy", 40.0, 10.0, 2)])
def test_traversals_bit_exact_under_table3_classes(ctx, name, period_ms, task_ms, share):
    """Sec. 5.5 / Table 3's workload classes: back-to-back BFS traversals while a
    non-cooperative task (saxpy launches sized to run about task_ms alone) takes N/share
    CTAs every period_ms and gives them back.  Every traversal's levels equal the
    oracle's, compared on the device after each one, and every task got its CTAs."""
    import torch
    g = gg.rmat(18, 16, seed=18)
    src = gg.max_out_degree_vertex(g)
    dg = DevGraph(g)
    ref = torch.from_numpy(oracle.bfs(g, src)).to(dg.device)
    lv = dg.empty()
    N = coop.coop_query(ctx)["max_ctas"]
    k = N // share
    x = torch.rand(1 << 22, device=dg.device)
    y = torch.rand(1 << 22, device=dg.device)
    cs = torch.cuda.Stream(device=dg.device, priority=-1)
    t0 = time.perf_counter()
    coop.coop_saxpy(k, 2.0, x, y, stream=cs)
    cs.synchronize()
    reps = max(1, int(task_ms / max((time.perf_counter() - t0) * 1e3, 0.01)))
    got_all, stop = [], threading.Event()

    def ticker():
        nxt = time.perf_counter()
        while not stop.is_set():
            got = coop.coop_request_resources(ctx, k, timeout_us=2_000_000)
            got_all.append(got)
            for _ in range(reps):
                coop.coop_saxpy(k, 2.0, x, y, stream=cs)
            cs.synchronize()
            coop.coop_release(ctx, got)
            nxt += period_ms / 1e3
            time.sleep(max(0.0, nxt - time.perf_counter()))

    stream = torch.cuda.Stream(device=dg.device)
    th = threading.Thread(target=ticker)
    th.start()
    n, bad = 0, 0
    t0 = time.perf_counter()
    try:
        while time.perf_counter() - t0 < 0.5:
            coop.coop_bfs(ctx, dg.csr, src, lv, stream=stream)
            stream.synchronize()
            bad += 0 if torch.equal(lv, ref) else 1
            n += 1
    finally:
        stop.set()
        th.join()
    assert coop.coop_sync(ctx) == coop.COOP_OK
    assert n > 10 and bad == 0, (name, n, bad)
    assert len(got_all) >= 3 and all(got == k for got in got_all), (name, got_all)


def test_request_log_records_every_request(ctx):
    """coop_get_request_log: one record per coop_request_resources call, in order, with
    the CTAs asked for and granted, and M as the device published it (0 for a request
    granted at once with no traversal in flight, else within [1, N])."""
    import torch
    g = gg.rmat(17, 16, seed=3)
    src = gg.max_out_degree_vertex(g)
    dg = DevGraph(g)
    lv = dg.empty()
    N = coop.coop_query(ctx)["max_ctas"]
    coop.coop_get_request_log(ctx, clear=True)
    got = coop.coop_request_resources(ctx, 5)
    coop.coop_release(ctx, got)
    asks, stop = [], threading.Event()

    def ticker():
        while not stop.is_set():
            n = 1 + len(asks) % (N // 2)
            got = coop.coop_request_resources(ctx, n, timeout_us=2_000_000)
            asks.append((n, got))
            coop.coop_release(ctx, got)
            time.sleep(0.0003)

    stream = torch.cuda.Stream()
    th = threading.Thread(target=ticker)
    th.start()
    try:
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 0.3:
            coop.coop_bfs(ctx, dg.csr, src, lv, stream=stream)
        stream.synchronize()
    finally:
        stop.set()
        th.join()
    coop.coop_sync(ctx)
    log = coop.coop_get_request_log(ctx, clear=True)
    assert len(log) == 1 + len(asks)
    assert log[0]["n_ctas"] == 5 and log[0]["granted"] == 5 and log[0]["active_at_post"] == 0
    assert [r["t_us"] for r in log] == sorted(r["t_us"] for r in log)
    for r, (n, got) in zip(log[1:], asks):
        assert r["n_ctas"] == n and r["granted"] == got == n and r["gather_us"] >= 0
        assert 0 <= r["lock_us"] <= r["post_us"] <= r["gather_us"]
        for m in (r["active_at_post"], r["active_at_grant"]):
            assert m == 0 or 1 <= m <= N
    assert any(r["active_at_post"] > 0 for r in log[1:]), "no request landed during a traversal"
    assert coop.coop_get_request_log(ctx) == []
    assert coop.coop_sync(ctx) == coop.COOP_OK
    np.testing.assert_array_equal(lv.cpu().numpy(), oracle.bfs(g, src))


def test_chunks_handed_back_mid_level_are_expanded_in_a_continuation(ctx):
    """Host requests that arrive in the middle of a wide level: the doomed CTAs hand the
    rest of their chunks back and leave within about one iteration; the returned ranges
    are expanded in a continuation interval of the same level (more barriers than levels).
    Every traversal's levels equal the oracle's, and every request is granted."""
    import torch
    g = gg.rmat(20, 16, seed=20)
    src = gg.max_out_degree_vertex(g)
    dg = DevGraph(g)
    ref = torch.from_numpy(oracle.bfs(g, src)).to(dg.device)
    lv = dg.empty()
    N = coop.coop_query(ctx)["max_ctas"]
    stop, grants = threading.Event(), []

    def ticker():
        i = 0
        while not stop.is_set():
            n = (N // 2, N // 4, N - 1, 3)[i % 4]
            got = coop.coop_request_resources(ctx, n, timeout_us=2_000_000)
            grants.append((n, got))
            time.sleep(0.00002)
            coop.coop_release(ctx, got)
            i += 1

    th = threading.Thread(target=ticker)
    th.start()
    runs, cont_runs, bad = 0, 0, 0
    try:
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 1.0:
            st = coop.coop_bfs(ctx, dg.csr, src, lv, stats=True)
            bad += 0 if torch.equal(lv, ref) else 1
            cont_runs += st.barriers > st.levels
            runs += 1
    finally:
        stop.set()
        th.join()
    assert coop.coop_sync(ctx) == coop.COOP_OK
    assert bad == 0, (bad, runs)
    assert all(got == n for n, got in grants) and len(grants) > 20
    assert cont_runs > 0, "no traversal expanded a returned range"


@pytest.mark.slow
def test_forked_ctas_join_a_running_level(ctx):
    """request_fork (Sec. 3.1) while a wide BFS level runs: the host lends half the CTAs
    before each R-MAT 22 traversal (which then starts on the other half) and gives them
    back while it runs.  The forked CTAs join the level in flight -- one CAS on the
    barrier's arrival word, then chunks from the level's shared cursor -- instead of
    waiting for its end.  Every traversal's levels equal the oracle's, every resize log
    is a legal Fork/Kill sequence, and some traversals record mid-level joiners."""
    import torch
    g = gg.rmat(22, 16, seed=22)
    src = gg.max_out_degree_vertex(g)
    dg = DevGraph(g)
    ref = torch.from_numpy(oracle.bfs(g, src)).to(dg.device)
    lv = dg.empty()
    N = coop.coop_query(ctx)["max_ctas"]
    half = N // 2
    s = torch.cuda.Stream(device=dg.device)
    runs_joined, joined_total = 0, 0
    for i in range(24):
        got = coop.coop_request_resources(ctx, half, timeout_us=2_000_000)  # idle: granted at once
        assert got == half
        coop.coop_bfs(ctx, dg.csr, src, lv, stream=s)  # on N - half CTAs, asynchronous
        time.sleep(0.00005 * (i % 6))
        coop.coop_release(ctx, got)
        s.synchronize()
        st = coop.coop_get_stats(ctx)
        assert st.status == coop.COOP_OK, st.status
        assert torch.equal(lv, ref), f"run {i}: levels differ from the oracle"
        assert st.initial_active == N - half
        assert 0 <= st.joined <= st.forks <= half, (st.joined, st.forks)
        _replay(ctx, st)
        runs_joined += st.joined > 0
        joined_total += st.joined
    assert coop.coop_sync(ctx) == coop.COOP_OK
    assert runs_joined > 0, "no forked CTA joined a running level"
