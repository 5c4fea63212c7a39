"""Pins for the operational model of the programming model (Sec. 3.1, Appendix A)."""
import os
import random

import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle.semantics import (CoopKernelModel, IllegalTransition, cooperative_bfs_model,
                              cooperative_sssp_model, replay_resize_log)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_fig1_worked_example():
    """Sec. 3.1's running example: N=4, kill 3 then 2, workgroup 0 forks ids 2 and 3."""
    model = None
    for raw in open(os.path.join(GOLDEN, "fig1_schedule.txt")):
        line = raw.split("#")[0].strip()
        if not line:
            continue
        tok = line.split()
        if tok[0] == "launch":
            model = CoopKernelModel.launch(int(tok[1][2:]), int(tok[2][2:]))
        elif tok[0] == "expect":
            assert model.M == int(tok[1][2:])
        elif tok[0] == "kill":
            assert model.offer_kill(int(tok[1]), accept=True)
        elif tok[0] == "fork":
            new = model.request_fork(int(tok[1]), int(tok[2]))
            assert new == [int(x) for x in tok[4:]]
    assert model.ids() == [0, 1, 2, 3]


def test_kill_rules():
    m = CoopKernelModel.launch(4, 4)
    # Kill-No-Op: always allowed
    assert not m.offer_kill(1, accept=False)
    # Kill: only the highest id
    with pytest.raises(IllegalTransition):
        m.offer_kill(1, accept=True)
    assert m.offer_kill(3, accept=True) and m.M == 3
    m2 = CoopKernelModel.launch(4, 1)
    # workgroup 0 is never killed (M = 1)
    with pytest.raises(IllegalTransition):
        m2.offer_kill(0, accept=True)
    assert not m2.offer_kill(0, accept=False)
    with pytest.raises(IllegalTransition):
        m.offer_kill(3, accept=False)  # no longer active


def test_fork_rules_and_transmit():
    m = CoopKernelModel.launch(6, 2)
    m.wgs[1]["level"] = 7
    m.wgs[0]["level"] = 3
    assert m.request_fork(1, 0) == []          # k = 0 always legal
    new = m.request_fork(1, 3)
    assert new == [2, 3, 4]
    assert all(m.wgs[i]["level"] == 7 for i in new)  # thread 0 of the forker transmits
    with pytest.raises(IllegalTransition):
        m.request_fork(0, 2)                    # k > N - M
    assert m.request_fork(0, 1) == [5]
    assert m.request_fork(2, 0) == []           # k = 0 is guaranteed when M = N
    with pytest.raises(IllegalTransition):
        m.request_fork(9, 0)                    # not an active workgroup
    with pytest.raises(IllegalTransition):
        CoopKernelModel.launch(4, 0)            # at least one workgroup is active


def test_resizing_barrier_keeps_prefix_and_transmits_from_wg0():
    rng = random.Random(3)
    for _ in range(200):
        N = rng.randint(1, 9)
        m = CoopKernelModel.launch(N, rng.randint(1, N))
        for i, wg in enumerate(m.wgs):
            wg["tag"] = i
        m.wgs[0]["level"] = 11
        before = list(m.wgs)
        M_new = rng.randint(1, N)
        m.resizing_barrier(M_new)
        assert m.M == M_new
        keep = min(len(before), M_new)
        assert all(m.wgs[i] is before[i] for i in range(keep))  # [0, min(M, M')-1] intact
        for i in range(keep, M_new):
            assert m.wgs[i]["level"] == 11 and m.wgs[i]["tag"] == 0
    with pytest.raises(IllegalTransition):
        CoopKernelModel.launch(3, 2).resizing_barrier(0)
    with pytest.raises(IllegalTransition):
        CoopKernelModel.launch(3, 2).resizing_barrier(4)


def test_replay_resize_log():
    log = [(4, 0, 2, 2), (2, 2, 0, 4), (4, 0, 0, 4), (4, 0, 3, 1), (1, 3, 3, 1)]
    model = replay_resize_log(4, 4, log)
    assert model.M == 1
    with pytest.raises(IllegalTransition):
        replay_resize_log(4, 4, [(4, 1, 0, 5)])   # fork beyond N
    with pytest.raises(IllegalTransition):
        replay_resize_log(4, 4, [(4, 0, 4, 0)])   # kills workgroup 0
    with pytest.raises(IllegalTransition):
        replay_resize_log(4, 4, [(3, 0, 0, 3)])   # inconsistent M_before
    with pytest.raises(IllegalTransition):
        replay_resize_log(4, 4, [(4, 0, 1, 4)])   # inconsistent M_after


def _random_schedule(seed):
    rng = random.Random(seed)

    def sched(b, M, N):
        r = rng.random()
        if r < 0.35:
            return rng.randint(1, N)
        return M
    return sched


@pytest.mark.parametrize("seed", range(12))
def test_schedule_invariance_bfs_model(seed):
    """Sec. 3.1: any kill/fork schedule must give the plain traversal's result."""
    g = gg.rmat(8, 6, seed=seed) if seed % 2 else gg.grid(9, 7)
    src = gg.max_out_degree_vertex(g)
    N = 1 + seed % 5
    lv, model = cooperative_bfs_model(g, src, N, 1 + seed % N, _random_schedule(seed))
    np.testing.assert_array_equal(np.array(lv), oracle.bfs(g, src))
    assert 1 <= model.M <= N


@pytest.mark.parametrize("seed", range(8))
def test_schedule_invariance_sssp_model(seed):
    g = gg.rmat(8, 6, seed=50 + seed)
    w = gg.weights(g, seed)
    src = gg.max_out_degree_vertex(g)
    d, _ = cooperative_sssp_model(g, w, src, 4, 2, _random_schedule(100 + seed))
    np.testing.assert_array_equal(np.array(d, dtype=np.uint64), oracle.dijkstra(g, w, src))


def test_rmat22_bench_schedules_both_kill_and_fork():
    """Every seeded schedule the bench and the full-size GPU test run on R-MAT 22 kills
    and forks within its five resizing barriers (model of the releaser's draws with the
    GPU's 152 CTAs), and never drops below the master CTA."""
    from schedule_model import RMAT22_RESIZING_BARRIERS, RMAT22_SCHEDULE, RMAT22_SEEDS, simulate
    for seed in RMAT22_SEEDS:
        kills, forks, spawned, M = simulate(seed, *RMAT22_SCHEDULE, 152, RMAT22_RESIZING_BARRIERS)
        assert kills > 0 and forks > 0 and spawned >= forks and 1 <= M <= 152, seed


def test_schedule_model_reproduces_the_earlier_fork_free_seeds():
    """The model against recorded device runs: with p_kill 0.3 and p_fork 0.5 on R-MAT 22,
    seeds 0, 1 and 2 recorded kills but no forks, seed 0 ending on the master CTA alone,
    and seed 3 recorded both."""
    from schedule_model import simulate
    runs = [simulate(s, 0.3, 0.5, 152, 5) for s in range(4)]
    assert all(k > 0 and f == 0 for k, f, _, _ in runs[:3])
    assert runs[0][3] == 1
    assert runs[3][0] > 0 and runs[3][1] > 0
