"""Operational model of the cooperative-kernel programming model.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Follows Sec. 3.1 (transmit, active workgroups, offer_kill, request_fork, global and
resizing barriers) and the rules of Appendix A (Thread-Step, Kill-No-Op, Kill, Fork,
Barrier, Resizing-Barrier).  A kernel state is (sigma, (w_0, ..., w_{M-1}, bottom^{N-M}));
sigma is left abstract and each active workgroup is represented by the transmitted
local state its threads hold (a dict).  Workgroup ids are list positions, so the
contiguity of ids in [0, M-1] is structural and the checks below concern which
transitions are legal.

Readings of garbled or conflicting passages:
  * Kill rule: the rule's side condition reads M > 0 while the text says a kill needs
    M > 1 and that workgroup 0 is never killed; the model requires M > 1.
  * request_fork by a workgroup "m <= M": only active workgroups execute, so m < M.
  * Resizing-Barrier rule: the rewritten state of w_0 is written with thread states of
    w_1 and the kill branch is written "for all i != 1"; the model reads index 0
    (workgroup 0 forks, every other workgroup offers to be killed).
  * Query barrier step (5), "ids larger than M - W": exactly W workgroups must leave,
    so the model kills ids >= M - W.

Besides the abstract machine this module has two *model traversals*: the cooperative
graph traversal of Sec. 3.2 Fig. 4 (BFS) and its frontier-relaxation analogue (SSSP),
executed step by step on the abstract machine under an arbitrary resize schedule.
They are slow pure-Python models used on small graphs to pin schedule invariance.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional


class IllegalTransition(AssertionError):
    """A transition the operational semantics does not allow."""


@dataclass
class CoopKernelModel:
    """Abstract kernel state: N (launch limit) and the active workgroups' transmitted state."""

    N: int
    wgs: List[dict] = field(default_factory=list)
    trace: List[tuple] = field(default_factory=list)

    @classmethod
    def launch(cls, N: int, M0: int, transmit: Optional[dict] = None) -> "CoopKernelModel":
        # "Initially, at least one workgroup is active" and at most N are requested.
        if not (1 <= M0 <= N):
            raise IllegalTransition(f"launch with M={M0}, N={N}")
        return cls(N=N, wgs=[dict(transmit or {}) for _ in range(M0)])

    @property
    def M(self) -> int:
        return len(self.wgs)

    def ids(self) -> List[int]:
        return list(range(self.M))

    def _check_active(self, m: int) -> None:
        if not (0 <= m < self.M):
            raise IllegalTransition(f"workgroup {m} is not active (M={self.M})")

    # -- offer_kill: rules Kill-No-Op and Kill ------------------------------------
    def offer_kill(self, m: int, accept: bool) -> bool:
        """Workgroup m offers to be killed; returns True when it ceased.

        A no-op when m < M-1 or M = 1; otherwise the scheduler may accept, which removes
        w_{M-1} and decrements M.  Workgroup 0 can never be killed.
        """
        self._check_active(m)
        killable = (m == self.M - 1) and self.M > 1
        if accept and not killable:
            raise IllegalTransition(f"kill of workgroup {m} with M={self.M}")
        if accept:
            self.wgs.pop()
            self.trace.append(("kill", m))
            return True
        self.trace.append(("kill-no-op", m))
        return False

    # -- request_fork: rule Fork -------------------------------------------------
    def request_fork(self, m: int, k: int) -> List[int]:
        """Workgroup m forks k in [0, N-M] workgroups with ids [M, M+k-1].

        Every new workgroup's transmitted state is thread 0 of w_m's.  Returns new ids.
        """
        self._check_active(m)
        if not (0 <= k <= self.N - self.M):
            raise IllegalTransition(f"fork k={k} with M={self.M}, N={self.N}")
        base = self.M
        self.wgs.extend(dict(self.wgs[m]) for _ in range(k))
        self.trace.append(("fork", m, k))
        return list(range(base, base + k))

    # -- barriers -----------------------------------------------------------------
    def global_barrier(self) -> None:
        """Rule Barrier: every active workgroup proceeds; M is unchanged."""
        self.trace.append(("barrier", self.M))

    def resizing_barrier(self, M_new: int) -> None:
        """Rule Resizing-Barrier: M becomes M_new in (0, N].

        Modelled as global_barrier; workgroup 0 forks max(0, M_new - M);
        global_barrier; every other workgroup offers to be killed (the top ones are
        accepted until M_new remain); global_barrier.  Forking precedes killing, so
        workgroups [0, min(M, M_new) - 1] are left intact.
        """
        if not (0 < M_new <= self.N):
            raise IllegalTransition(f"resize to M'={M_new} with N={self.N}")
        self.global_barrier()
        if M_new > self.M:
            self.request_fork(0, M_new - self.M)
        self.global_barrier()
        for m in range(self.M - 1, 0, -1):
            self.offer_kill(m, accept=(m >= M_new))
        self.global_barrier()
        if self.M != M_new:
            raise IllegalTransition("resize did not reach its target")

    def apply_resize(self, k: int, W: int) -> None:
        """One resizing barrier that forks k from workgroup 0 and then kills W from the top.

        This is how the device runtime logs each resize (admit k joiners, then let the
        W highest logical ids leave); both steps must be legal rule applications.
        """
        self.global_barrier()
        self.request_fork(0, k)
        self.global_barrier()
        for _ in range(W):
            self.offer_kill(self.M - 1, accept=True)
        self.global_barrier()


def replay_resize_log(N: int, M0: int, log) -> CoopKernelModel:
    """Replay a device log of (M_before, k, W, M_after) records; raises if any is illegal."""
    model = CoopKernelModel.launch(N, M0)
    for i, (m_before, k, W, m_after) in enumerate(log):
        if m_before != model.M:
            raise IllegalTransition(f"record {i}: M_before={m_before}, model has M={model.M}")
        model.apply_resize(k, W)
        if m_after != model.M:
            raise IllegalTransition(f"record {i}: M_after={m_after}, model has M={model.M}")
    return model


# ---- model traversals on the abstract machine ------------------------------------

Schedule = Callable[[int, int, int], int]  # (barrier index, M, N) -> M'


def _strided_work(model: CoopKernelModel, T: int, items: list):
    """Fig. 4's work split: thread (m, t) takes items tid, tid + stride, ... with
    tid = m*T + t and stride = M*T recomputed from the current M."""
    stride = model.M * T
    for m in model.ids():
        for t in range(T):
            for i in range(m * T + t, len(items), stride):
                yield items[i]


def cooperative_bfs_model(g, src: int, N: int, M0: int, schedule: Schedule, T: int = 2):
    """Sec. 3.2 Fig. 4 on the abstract machine: returns (level, model).

    Transmitted variables: level, in_nodes, out_nodes.  Two resizing barriers per
    frontier (after the swap, and after the reset / level increment).
    """
    V = g.num_vertices
    lvl = [-1] * V
    lvl[src] = 0
    model = CoopKernelModel.launch(N, M0, {"level": 0})
    in_nodes, out_nodes = [src], []
    level = 0
    b = 0
    while in_nodes:
        for u in _strided_work(model, T, in_nodes):
            for e in range(g.row_off[u], g.row_off[u + 1]):
                v = int(g.col[e])
                if lvl[v] == -1:
                    lvl[v] = level + 1
                    out_nodes.append(v)
        in_nodes, out_nodes = out_nodes, in_nodes
        model.resizing_barrier(schedule(b, model.M, N))
        b += 1
        out_nodes = []
        level += 1
        for wg in model.wgs:
            wg["level"] = level
        model.resizing_barrier(schedule(b, model.M, N))
        b += 1
    return lvl, model


def cooperative_sssp_model(g, w, src: int, N: int, M0: int, schedule: Schedule, T: int = 2):
    """Frontier relaxation in Fig. 4's shape: a vertex whose distance dropped in this
    round is pushed once into the next frontier.  Returns (dist, model)."""
    V = g.num_vertices
    INF = None
    dist = [INF] * V
    dist[src] = 0
    model = CoopKernelModel.launch(N, M0, {"round": 0})
    in_nodes = [src]
    rnd = 0
    b = 0
    while in_nodes:
        queued = set()
        out_nodes = []
        for u in _strided_work(model, T, in_nodes):
            for e in range(g.row_off[u], g.row_off[u + 1]):
                v = int(g.col[e])
                nd = dist[u] + int(w[e])
                if dist[v] is INF or nd < dist[v]:
                    dist[v] = nd
                    if v not in queued:
                        queued.add(v)
                        out_nodes.append(v)
        in_nodes = out_nodes
        model.resizing_barrier(schedule(b, model.M, N))
        b += 1
        rnd += 1
        for wg in model.wgs:
            wg["round"] = rnd
        model.resizing_barrier(schedule(b, model.M, N))
        b += 1
    return [0xFFFFFFFF if d is INF else d for d in dist], model
