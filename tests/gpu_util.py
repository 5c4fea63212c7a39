"""Helpers shared by the GPU tests: move seeded host graphs to the device, run, compare."""
import numpy as np

import paper_1707_01989_gb300 as coop


class DevGraph:
    """A host CSR (graphgen.CSR) mirrored on the device; keeps the tensors alive."""

    def __init__(self, g, w=None, device="cuda:0"):
        import torch
        self.g = g
        self.ro = torch.from_numpy(np.array(g.row_off)).to(device)
        self.col = torch.from_numpy(np.array(g.col)).to(device)
        self.w = None if w is None else torch.from_numpy(np.ascontiguousarray(w).view(np.int32)).to(device)
        self.csr = coop.make_csr(self.ro, self.col)
        self.device = device

    def empty(self):
        import torch
        return torch.empty(self.g.num_vertices, dtype=torch.int32, device=self.device)


def run_bfs(ctx, dg, src, baseline=False, ok=(coop.COOP_OK,)):
    out = dg.empty()
    f = coop.coop_bfs_baseline if baseline else coop.coop_bfs
    st = f(ctx, dg.csr, src, out, stats=True, ok=ok)
    return out.cpu().numpy(), st


def run_sssp(ctx, dg, src, baseline=False, ok=(coop.COOP_OK,)):
    out = dg.empty()
    f = coop.coop_sssp_baseline if baseline else coop.coop_sssp
    st = f(ctx, dg.csr, dg.w, src, out, stats=True, ok=ok)
    return out.cpu().numpy().view(np.uint32), st


def assert_same(got, exp, what):
    got = np.asarray(got)
    exp = np.asarray(exp)
    assert got.shape == exp.shape, (what, got.shape, exp.shape)
    bad = np.flatnonzero(got != exp)
    assert bad.size == 0, f"{what}: {bad.size} mismatches, first at {bad[0]}: got {got[bad[0]]} expected {exp[bad[0]]}"


def hub_graph(seed, n=20000, hubs=(2048, 2300, 5000, 9000), base_edges=60000):
    """A sparse random graph on n vertices with heavy rows: hub i (vertex 1 + i) has
    hubs[i] out-edges.  Vertex 0 reaches every hub twice -- by a direct edge of weight 255
    and later by a two-edge path of weight 2 -- so shortest-path relaxation lowers each
    hub in two different iterations.  Returns (graph, weights in CSR order, source 0)."""
    import graphgen as gg
    rng = np.random.default_rng(seed)
    src = [rng.integers(0, n, base_edges)]
    dst = [rng.integers(0, n, base_edges)]
    want = {}
    for i, d in enumerate(hubs):
        h, mid = 1 + i, 1 + len(hubs) + i
        src.append(np.full(d, h))
        dst.append(rng.choice(n, size=d, replace=False))
        src.append(np.array([0, 0, mid]))
        dst.append(np.array([h, mid, h]))
        want[(0, h)], want[(0, mid)], want[(mid, h)] = 255, 1, 1
    g = gg.from_edges(n, np.concatenate(src), np.concatenate(dst), name=f"hubs{seed}")
    w = gg.weights(g, seed + 1)
    ro, col = np.array(g.row_off), np.array(g.col)
    for (u, v), x in want.items():
        row = col[ro[u]:ro[u + 1]]
        k = int(np.searchsorted(row, v))
        assert k < row.size and row[k] == v
        w[ro[u] + k] = x
    return g, w, 0
