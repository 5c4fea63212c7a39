"""The allocation-free BFS entry point agrees with coop_bfs and with the oracle.

coop_bfs_noalloc is for callers that must not allocate device memory (they reserve
their whole budget up front, run inside allocator callbacks, or cannot take
cudaMalloc's implicit synchronisation); its scratch is a static device array in the
library.  Two calls in a row on different graphs must each give exactly coop_bfs's
levels and the oracle's (integer output, so the tolerance is zero) -- the second call
also shows that the array's leftover contents from the first are cleared.  A graph at
the static limit (2^20 vertices, close to 2^25 edges) fills every part of the array.
This file is collected last.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_1707_01989_gb300 as coop
from gpu_util import DevGraph, assert_same

pytestmark = pytest.mark.gpu


def test_noalloc_matches_coop_bfs_on_two_calls(cuda_device):
    import torch
    ctx = coop.coop_init(0)
    try:
        cases = [(gg.rmat(16, 16, seed=31), None), (gg.grid(200, 150), 0)]
        for g, src in cases:
            src = gg.max_out_degree_vertex(g) if src is None else src
            dg = DevGraph(g)
            ref = dg.empty()
            coop.coop_bfs(ctx, dg.csr, src, ref, stats=True)
            got = dg.empty()
            status = torch.full((1,), 12345, dtype=torch.int32, device=cuda_device)
            coop.coop_bfs_noalloc(dg.csr, src, got, status)
            torch.cuda.synchronize()
            assert int(status.item()) == coop.COOP_OK
            assert_same(got.cpu().numpy(), ref.cpu().numpy(), f"noalloc vs coop_bfs on {g}")
            assert_same(got.cpu().numpy(), oracle.bfs(g, src), f"noalloc vs the oracle on {g}")
    finally:
        coop.coop_destroy(ctx)


@pytest.mark.slow
def test_noalloc_at_the_static_limit(cuda_device):
    """R-MAT scale 20 with edge factor 32: exactly 2^20 vertices and just under 2^25 edges,
    so the bitmap, both queues and both chunk indexes of the static array are used up to
    their ends; the levels equal the oracle's and the status is COOP_OK."""
    import torch
    g = gg.rmat(20, 32, seed=77)
    assert g.num_vertices == 1 << 20 and (1 << 24) < g.num_edges <= 1 << 25
    src = gg.max_out_degree_vertex(g)
    dg = DevGraph(g)
    for _ in range(2):
        got = dg.empty()
        status = torch.full((1,), 12345, dtype=torch.int32, device=cuda_device)
        coop.coop_bfs_noalloc(dg.csr, src, got, status)
        torch.cuda.synchronize()
        assert int(status.item()) == coop.COOP_OK
        assert_same(got.cpu().numpy(), oracle.bfs(g, src), "noalloc at the static limit vs the oracle")


def test_noalloc_rejects_graphs_over_the_limit(cuda_device):
    import torch
    V = (1 << 20) + 1
    ro = torch.zeros(V + 1, dtype=torch.int32, device=cuda_device)
    col = torch.zeros(0, dtype=torch.int32, device=cuda_device)
    out = torch.empty(V, dtype=torch.int32, device=cuda_device)
    with pytest.raises(coop.CoopError) as ei:
        coop.coop_bfs_noalloc(coop.make_csr(ro, col), 0, out)
    assert ei.value.status == coop.COOP_EINVAL
    assert "static scratch limit" in coop.coop_last_cuda_error()
