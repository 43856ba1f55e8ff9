"""The allocation-free entry point against the allocating one (GPU).

harp_count4_noalloc serves callers that may not allocate device memory while they run; it keeps its
scratch in a static device array shared by every call.  Two calls in a row on different graphs (and
the first graph again) must give exactly the counts and statistics of harp_count4_stats, which shows
that nothing stale survives from one call to the next.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import graphgen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def harp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_12074_gb300 import _build, harp as H
    _build.build()
    H.lib()
    return H


def _noalloc_vs_alloc(H, g):
    csr = H.harp_build_csr(g.n, torch.from_numpy(g.src).cuda(), torch.from_numpy(g.dst).cuda())
    try:
        info = csr.info()
        off, cols = H.harp_csr_arrays(csr)
        want_counts, want_stats = H.harp_count4_stats(csr)
        out = torch.full((16,), -1, dtype=torch.int64, device="cuda")
        H.harp_count4_noalloc(info["n"], info["m"], off, cols, out.data_ptr())
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint64)
        assert got[:6].tolist() == want_counts.tolist(), g.name
        assert got[8:16].tolist() == want_stats.tolist(), g.name
    finally:
        csr.close()


def test_noalloc_two_calls_in_a_row_match_allocating_path(harp):
    g1 = graphgen.rmat(14, 16, seed=5)
    g2 = graphgen.ba(20000, 8, 3)
    _noalloc_vs_alloc(harp, g1)
    _noalloc_vs_alloc(harp, g2)
    _noalloc_vs_alloc(harp, g1)


def test_noalloc_rejects_sizes_beyond_the_static_scratch(harp):
    out = torch.zeros(16, dtype=torch.int64, device="cuda")
    with pytest.raises(harp.HarpError) as ei:
        harp.harp_count4_noalloc(262145, 10, 0, 0, out.data_ptr())
    assert ei.value.status == harp.HARP_ENOMEM
    with pytest.raises(harp.HarpError) as ei:
        harp.harp_count4_noalloc(1000, 524289, 0, 0, out.data_ptr())
    assert ei.value.status == harp.HARP_ENOMEM
