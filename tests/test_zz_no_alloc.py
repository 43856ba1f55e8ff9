"""The allocation-free entry point against the allocating one (GPU).

harp_count4_noalloc serves callers that may not allocate device memory while they run; it keeps its
scratch in a static device array shared by every call.  Two calls in a row on different graphs (and
the first graph again) must give exactly the counts and statistics of harp_count4_stats, which shows
that nothing stale survives from one call to the next.  A graph at the size limits (n = 262,144,
m close to 524,288, with a 1024-vertex clique whose lowest vertex has out-degree 1023, the largest
the CTA tier takes) checks that the fixed scratch holds the largest admitted workspace, and one call
runs on a side stream.  A CSR whose m disagrees with its offsets is refused on the device: the
self-check word d_out[6] is set and nothing is counted.  This file is collected last on purpose.
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


def _noalloc_vs_alloc(H, g, stream=None):
    csr = H.harp_build_csr(g.n, torch.from_numpy(g.src).cuda(), torch.from_numpy(g.dst).cuda())
    try:
        info = csr.info()
        off, cols = H.harp_csr_arrays(csr)
        want_counts, want_stats = H.harp_count4_stats(csr)
        torch.cuda.synchronize()
        out = torch.full((16,), -1, dtype=torch.int64, device="cuda")
        if stream is None:
            H.harp_count4_noalloc(info["n"], info["m"], off, cols, out.data_ptr())
            torch.cuda.synchronize()
        else:
            stream.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(stream):
                H.harp_count4_noalloc(info["n"], info["m"], off, cols, out.data_ptr(), stream)
            stream.synchronize()
        got = out.cpu().numpy().view(np.uint64)
        assert got[6] == 0, (g.name, "device self-check fired")
        assert got[:6].tolist() == want_counts.tolist(), g.name
        assert got[8:16].tolist() == want_stats.tolist(), g.name
    finally:
        csr.close()


def _clique_plus_filler(n=262144, k=1024, m_max=524288, seed=9):
    """K_k on the first k ids plus a sparse random matching on the rest, m <= m_max."""
    iu, ju = np.triu_indices(k, 1)
    rng = np.random.default_rng(seed)
    spare = m_max - iu.size
    a = rng.integers(k, n, size=spare)
    b = rng.integers(k, n, size=spare)
    src = np.concatenate([iu, a]).astype(np.int32)
    dst = np.concatenate([ju, b]).astype(np.int32)
    return graphgen.Graph(n, src, dst, f"K_{k} + {spare} random edges, n={n}")


def test_noalloc_two_calls_in_a_row_match_allocating_path(harp):
    g1 = graphgen.rmat(14, 16, seed=5)
    g2 = graphgen.ba(20000, 8, 3)
    _noalloc_vs_alloc(harp, g1)
    _noalloc_vs_alloc(harp, g2)
    _noalloc_vs_alloc(harp, g1)


def test_noalloc_at_the_size_limits_and_on_a_side_stream(harp):
    g = _clique_plus_filler()
    _noalloc_vs_alloc(harp, g)
    _noalloc_vs_alloc(harp, g, stream=torch.cuda.Stream())


def test_noalloc_refuses_a_csr_whose_m_disagrees_with_its_offsets(harp):
    g = graphgen.ba(3000, 4, 2)
    csr = harp.harp_build_csr(g.n, torch.from_numpy(g.src).cuda(), torch.from_numpy(g.dst).cuda())
    try:
        info = csr.info()
        off, cols = harp.harp_csr_arrays(csr)
        out = torch.full((16,), -1, dtype=torch.int64, device="cuda")
        harp.harp_count4_noalloc(info["n"], info["m"] // 2, off, cols, out.data_ptr())
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint64)
        assert got[6] != 0
        assert got[:6].tolist() == [0] * 6
        # the same array afterwards, with the right m, counts normally
        _noalloc_vs_alloc(harp, g)
    finally:
        csr.close()


def test_noalloc_rejects_sizes_beyond_the_static_scratch(harp):
    out = torch.zeros(16, dtype=torch.int64, device="cuda")
    with pytest.raises(harp.HarpError) as ei:
        harp.harp_count4_noalloc(262145, 10, 0, 0, out.data_ptr())
    assert ei.value.status == harp.HARP_ENOMEM
    with pytest.raises(harp.HarpError) as ei:
        harp.harp_count4_noalloc(1000, 524289, 0, 0, out.data_ptr())
    assert ei.value.status == harp.HARP_ENOMEM
