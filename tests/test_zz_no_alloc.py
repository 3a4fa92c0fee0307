"""gg_sample_csc_noalloc: the sampling step for callers that cannot allocate
device memory (allocator callbacks, memory budgets handed out up front,
loops that must not call into the allocator). It must give exactly what
gg_sample_edges gives for the same in-edge list, call after call, with its
working memory in a fixed array inside the library. Kept in its own file so
that it runs last."""
import numpy as np
import pytest

import graphgen
from tests import gpu_common as gc


@pytest.mark.gpu
def test_noalloc_sampler_matches_gg_sample_edges_twice():
    import torch
    gg = gc.lib()
    for g in (graphgen.rmat(14, seed=5), graphgen.rmat(13, seed=6, symmetric=True),
              graphgen.from_arcs(9, [(0, 1), (1, 1), (2, 0), (8, 3), (3, 8), (3, 8)])):
        h = gc.load(gg, g)
        try:
            in_ptr = torch.from_numpy(gg.result_array(h, gg.GG_RESULT_CSC_PTR)).cuda()
            in_src = torch.from_numpy(gg.result_array(h, gg.GG_RESULT_CSC_SRC)).cuda()
            words = max((g.m + 31) // 32, 1)
            mask = torch.zeros(words, dtype=torch.int32, device="cuda")
            sp_ptr = torch.empty(g.n + 1, dtype=torch.int32, device="cuda")
            sp_src = torch.empty(max(g.m, 1), dtype=torch.int32, device="cuda")
            sp_nnz = torch.empty(1, dtype=torch.int32, device="cuda")
            for sigma, seed in ((0.5, 11), (0.3, 12)):   # two calls in a row
                torch.cuda.synchronize()
                gg.gg_sample_csc_noalloc(g.n, g.m, in_ptr, in_src, sigma, seed, g.symmetric,
                                         mask, sp_ptr, sp_src, sp_nnz,
                                         torch.cuda.current_stream().cuda_stream)
                torch.cuda.synchronize()
                gg.gg_sample_edges(h, sigma, seed)
                want_mask = gg.mask_bits(h, g.m)
                got_bits = np.unpackbits(mask.cpu().numpy().view(np.uint8), bitorder="little")[:g.m]
                assert np.array_equal(got_bits, want_mask)
                assert np.array_equal(sp_ptr.cpu().numpy(), gg.result_array(h, gg.GG_RESULT_SPARSE_PTR))
                want_src = gg.result_array(h, gg.GG_RESULT_SPARSE_SRC)
                nnz = int(sp_nnz.cpu().numpy()[0])
                assert nnz == want_src.shape[0]
                assert np.array_equal(sp_src.cpu().numpy()[:nnz], want_src)
        finally:
            gg.gg_free_graph(h)


@pytest.mark.gpu
def test_noalloc_sampler_rejects_sizes_beyond_its_scratch():
    gg = gc.lib()
    n = 1 << 20
    m = gg.GG_NOALLOC_MAX_ITEMS - n + 1
    with pytest.raises(gg.GGError) as e:
        gg.gg_sample_csc_noalloc(n, m, 1, 1, 0.5, 1, False, 1, 1, 1, 1)
    assert e.value.status == gg.GG_ERR_INVALID_ARG
    assert "GG_NOALLOC_MAX_ITEMS" in str(e.value)
