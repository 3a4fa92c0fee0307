"""gg_sample_csc_noalloc: the sampling step for callers that cannot allocate
device memory (allocator callbacks, memory budgets handed out up front,
loops that must not call into the allocator). It must give exactly the
oracle's sampled flags and packed in-edges (Sec. 3.4) and what
gg_sample_edges gives for the same in-edge list, call after call, with its
working memory in a fixed array inside the library. Kept in its own file so
that it runs last."""
import numpy as np
import pytest

import graphgen
import oracle
from tests import gpu_common as gc


@pytest.mark.gpu
def test_noalloc_sampler_matches_the_oracle_twice():
    import torch
    gg = gc.lib()
    for g in (graphgen.rmat(14, seed=5), graphgen.rmat(13, seed=6, symmetric=True),
              graphgen.from_arcs(9, [(0, 1), (1, 1), (2, 0), (8, 3), (3, 8), (3, 8)])):
        h = gc.load(gg, g)
        try:
            ip, isrc, _, _ = oracle.csc_from_csr(g.n, g.rowptr, g.colidx)   # the oracle's in-edge list
            in_ptr = torch.from_numpy(np.ascontiguousarray(ip, np.int32)).cuda()
            in_src = torch.from_numpy(np.ascontiguousarray(isrc if g.m else np.zeros(1), np.int32)).cuda()
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
                got_bits = np.unpackbits(mask.cpu().numpy().view(np.uint8), bitorder="little")[:g.m]
                got_ptr = sp_ptr.cpu().numpy()
                nnz = int(sp_nnz.cpu().numpy()[0])
                got_src = sp_src.cpu().numpy()[:nnz]
                # against the oracle: flags, packed row pointers and sources
                want = oracle.sample_mask(g.n, ip, isrc, sigma, seed, symmetric=g.symmetric)
                assert np.array_equal(got_bits, want)
                cs = np.concatenate([[0], np.cumsum(want.astype(np.int64))])
                assert np.array_equal(got_ptr, cs[ip])
                assert np.array_equal(got_src, isrc[want.astype(bool)])
                # against the allocating entry point on the same graph
                gg.gg_sample_edges(h, sigma, seed)
                assert np.array_equal(got_bits, gg.mask_bits(h, g.m))
                assert np.array_equal(got_ptr, gg.result_array(h, gg.GG_RESULT_SPARSE_PTR))
                assert np.array_equal(got_src, gg.result_array(h, gg.GG_RESULT_SPARSE_SRC))
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


@pytest.mark.gpu
def test_noalloc_sampler_rejects_row_pointers_on_the_device():
    """Row pointers that do not end at m (or decrease) are caught on the
    device: no flag or packed entry is written and *sp_nnz = 0xFFFFFFFF; a
    valid call afterwards works as before."""
    import torch
    gg = gc.lib()
    n, m = 5, 6
    src = torch.tensor([0, 1, 2, 3, 4, 0], dtype=torch.int32, device="cuda")
    mask = torch.full((1,), 0x55, dtype=torch.int32, device="cuda")
    sp_ptr = torch.full((n + 1,), -7, dtype=torch.int32, device="cuda")
    sp_src = torch.full((m,), -7, dtype=torch.int32, device="cuda")
    sp_nnz = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for bad in ([0, 2, 1, 4, 5, 6], [0, 1, 2, 3, 4, 5], [1, 2, 3, 4, 5, 6]):
        rp = torch.tensor(bad, dtype=torch.int32, device="cuda")
        gg.gg_sample_csc_noalloc(n, m, rp, src, 0.5, 3, False, mask, sp_ptr, sp_src, sp_nnz, stream)
        torch.cuda.synchronize()
        assert int(sp_nnz.cpu()[0]) == -1
        assert int(mask.cpu()[0]) == 0x55
        assert (sp_ptr.cpu() == -7).all() and (sp_src.cpu() == -7).all()
    rp = torch.tensor([0, 2, 2, 4, 5, 6], dtype=torch.int32, device="cuda")
    gg.gg_sample_csc_noalloc(n, m, rp, src, 1.0, 3, False, mask, sp_ptr, sp_src, sp_nnz, stream)
    torch.cuda.synchronize()
    assert int(sp_nnz.cpu()[0]) == m
    assert sp_ptr.cpu().tolist() == [0, 2, 2, 4, 5, 6] and sp_src.cpu().tolist() == src.cpu().tolist()
