"""Helpers for the GPU parity tests: load a graphgen graph through the C ABI,
run it, and fetch results. Oracle-side expectations come from ``oracle/``."""
import numpy as np

import graphgen
import oracle


def lib():
    from paper_2104_10039_gb300 import build
    build.build()
    from paper_2104_10039_gb300 import gg
    return gg


def load(gg, g: graphgen.Graph, device_ptrs=False):
    flags = gg.GG_SYMMETRIC if g.symmetric else gg.GG_DIRECTED
    if device_ptrs:
        import torch
        rp = torch.from_numpy(g.rowptr).cuda()
        ci = torch.from_numpy(g.colidx if g.m else np.zeros(1, np.int32)).cuda()
        w = None if g.weights is None else torch.from_numpy(g.weights.view(np.int32)).cuda()
        h = gg.gg_load_csr(g.n, g.m, rp, ci, w, flags | gg.GG_DEVICE_PTRS)
        torch.cuda.synchronize()
        return h
    return gg.gg_load_csr(g.n, g.m, g.rowptr, g.colidx if g.m else np.zeros(1, np.int32),
                          g.weights, flags)


def rel_l1(got, want):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    return float(np.abs(got - want).sum() / max(np.abs(want).sum(), 1e-300))


def correction_indices(policy, alpha, T):
    idx = []
    for i in range(T):
        if oracle.iteration_mode(policy, alpha, i) == oracle.MODE_CORRECTION:
            idx.append(i)
    return idx


def gpu_run(gg, h, g, app, policy, sigma=0.5, alpha=4, theta=0.05, T=20, source=0, seed=1,
            flags=0, damping=0.85, epsilon=0.0, trigger_ratio=0.5):
    p = gg.make_params(alpha=alpha, theta=theta, max_iters=T, damping=damping, epsilon=epsilon,
                       source=source, seed=seed, flags=flags, trigger_ratio=trigger_ratio)
    gg.gg_run(h, app, sigma, policy, p)
    vals = gg.values(h, app)
    mask = gg.mask_bits(h, g.m) if policy != "exact" else None
    return vals, mask, gg.stats(h)


def pagerank_with_replay(gg, h, g, policy, sigma, alpha, theta, T, seed, tol=1e-5):
    """GPU PageRank plus the oracle run that adopts the GPU's post-correction
    flags (mask replay); returns (gpu_values, oracle_result)."""
    masks = []
    for c in correction_indices(policy, alpha, T):
        _, mk, _ = gpu_run(gg, h, g, "pagerank", policy, sigma, alpha, theta, T=c + 1, seed=seed)
        masks.append(mk)
    vals, _, st = gpu_run(gg, h, g, "pagerank", policy, sigma, alpha, theta, T=T, seed=seed)
    ref = oracle.run(g.n, g.rowptr, g.colidx, app="pagerank", policy=policy, sigma=sigma, seed=seed,
                     alpha=alpha, theta=theta, max_iters=T, symmetric=g.symmetric,
                     replay_masks=masks, replay_tol=tol, nthreads=0)
    return vals, ref, st
