"""Host side of the batched-serving workload (CPU): graph scales, query mix
and sources, at reduced scales."""
import numpy as np

from paper_2104_10039_gb300 import serve


def test_workload_composition():
    graphs, queries, scales = serve.make_workload(n_graphs=64, n_queries=512, scale_lo=6, scale_hi=12)
    assert len(graphs) == 64 and len(queries) == 512
    assert scales.min() >= 6 and scales.max() <= 12
    # scale = lo + floor((hi - lo + 1) u^2): small graphs are the more frequent
    counts = np.bincount(scales - 6, minlength=7)
    assert counts[:2].sum() > counts[-2:].sum()
    for g, s in zip(graphs, scales):
        assert g.n == 1 << int(s) and g.m == 16 * g.n and g.weights is not None
    apps = [q[1] for q in queries]
    assert (apps.count("bfs"), apps.count("sssp"), apps.count("ppr")) == (171, 171, 170)   # one third each
    for gi, app, src, iters in queries:
        g = graphs[gi]
        assert g.rowptr[src + 1] > g.rowptr[src]           # the source has out-arcs
        assert iters == (20 if app == "ppr" else 0)
    # the same seed gives the same workload
    _, q2, s2 = serve.make_workload(n_graphs=64, n_queries=512, scale_lo=6, scale_hi=12)
    assert q2 == queries and np.array_equal(s2, scales)
