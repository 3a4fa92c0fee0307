"""Textbook references used to pin the oracle on tiny graphs.

Each is a different algorithm from the oracle's synchronous pull iteration:
Dijkstra with a binary heap, FIFO breadth-first search, union-find, and
PageRank as a dense FP64 matrix power iteration. None of them shares code with
``oracle/`` or with the CUDA library.
"""
import heapq

import numpy as np

INF = 0xFFFFFFFF


def arcs_of(g):
    """(src, dst, w) triples of a graphgen.Graph in CSR order."""
    out = []
    for s in range(g.n):
        for e in range(g.rowptr[s], g.rowptr[s + 1]):
            w = 1 if g.weights is None else int(g.weights[e])
            out.append((s, int(g.colidx[e]), w))
    return out


def dijkstra(g, source):
    adj = [[] for _ in range(g.n)]
    for s, d, w in arcs_of(g):
        adj[s].append((d, w))
    dist = [None] * g.n
    heap = [(0, source)]
    while heap:
        dv, v = heapq.heappop(heap)
        if dist[v] is not None:
            continue
        dist[v] = dv
        for u, w in adj[v]:
            if dist[u] is None:
                heapq.heappush(heap, (dv + w, u))
    return np.array([INF if x is None else x for x in dist], np.uint64).astype(np.uint32)


def bfs_levels(g, source):
    adj = [[] for _ in range(g.n)]
    for s, d, _ in arcs_of(g):
        adj[s].append(d)
    lvl = [None] * g.n
    lvl[source] = 0
    queue = [source]
    head = 0
    while head < len(queue):
        v = queue[head]
        head += 1
        for u in adj[v]:
            if lvl[u] is None:
                lvl[u] = lvl[v] + 1
                queue.append(u)
    return np.array([INF if x is None else x for x in lvl], np.uint64).astype(np.uint32)


def cc_min_labels(g):
    """Union-find over the (undirected) arcs; every vertex gets the smallest
    vertex id of its component."""
    parent = list(range(g.n))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for s, d, _ in arcs_of(g):
        a, b = find(s), find(d)
        if a != b:
            parent[max(a, b)] = min(a, b)
    roots = [find(v) for v in range(g.n)]
    smallest = {}
    for v in range(g.n):
        r = roots[v]
        smallest[r] = min(smallest.get(r, v), v)
    return np.array([smallest[roots[v]] for v in range(g.n)], np.uint32)


def pagerank_dense(g, damping, iters):
    """x_{t+1} = (1-d)/N + d * A^T D^-1 x_t with A counting parallel arcs and
    D the full out-degree; vertices without out-arcs pass nothing on."""
    n = g.n
    d = float(np.float32(damping))
    A = np.zeros((n, n), np.float64)
    for s, t, _ in arcs_of(g):
        A[s, t] += 1.0
    outdeg = A.sum(axis=1)
    P = np.zeros_like(A)
    nz = outdeg > 0
    P[nz] = A[nz] / outdeg[nz, None]
    x = np.full(n, 1.0 / n)
    for _ in range(iters):
        x = (1.0 - d) / n + d * (P.T @ x)
    return x


def ppr_dense(g, damping, iters, source):
    """Personalized PageRank by dense power iteration:
    x_0 = e_s, x_{t+1} = (1-d) e_s + d * A^T D^-1 x_t."""
    n = g.n
    d = float(np.float32(damping))
    A = np.zeros((n, n), np.float64)
    for s, t, _ in arcs_of(g):
        A[s, t] += 1.0
    outdeg = A.sum(axis=1)
    P = np.zeros_like(A)
    nz = outdeg > 0
    P[nz] = A[nz] / outdeg[nz, None]
    e = np.zeros(n)
    e[source] = 1.0
    x = e.copy()
    for _ in range(iters):
        x = (1.0 - d) * e + d * (P.T @ x)
    return x


def graphguess_pagerank_rational(g, damping, iters, initial_flags, alpha, theta, policy="gg",
                                 renorm=False, share=False):
    """GraphGuess PageRank (Alg. 2, Sec. 3.4) on a tiny graph in exact rational
    arithmetic, written as a different program from the oracle: in-edges
    listed by sorting the arcs on (destination, source) with Python's stable
    sort, ranks as fractions, each iteration a fresh pass over that list.

    * Iteration i of policy "gg" is a correction when i mod (alpha+1) = alpha,
      otherwise approximate; policy "sms" is approximate before alpha, a
      correction at alpha and accurate (every arc, flags kept) after it.
    * Approximate: u gathers rank(v)/outdeg(v) over its flagged in-arcs only
      (the full out-degree: the graph itself is unchanged); accurate and
      correction iterations gather over every in-arc.
    * A correction gives in-arc e of u the influence (acc_after - acc_before)
      / acc_after of the running sum over u's in-arcs in source order (0 when
      the sum is 0), and e stays active iff that influence exceeds theta.
    * rank'(u) = (1 - d)/N + d * sum (synchronous), rank_0 = 1/N.
    * renorm: an approximate iteration divides by the source's number of
      active out-arcs instead (none active: it passes nothing on).
    * share: a correction keeps arc e of u iff its contribution exceeds theta
      times the total over all of u's in-arcs (order-free; total 0: 0 > theta).

    initial_flags: dict (src, dst, CSR index) -> 0/1 from the sampler.
    Returns (ranks float64[n], flags uint8 in (dst, src)-sorted order,
    smallest |influence - theta| met at a correction)."""
    from fractions import Fraction
    n = g.n
    arcs = arcs_of(g)
    outdeg = [0] * n
    for s, _, _ in arcs:
        outdeg[s] += 1
    order = sorted(range(len(arcs)), key=lambda e: (arcs[e][1], arcs[e][0]))
    flag = {e: initial_flags[e] for e in range(len(arcs))}
    d = Fraction(float(np.float32(damping)))
    th = Fraction(float(np.float32(theta)))
    rank = [Fraction(1, n)] * n
    margin = None
    for i in range(iters):
        if policy == "gg":
            mode = "correct" if i % (alpha + 1) == alpha else "approx"
        else:
            mode = "approx" if i < alpha else ("correct" if i == alpha else "accurate")
        deg = outdeg
        if renorm and mode == "approx":
            deg = [0] * n
            for e in range(len(arcs)):
                if flag[e]:
                    deg[arcs[e][0]] += 1
        acc = [Fraction(0)] * n
        contrib = {}
        for e in order:
            s, t, _ = arcs[e]
            if mode == "approx" and not flag[e]:
                continue
            contrib[e] = rank[s] / deg[s]
            before = acc[t]
            acc[t] = before + contrib[e]
            if mode == "correct" and not share:
                infl = (acc[t] - before) / acc[t] if acc[t] != 0 else Fraction(0)
                gap = abs(infl - th)
                margin = gap if margin is None or gap < margin else margin
                flag[e] = 1 if infl > th else 0
        if mode == "correct" and share:
            for e in order:
                t = arcs[e][1]
                gap = abs(contrib[e] - th * acc[t]) / (acc[t] if acc[t] != 0 else 1)
                margin = gap if margin is None or gap < margin else margin
                flag[e] = 1 if (contrib[e] > th * acc[t] if acc[t] != 0 else 0 > th) else 0
        rank = [(1 - d) / n + d * acc[u] for u in range(n)]
    return (np.array([float(r) for r in rank]), np.array([flag[e] for e in order], np.uint8),
            None if margin is None else float(margin))


def graphguess_min_replica(g, app, source, iters, initial_flags, alpha, theta, policy="gg", strict=False):
    """GraphGuess for the min applications (SSSP, BFS, CC) on a tiny graph,
    written as a different program from the oracle: in-edges from a stable
    sort of the arcs on (destination, source), values in Python integers
    (unbounded, so saturation is an explicit comparison), influence as an
    exact fraction.

    * Initial values: SSSP / BFS: 0 at the source, unreached elsewhere; CC: the
      vertex id. Unreached = 2^32 - 1, and a candidate that would reach it is
      no candidate.
    * Candidates of arc v->u: val(v) + w (SSSP), val(v) + 1 (BFS), val(v) (CC);
      none when v is unreached.
    * Modes as in the PageRank replica ("gg": correction when i mod (alpha+1)
      = alpha; "sms": approximate before alpha, correction at alpha, accurate
      after; "sp": always approximate).
    * A correction gives every arc with a candidate the influence of the
      running minimum over u's in-arcs in source order: 1 for the first
      candidate, (acc - cand) / acc when the candidate lowers the minimum
      (CC: 1), 0 otherwise; the arc stays active iff influence > theta. Arcs
      without a candidate keep their flag (strict: they are cleared).
    * new(u) = min(old(u), acc); the run stops after a correction or accurate
      iteration that changed nothing (SP: after any quiet iteration).

    Returns (values uint32[n], flags uint8 in (dst, src)-sorted order)."""
    from fractions import Fraction
    inf = INF
    n = g.n
    arcs = arcs_of(g)
    order = sorted(range(len(arcs)), key=lambda e: (arcs[e][1], arcs[e][0]))
    flag = {e: initial_flags[e] for e in range(len(arcs))}
    th = Fraction(float(np.float32(theta)))
    if app == "cc":
        val = list(range(n))
    else:
        val = [inf] * n
        val[source] = 0
    for i in range(iters):
        if policy == "gg":
            mode = "correct" if i % (alpha + 1) == alpha else "approx"
        elif policy == "sms":
            mode = "approx" if i < alpha else ("correct" if i == alpha else "accurate")
        else:
            mode = "approx"
        acc = [inf] * n
        for e in order:
            s, t, w = arcs[e]
            if mode == "approx" and not flag[e]:
                continue
            if val[s] == inf:
                cand = None
            else:
                cand = val[s] + (w if app == "sssp" else 1 if app == "bfs" else 0)
                if cand >= inf:
                    cand = None
            if cand is None:
                if mode == "correct" and strict:
                    flag[e] = 0
                continue
            if mode == "correct":
                if cand < acc[t]:
                    infl = Fraction(1) if (acc[t] == inf or app == "cc") else Fraction(acc[t] - cand, acc[t])
                else:
                    infl = Fraction(0)
                flag[e] = 1 if infl > th else 0
            if cand < acc[t]:
                acc[t] = cand
        new = [min(val[u], acc[u]) for u in range(n)]
        changed = new != val
        val = new
        if not changed and (mode != "approx" or policy == "sp"):
            break
    return np.array(val, np.uint32), np.array([flag[e] for e in order], np.uint8)
