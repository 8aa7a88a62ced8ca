"""Seeded synthetic graphs, source lists and the CSR builder.

This module produces inputs only. It computes no distance, path count or
dependency, so the tests, the benchmark and the CPU oracle checks can all draw
from it without sharing any of the method's arithmetic.

Randomness comes from a counter-based splitmix64 stream (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): value i of a
stream keyed by ``key`` is ``mix64(key + (i + 1) * 0x9E3779B97F4A7C15)``. Every
draw is plain uint64 arithmetic in numpy, so the same seed gives the same bytes
on x86 and Arm and on any numpy version.

Graph model (Section 1.1 of the paper): undirected, vertices 0..n-1, positive
integer edge weights (unweighted = all ones). The CSR holds both arcs of every
undirected edge; self-loops and duplicate edges are rejected.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
BASE_SEED = 20080919


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class Stream:
    """Counter-based splitmix64 stream; ``tag`` separates independent streams."""

    def __init__(self, seed: int, tag: int = 0):
        with np.errstate(over="ignore"):
            k = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * _GOLDEN + np.uint64(tag & 0xFFFFFFFFFFFFFFFF)
        self.key = _mix64(np.asarray([k], dtype=np.uint64))[0]
        self.ctr = 0

    def u64(self, k: int) -> np.ndarray:
        idx = np.arange(self.ctr + 1, self.ctr + k + 1, dtype=np.uint64)
        self.ctr += k
        with np.errstate(over="ignore"):
            return _mix64(self.key + idx * _GOLDEN)

    def uniform(self, k: int) -> np.ndarray:
        """k doubles in [0, 1) with 53 random bits each."""
        return (self.u64(k) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def below(self, k: int, bound: int) -> np.ndarray:
        """k integers in [0, bound), bound < 2**32 (multiply-shift on the top 32 bits)."""
        if not 0 < bound < (1 << 32):
            raise ValueError("bound out of range")
        hi = self.u64(k) >> np.uint64(32)
        with np.errstate(over="ignore"):
            return ((hi * np.uint64(bound)) >> np.uint64(32)).astype(np.int64)

    def permutation(self, n: int) -> np.ndarray:
        return np.argsort(self.u64(n), kind="stable").astype(np.int64)


@dataclasses.dataclass
class Graph:
    """Graph in CSR form. Undirected (the default): both arcs of each edge
    stored. Directed: each arc once, in the row of its tail."""

    n: int
    row_ptr: np.ndarray  # int32 [n+1]
    col: np.ndarray  # int32 [arcs], heads of each row sorted ascending
    w: np.ndarray | None  # int32 [arcs] arc weights (None = unweighted)
    name: str = ""
    directed: bool = False

    @property
    def m(self) -> int:
        """Undirected edges, or arcs of a directed graph."""
        return int(self.col.shape[0]) if self.directed else int(self.col.shape[0]) // 2

    @property
    def weighted(self) -> bool:
        return self.w is not None

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))

    def edges(self):
        """Undirected edge list (u < v) with weights (or None)."""
        src = np.repeat(np.arange(self.n, dtype=np.int64), self.degrees())
        keep = src < self.col
        return src[keep], self.col[keep].astype(np.int64), (None if self.w is None else self.w[keep].astype(np.int64))


def csr_from_edges(n: int, u, v, w=None, name: str = "") -> Graph:
    """Build a CSR from an undirected edge list.

    Raises ValueError on out-of-range ids, self-loops, duplicate edges or
    non-positive weights: the paper's model has none of them.
    """
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    if u.shape != v.shape:
        raise ValueError("u and v differ in length")
    if n < 0 or n >= (1 << 31):
        raise ValueError("n out of range")
    if u.size and (u.min() < 0 or v.min() < 0 or u.max() >= n or v.max() >= n):
        raise ValueError("vertex id out of range")
    if np.any(u == v):
        raise ValueError("self-loop")
    a, b = np.minimum(u, v), np.maximum(u, v)
    key = a * n + b
    if np.unique(key).size != key.size:
        raise ValueError("duplicate edge")
    if 2 * u.size >= (1 << 31):
        raise ValueError("too many edges for int32 CSR")
    src = np.concatenate([u, v])
    dst = np.concatenate([v, u])
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(src, minlength=n), out=row_ptr[1:])
    ww = None
    if w is not None:
        w = np.asarray(w, dtype=np.int64)
        if w.shape != u.shape:
            raise ValueError("weights differ in length")
        if w.size and (w.min() <= 0 or w.max() >= (1 << 31)):
            raise ValueError("weights must be positive int32")
        ww = np.concatenate([w, w])[order].astype(np.int32)
    return Graph(n, row_ptr.astype(np.int32), dst.astype(np.int32), ww, name)


def csr_from_arcs(n: int, u, v, w=None, name: str = "") -> Graph:
    """Build a directed CSR from an arc list (u -> v).

    Raises ValueError on out-of-range ids, self-loops, duplicate arcs or
    non-positive weights.
    """
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    if u.shape != v.shape:
        raise ValueError("u and v differ in length")
    if n < 0 or n >= (1 << 31):
        raise ValueError("n out of range")
    if u.size and (u.min() < 0 or v.min() < 0 or u.max() >= n or v.max() >= n):
        raise ValueError("vertex id out of range")
    if np.any(u == v):
        raise ValueError("self-loop")
    key = u * n + v
    if np.unique(key).size != key.size:
        raise ValueError("duplicate arc")
    if u.size >= (1 << 31):
        raise ValueError("too many arcs for int32 CSR")
    order = np.lexsort((v, u))
    src, dst = u[order], v[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(src, minlength=n), out=row_ptr[1:])
    ww = None
    if w is not None:
        w = np.asarray(w, dtype=np.int64)
        if w.shape != u.shape:
            raise ValueError("weights differ in length")
        if w.size and (w.min() <= 0 or w.max() >= (1 << 31)):
            raise ValueError("weights must be positive int32")
        ww = w[order].astype(np.int32)
    return Graph(n, row_ptr.astype(np.int32), dst.astype(np.int32), ww, name, directed=True)


def transpose(g: Graph) -> Graph:
    """The in-arc CSR of a directed graph: row v lists the tails u of the arcs
    (u, v), with their weights."""
    src = np.repeat(np.arange(g.n, dtype=np.int64), g.degrees())
    t = csr_from_arcs(g.n, g.col.astype(np.int64), src, None if g.w is None else g.w, g.name + "^T")
    return t


def directed_path(n: int) -> Graph:
    """0 -> 1 -> ... -> n-1."""
    return csr_from_arcs(n, np.arange(n - 1), np.arange(1, n), name=f"dpath{n}")


def directed_cycle(n: int) -> Graph:
    """0 -> 1 -> ... -> n-1 -> 0."""
    a = np.arange(n)
    return csr_from_arcs(n, a, (a + 1) % n, name=f"dcycle{n}")


def directed_random(n: int, p: float, seed: int, wmax: int = 0) -> Graph:
    """Each ordered pair (u, v), u != v, an arc with probability p (seeded);
    weights U{1..wmax} when wmax > 0."""
    st = Stream(seed)
    r = st.uniform(n * n).reshape(n, n)
    np.fill_diagonal(r, 1.0)
    u, v = np.nonzero(r < p)
    w = None if wmax <= 0 else 1 + st.below(u.size, wmax)
    return csr_from_arcs(n, u, v, w, name=f"dG({n},{p})")


def kkp_tripartite(n: int) -> Graph:
    """Section 2's directed tripartite graph on u_i, v_j, w_k (0 <= i,j,k < n):
    arcs u_i -> v_j and v_j -> w_k, weighted so that every shortest u_i - w_k
    path goes through v_0 alone: weight 1 on arcs into and out of v_0, 2 on
    the others (paths through v_0 have length 2, all others 4). Vertex ids:
    u_i = i, v_j = n + j, w_k = 2n + k."""
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    i, j = i.ravel(), j.ravel()
    uv_u, uv_v, uv_w = i, n + j, np.where(j == 0, 1, 2)
    vw_u, vw_v, vw_w = n + i, 2 * n + j, np.where(i == 0, 1, 2)
    return csr_from_arcs(3 * n, np.concatenate([uv_u, vw_u]), np.concatenate([uv_v, vw_v]),
                         np.concatenate([uv_w, vw_w]), name=f"kkp{n}")


def _dedupe_pairs(a: np.ndarray, b: np.ndarray, n: int):
    """Keep the first occurrence of each undirected pair (order preserved)."""
    key = np.minimum(a, b) * n + np.maximum(a, b)
    _, first = np.unique(key, return_index=True)
    first.sort()
    return a[first], b[first]


# ---------------------------------------------------------------- workloads

def er_hamiltonian(n: int = 1024, m: int = 4096, seed: int = BASE_SEED + 1) -> Graph:
    """G(n, m): m distinct uniform pairs (no loops), plus the edges of a random
    Hamiltonian path so the graph is connected (duplicates dropped)."""
    rs = Stream(seed, 1)
    us, vs = np.empty(0, np.int64), np.empty(0, np.int64)
    while us.size < m:
        k = 2 * (m - us.size) + 64
        a, b = rs.below(k, n), rs.below(k, n)
        keep = a != b
        us, vs = _dedupe_pairs(np.concatenate([us, a[keep]]), np.concatenate([vs, b[keep]]), n)
    us, vs = us[:m], vs[:m]
    perm = Stream(seed, 2).permutation(n)
    us, vs = _dedupe_pairs(np.concatenate([us, perm[:-1]]), np.concatenate([vs, perm[1:]]), n)
    return csr_from_edges(n, us, vs, name=f"er_n{n}_m{m}")


def largest_component(n: int, u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Vertex ids of the largest connected component (ties: lowest component label)."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    adj = sp.coo_matrix((np.ones(u.size, dtype=np.int8), (u, v)), shape=(n, n)).tocsr()
    _, lab = connected_components(adj, directed=False)
    counts = np.bincount(lab)
    return np.nonzero(lab == int(np.argmax(counts)))[0]


def rmat_lcc(scale: int = 16, edge_factor: int = 16, abcd=(0.57, 0.19, 0.19, 0.05),
             seed: int = BASE_SEED + 2) -> Graph:
    """R-MAT (Chakrabarti, Zhan, Faloutsos 2004): edge_factor * 2**scale generated
    edges, seeded vertex relabelling, symmetrised, self-loops and duplicates
    dropped, restricted to the largest connected component and relabelled in
    increasing id order."""
    a, b, c, _ = abcd
    n = 1 << scale
    ne = edge_factor * n
    rs = Stream(seed, 3)
    src = np.zeros(ne, dtype=np.int64)
    dst = np.zeros(ne, dtype=np.int64)
    for bit in range(scale):
        r = rs.uniform(ne)
        sbit = r >= a + b
        dbit = ((r >= a) & (r < a + b)) | (r >= a + b + c)
        src |= sbit.astype(np.int64) << bit
        dst |= dbit.astype(np.int64) << bit
    perm = Stream(seed, 4).permutation(n)
    src, dst = perm[src], perm[dst]
    keep = src != dst
    src, dst = _dedupe_pairs(src[keep], dst[keep], n)
    comp = largest_component(n, src, dst)
    newid = np.full(n, -1, dtype=np.int64)
    newid[comp] = np.arange(comp.size)
    keep = newid[src] >= 0
    return csr_from_edges(comp.size, newid[src[keep]], newid[dst[keep]],
                          name=f"rmat_s{scale}_ef{edge_factor}_lcc")


def rmat_directed(scale: int = 16, edge_factor: int = 16, abcd=(0.57, 0.19, 0.19, 0.05),
                  seed: int = BASE_SEED + 2) -> Graph:
    """The same R-MAT draw as rmat_lcc, kept directed: each generated pair is
    the arc u -> v (self-loops and repeated arcs dropped), restricted to the
    vertices of the largest weakly connected component and relabelled."""
    a, b, c, _ = abcd
    n = 1 << scale
    ne = edge_factor * n
    rs = Stream(seed, 3)
    src = np.zeros(ne, dtype=np.int64)
    dst = np.zeros(ne, dtype=np.int64)
    for bit in range(scale):
        r = rs.uniform(ne)
        sbit = r >= a + b
        dbit = ((r >= a) & (r < a + b)) | (r >= a + b + c)
        src |= sbit.astype(np.int64) << bit
        dst |= dbit.astype(np.int64) << bit
    perm = Stream(seed, 4).permutation(n)
    src, dst = perm[src], perm[dst]
    keep = src != dst
    src, dst = src[keep], dst[keep]
    _, first = np.unique(src * n + dst, return_index=True)
    first.sort()
    src, dst = src[first], dst[first]
    comp = largest_component(n, *_dedupe_pairs(src, dst, n))
    newid = np.full(n, -1, dtype=np.int64)
    newid[comp] = np.arange(comp.size)
    keep = newid[src] >= 0
    return csr_from_arcs(comp.size, newid[src[keep]], newid[dst[keep]],
                         name=f"rmat_s{scale}_ef{edge_factor}_directed")


def gnp_weighted(n: int = 4096, p: float = 0.05, wmax: int = 10, seed: int = BASE_SEED + 6) -> Graph:
    """G(n, p) as gnp(), every undirected edge with an integer weight uniform in [1, wmax]."""
    g = gnp(n, p, seed)
    u, v, _ = g.edges()
    w = 1 + Stream(seed, 8).below(u.size, wmax)
    return csr_from_edges(n, u, v, w, name=f"gnp_n{n}_p{p}_w{wmax}")


def grid_longrange(side: int = 512, frac: float = 0.05, wmax: int = 100,
                   seed: int = BASE_SEED + 3) -> Graph:
    """side x side 4-neighbour grid plus round(frac * grid_edges) uniform random
    long-range edges (no loops, no duplicates of any edge); every undirected
    edge gets an integer weight uniform in [1, wmax]."""
    n = side * side
    r, c = np.divmod(np.arange(n, dtype=np.int64), side)
    hu = np.nonzero(c < side - 1)[0]
    vu = np.nonzero(r < side - 1)[0]
    gu = np.concatenate([hu, vu])
    gv = np.concatenate([hu + 1, vu + side])
    ng = gu.size
    k = int(round(frac * ng))
    rs = Stream(seed, 5)
    existing = set((np.minimum(gu, gv) * n + np.maximum(gu, gv)).tolist())
    lu, lv = [], []
    while len(lu) < k:
        a, b = rs.below(2 * k, n), rs.below(2 * k, n)
        for x, y in zip(a.tolist(), b.tolist()):
            if x == y:
                continue
            key = min(x, y) * n + max(x, y)
            if key in existing:
                continue
            existing.add(key)
            lu.append(x)
            lv.append(y)
            if len(lu) == k:
                break
    u = np.concatenate([gu, np.asarray(lu, dtype=np.int64)])
    v = np.concatenate([gv, np.asarray(lv, dtype=np.int64)])
    w = Stream(seed, 6).below(u.size, wmax) + 1
    return csr_from_edges(n, u, v, w, name=f"grid{side}_lr{frac}_w{wmax}")


def induced_subgrid(g: Graph, side: int, k: int) -> Graph:
    """Induced subgraph on the top-left k x k block of a side x side grid graph
    (grid and long-range edges inside the block), ids r*k + c."""
    u, v, w = g.edges()
    ru, cu = np.divmod(u, side)
    rv, cv = np.divmod(v, side)
    keep = (ru < k) & (cu < k) & (rv < k) & (cv < k)
    return csr_from_edges(k * k, ru[keep] * k + cu[keep], rv[keep] * k + cv[keep],
                          None if w is None else w[keep], name=f"{g.name}_sub{k}")


def gnp(n: int = 8192, p: float = 0.05, seed: int = BASE_SEED + 4) -> Graph:
    """G(n, p): every pair i < j is an edge with probability p (row by row)."""
    rs = Stream(seed, 7)
    us, vs = [], []
    rows = max(1, (1 << 22) // max(n, 1))
    for i0 in range(0, n, rows):
        for i in range(i0, min(n, i0 + rows)):
            cnt = n - 1 - i
            if cnt <= 0:
                continue
            hit = np.nonzero(rs.uniform(cnt) < p)[0]
            us.append(np.full(hit.size, i, dtype=np.int64))
            vs.append(hit + i + 1)
    u = np.concatenate(us) if us else np.empty(0, np.int64)
    v = np.concatenate(vs) if vs else np.empty(0, np.int64)
    return csr_from_edges(n, u, v, name=f"gnp_n{n}_p{p}")


def barabasi_albert(n: int, m: int = 3, seed: int = BASE_SEED + 5) -> Graph:
    """Barabasi-Albert growth from K_{m+1}: each new vertex joins m distinct
    existing vertices chosen with probability proportional to degree."""
    if n <= m:
        raise ValueError("n must exceed m")
    rs = Stream(seed, 8)
    us, vs = [], []
    ends = []
    for i in range(m + 1):
        for j in range(i + 1, m + 1):
            us.append(i)
            vs.append(j)
            ends += [i, j]
    buf = rs.u64(8 * m * n + 64)
    pos = 0
    for x in range(m + 1, n):
        chosen = []
        while len(chosen) < m:
            r = int(buf[pos]) >> 32
            pos += 1
            if pos == buf.size:
                buf, pos = rs.u64(8 * m * n), 0
            t = ends[(r * len(ends)) >> 32]
            if t not in chosen:
                chosen.append(t)
        for t in chosen:
            us.append(x)
            vs.append(t)
            ends += [x, t]
    return csr_from_edges(n, us, vs, name=f"ba_n{n}_m{m}")


def many_graph_sizes(count: int = 2000, nmin: int = 50, nmax: int = 5000,
                     seed: int = BASE_SEED + 5) -> np.ndarray:
    """Vertex counts of the many-graph set: n = round(exp(U(ln nmin, ln nmax)))."""
    u = Stream(seed, 9).uniform(count)
    return np.rint(np.exp(math.log(nmin) + u * (math.log(nmax) - math.log(nmin)))).astype(np.int64)


def many_graph(i: int, n: int, seed: int = BASE_SEED + 5) -> Graph:
    """Member i of the many-graph set with n vertices. Even index: G(n, 3n)
    plus a Hamiltonian path; odd index: BA(m=3)."""
    if i % 2 == 0:
        return er_hamiltonian(n, min(3 * n, n * (n - 1) // 2 - n), seed * 7919 + i)
    return barabasi_albert(n, 3, seed * 7919 + i)


def many_graphs(count: int = 2000, nmin: int = 50, nmax: int = 5000,
                seed: int = BASE_SEED + 5) -> list[Graph]:
    """The many-graph set: member i is many_graph(i, n_i)."""
    ns = many_graph_sizes(count, nmin, nmax, seed)
    return [many_graph(i, n, seed) for i, n in enumerate(ns.tolist())]


def sample_sources(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct source ids uniform without replacement, in draw order."""
    if k > n:
        raise ValueError("k > n")
    return Stream(seed, 10).permutation(n)[:k].astype(np.int32)


# ------------------------------------------------------- closed-form graphs

def path_graph(n: int) -> Graph:
    i = np.arange(n - 1)
    return csr_from_edges(n, i, i + 1, name=f"P{n}")


def cycle_graph(n: int) -> Graph:
    i = np.arange(n)
    return csr_from_edges(n, i, (i + 1) % n, name=f"C{n}")


def star_graph(n: int) -> Graph:
    """Centre 0 joined to leaves 1..n-1."""
    i = np.arange(1, n)
    return csr_from_edges(n, np.zeros_like(i), i, name=f"S{n}")


def complete_graph(n: int) -> Graph:
    a, b = np.triu_indices(n, 1)
    return csr_from_edges(n, a, b, name=f"K{n}")


def complete_bipartite(a: int, b: int) -> Graph:
    """Side A = 0..a-1, side B = a..a+b-1."""
    x, y = np.meshgrid(np.arange(a), np.arange(a, a + b), indexing="ij")
    return csr_from_edges(a + b, x.ravel(), y.ravel(), name=f"K{a},{b}")


def grid_graph(k: int, w: int | None = None) -> Graph:
    """k x k 4-neighbour grid, ids r*k + c, all weights w (None = unweighted)."""
    n = k * k
    r, c = np.divmod(np.arange(n), k)
    hu = np.nonzero(c < k - 1)[0]
    vu = np.nonzero(r < k - 1)[0]
    u = np.concatenate([hu, vu])
    v = np.concatenate([hu + 1, vu + k])
    return csr_from_edges(n, u, v, None if w is None else np.full(u.size, w), name=f"grid{k}")


def layered_biclique(layers: int, width: int) -> Graph:
    """Vertex 0, then `layers` layers of `width` vertices; vertex 0 joins all of
    layer 1 and consecutive layers are complete bipartite."""
    us, vs = [], []
    prev = [0]
    nxt = 1
    for _ in range(layers):
        cur = list(range(nxt, nxt + width))
        nxt += width
        for a in prev:
            for b in cur:
                us.append(a)
                vs.append(b)
        prev = cur
    return csr_from_edges(nxt, us, vs, name=f"biclique{layers}x{width}")


def random_small(n: int, p: float, seed: int, wmax: int = 1, connect: bool = True) -> Graph:
    """Small random graph for exhaustive checks: G(n, p), optionally plus a
    random spanning path, weights uniform in [1, wmax] (wmax=1: unweighted)."""
    rs = Stream(seed, 11)
    a, b = np.triu_indices(n, 1)
    keep = rs.uniform(a.size) < p
    u, v = a[keep], b[keep]
    if connect and n > 1:
        perm = Stream(seed, 12).permutation(n)
        u, v = _dedupe_pairs(np.concatenate([u, perm[:-1]]), np.concatenate([v, perm[1:]]), n)
    w = None if wmax <= 1 else Stream(seed, 13).below(u.size, wmax) + 1
    return csr_from_edges(n, u, v, w, name=f"small{n}_{seed}")


def from_adjacency_bits(n: int, bits: int) -> Graph:
    """Graph whose edge set is bit k of `bits` over the pairs (i<j) in
    lexicographic order (used to enumerate every labelled graph)."""
    a, b = np.triu_indices(n, 1)
    sel = np.array([(bits >> k) & 1 for k in range(a.size)], dtype=bool)
    return csr_from_edges(n, a[sel], b[sel], name=f"g{n}_{bits}")
