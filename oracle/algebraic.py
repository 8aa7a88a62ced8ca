"""Section 3.1's matrix forms and Algorithm 2 -- TEST INFRASTRUCTURE.

Dense numpy restatements for small unweighted graphs (n up to a few hundred):

* :func:`path_count_literal` -- ComputePathCount exactly as printed (Section
  3.1.1): it masks with the previous iteration's matrix only, so a pair first
  reached at level l is overwritten at level l+2 by a walk count. Kept to pin
  that reading: it disagrees with the true counts once Diam(G) >= 3.
* :func:`path_count` -- the same loop with the mask the correctness argument
  asks for (entries already set are never overwritten), in frontier form:
  C_0 = I, C_l = (C_{l-1} . A) masked to pairs not yet reached, Lambda = sum C_l.
  The first non-zero walk count of a pair is its shortest-path count.
* :func:`dependency` -- ComputeDependency (Section 3.1.2):
  Delta_{l-1} = Mask(((D_l + Delta_l) div Lambda) . A, l-1) mult Lambda,
  summed over l = Diam..1. Its diagonal comes out as reach-1 and is not part
  of BC (the definition excludes s = v).
* :func:`algorithm2` -- Section 4.2.1's pair formula: for every ordered pair
  s != t and v outside {s, t} with d(s,t) = d(s,v) + d(v,t),
  BC(v) += lambda_sv * lambda_vt / lambda_st.
* :func:`apsp_minplus` -- distances by repeated (min,+) squaring of the weight
  matrix (the distance product of Definition 3.7); works for integer weights.
"""
from __future__ import annotations

import numpy as np

INF = np.iinfo(np.int64).max // 4


def adjacency_matrix(g) -> np.ndarray:
    """0/1 int64 adjacency matrix A."""
    a = np.zeros((g.n, g.n), dtype=np.int64)
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr.astype(np.int64)))
    a[src, g.col] = 1
    return a


def weight_matrix(g) -> np.ndarray:
    """w(i,j) on edges, 0 on the diagonal, INF elsewhere."""
    wm = np.full((g.n, g.n), INF, dtype=np.int64)
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr.astype(np.int64)))
    wm[src, g.col] = 1 if g.w is None else g.w.astype(np.int64)
    np.fill_diagonal(wm, 0)
    return wm


def apsp_minplus(g) -> np.ndarray:
    """All-pairs distances by (min,+) products W*W*... until stable (INF = unreachable)."""
    d = weight_matrix(g)
    while True:
        nd = np.min(d[:, :, None] + d[None, :, :], axis=1)
        nd = np.minimum(nd, INF)
        if np.array_equal(nd, d):
            return d
        d = nd


def path_count_literal(a: np.ndarray, diam: int) -> np.ndarray:
    """ComputePathCount as printed: mask with Lambda_prev only."""
    n = a.shape[0]
    z = np.eye(n, dtype=object)
    lam = np.eye(n, dtype=object)
    prev = np.zeros((n, n), dtype=object)
    ao = a.astype(object)
    for _ in range(diam):
        z = z.dot(ao)
        cur = np.where(prev > 0, 0, z)
        lam = lam + cur
        prev = cur
    np.fill_diagonal(lam, 1)
    return lam


def path_count(a: np.ndarray):
    """Corrected ComputePathCount in frontier form.

    Returns (Lambda, D): Lambda[i][j] shortest-path counts (object ints,
    Lambda_ii = 1), D[i][j] distances (-1 unreachable)."""
    n = a.shape[0]
    ao = a.astype(object)
    c = np.eye(n, dtype=object)
    lam = np.eye(n, dtype=object)
    dist = np.where(np.eye(n, dtype=bool), 0, -1).astype(np.int64)
    reached = np.eye(n, dtype=bool)
    level = 0
    while True:
        level += 1
        nxt = c.dot(ao)
        nxt = np.where(reached, 0, nxt)
        hit = nxt != 0
        if not hit.any():
            return lam, dist
        lam = lam + nxt
        dist[hit] = level
        reached |= hit
        c = nxt


def dependency(a: np.ndarray, dist: np.ndarray, lam) -> np.ndarray:
    """ComputeDependency (Delta, FP64). dist: -1 marks unreachable pairs."""
    n = a.shape[0]
    lamf = np.array(lam, dtype=np.float64)
    lam_safe = np.where(lamf == 0, 1.0, lamf)
    af = a.astype(np.float64)
    diam = int(dist.max()) if dist.size else 0
    delta = np.zeros((n, n))
    delta_l = np.zeros((n, n))
    for l in range(diam, 0, -1):
        d_l = (dist == l).astype(np.float64)
        x = ((d_l + delta_l) / lam_safe).dot(af)
        x = np.where(dist == l - 1, x, 0.0)  # Mask(X, l-1)
        delta_l = x * lamf
        delta += delta_l
    return delta


def bc_from_dependency(delta: np.ndarray) -> np.ndarray:
    """BC(v) = sum_{s != v} delta_s*(v)."""
    d = delta.copy()
    np.fill_diagonal(d, 0.0)
    return d.sum(axis=0)


def algorithm2(dist: np.ndarray, lam) -> np.ndarray:
    """Pair formula over ordered pairs (dist -1 = unreachable). Exact in FP64
    up to one rounding per term."""
    n = dist.shape[0]
    lamf = np.array(lam, dtype=np.float64)
    reach = dist >= 0
    bc = np.zeros(n)
    for v in range(n):
        ok = reach[:, v][:, None] & reach[v, :][None, :] & reach
        ok &= dist == (dist[:, v][:, None] + dist[v, :][None, :])
        ok[v, :] = False
        ok[:, v] = False
        np.fill_diagonal(ok, False)
        num = lamf[:, v][:, None] * lamf[v, :][None, :]
        bc[v] = np.sum(np.where(ok, num / np.where(ok, lamf, 1.0), 0.0))
    return bc
