"""Displacement and Lagrange-multiplier aggregation (oracle).

Displacement aggregates (Sec. 4.2): aggregation runs on the node graph of the level's K
block with every coupling between the two bodies dropped on the fly, so no aggregate
crosses the contact interface.  The paper uses a standard (uncoupled) aggregation; here the
standard scheme is a deterministic distance-2 maximal independent set (MIS-2) of roots with
hash priorities, followed by two fill phases:

* priority of node i: (fmix32(i xor seed), i), fmix32 = MurmurHash3's 32-bit finaliser
  (Appleby), compared lexicographically, so every priority is distinct;
* root selection, repeated until no node is undecided: an undecided node whose priority is
  the largest among the undecided nodes of its distance-2 neighbourhood becomes a root, and
  every undecided node within distance 2 of a new root is marked "out";
* phase 2: every neighbour of a root joins the root's aggregate;
* phase 3: each node still unassigned joins the phase-2 aggregate it shares most edges with
  (ties to the smallest aggregate id), reading only the phase-2 assignment;
* aggregates are numbered by ascending root id.

Multiplier aggregates follow Algorithm 1 (LagMultAggregation, Sec. 4.3) literally: loop over
the slave displacement DOFs (rows of D) in increasing order, take the aggregate k of the DOF's
node, and for every multiplier DOF j with D_ij != 0 either open a new multiplier aggregate
{node(j)} for k or add node(j) to the aggregate already associated with k.  A multiplier node
that was already placed keeps its first aggregate (the algorithm never meets that case when D
is diagonal).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

UNDECIDED, ROOT, OUT = 0, 1, 2


def fmix32(h: np.ndarray) -> np.ndarray:
    """MurmurHash3 32-bit finaliser (A. Appleby), vectorised over uint32 values."""
    h = np.asarray(h, dtype=np.uint64) & np.uint64(0xFFFFFFFF)
    h ^= h >> np.uint64(16)
    h = (h * np.uint64(0x85EBCA6B)) & np.uint64(0xFFFFFFFF)
    h ^= h >> np.uint64(13)
    h = (h * np.uint64(0xC2B2AE35)) & np.uint64(0xFFFFFFFF)
    h ^= h >> np.uint64(16)
    return h


def priorities(n: int, seed: int) -> np.ndarray:
    """Distinct uint64 priority per node: fmix32(i ^ seed) * 2^32 + i."""
    i = np.arange(n, dtype=np.uint64)
    h = fmix32(i ^ np.uint64(seed & 0xFFFFFFFF))
    # key = h * 2^32 + i fits in uint64; compare as uint64
    return (h << np.uint64(32)) | i


def aggregation_graph(Kpat: sp.csr_matrix, body: np.ndarray) -> sp.csr_matrix:
    """Node graph of K without the diagonal and without inter-body couplings (Sec. 4.2)."""
    P = Kpat.tocsr()
    rows = np.repeat(np.arange(P.shape[0]), np.diff(P.indptr))
    cols = P.indices
    keep = (rows != cols) & (body[rows] == body[cols])
    G = sp.csr_matrix((np.ones(int(keep.sum())), (rows[keep], cols[keep])), shape=P.shape)
    G.sort_indices()
    return G


def _closed_max(G: sp.csr_matrix, v: np.ndarray) -> np.ndarray:
    """max over the closed neighbourhood {i} U N(i) of v (uint64)."""
    out = v.copy()
    rows = np.repeat(np.arange(G.shape[0]), np.diff(G.indptr))
    np.maximum.at(out, rows, v[G.indices])
    return out


def _closed_any(G: sp.csr_matrix, b: np.ndarray) -> np.ndarray:
    out = b.copy()
    rows = np.repeat(np.arange(G.shape[0]), np.diff(G.indptr))
    np.logical_or.at(out, rows, b[G.indices])
    return out


def mis2_roots(G: sp.csr_matrix, seed: int):
    """Root selection of the MIS-2 aggregation. Returns (state array, number of rounds)."""
    n = G.shape[0]
    key = priorities(n, seed)
    state = np.full(n, UNDECIDED, dtype=np.int8)
    rounds = 0
    while np.any(state == UNDECIDED):
        rounds += 1
        und = state == UNDECIDED
        kv = np.where(und, key + np.uint64(1), np.uint64(0))   # 0 = "no undecided node"
        m1 = _closed_max(G, kv)
        m2 = _closed_max(G, m1)
        new_root = und & (kv == m2)
        state[new_root] = ROOT
        near = _closed_any(G, _closed_any(G, new_root))
        state[und & ~new_root & near] = OUT
    return state, rounds


def aggregate_nodes(G: sp.csr_matrix, seed: int):
    """MIS-2 aggregation: returns (agg_of_node int64, root node per aggregate)."""
    n = G.shape[0]
    state, _ = mis2_roots(G, seed)
    roots = np.nonzero(state == ROOT)[0]            # ascending node id = aggregate id
    agg = np.full(n, -1, dtype=np.int64)
    agg[roots] = np.arange(roots.size)
    rows = np.repeat(np.arange(n), np.diff(G.indptr))
    cols = G.indices
    # phase 2: neighbours of roots
    e = (state[cols] == ROOT) & (agg[rows] < 0)
    agg2 = agg.copy()
    agg2[rows[e]] = agg[cols[e]]
    # phase 3: most shared edges with a phase-2 aggregate, ties -> smallest id
    rem = agg2 < 0
    e3 = rem[rows] & (agg2[cols] >= 0)
    r3, a3 = rows[e3], agg2[cols[e3]]
    final = agg2.copy()
    if r3.size:
        pair = np.unique(np.stack([r3, a3], axis=1), axis=0, return_counts=True)
        pr, cnt = pair[0], pair[1]
        order = np.lexsort((pr[:, 1], -cnt, pr[:, 0]))
        pr = pr[order]
        first = np.ones(pr.shape[0], dtype=bool)
        first[1:] = pr[1:, 0] != pr[:-1, 0]
        final[pr[first, 0]] = pr[first, 1]
    if np.any(final < 0):
        raise RuntimeError("node left unaggregated")
    return final, roots


def lagmult_aggregation(agg: np.ndarray, D_rows: list, bu: int):
    """Algorithm 1 (LagMultAggregation).

    agg    -- displacement aggregate of every displacement node
    D_rows -- for each slave displacement DOF i (sorted ascending), the sorted list of
              multiplier DOFs j with D_ij != 0, given as a list of (i, [j...]) pairs
    bu     -- displacement DOFs per node at this level (node(i) = i // bu); multiplier
              nodes carry 3 DOFs (node(j) = j // 3)
    Returns (lagg: multiplier node -> aggregate id, d: dict displacement aggregate -> LM aggregate).
    """
    d = {}
    lagg = {}
    count = 0
    for i, js in D_rows:
        k = int(agg[i // bu])
        for j in js:
            nl = j // 3
            if k not in d:
                d[k] = count
                count += 1
                lagg.setdefault(nl, d[k])
            else:
                lagg.setdefault(nl, d[k])
    return lagg, d, count
