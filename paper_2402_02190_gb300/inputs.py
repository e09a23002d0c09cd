"""Seeded synthetic inputs shared by the CUDA path, the tests and the oracle.

This module holds no arithmetic of the CPRA method itself: it only builds
graphs (the instances G(V, E) of the Background section and App. C.3),
penalty grids, and
seeded parameter / relaxed-solution arrays that both sides receive as inputs.

Graph conventions (App. B, Eq. GCN; App. C.3):
  * symmetric CSR, ``rowptr`` int64[N+1], ``col`` int32[nnz], columns sorted
    ascending within each row, no self-loops, no duplicate entries;
  * ``nnz`` = 2|E| (each undirected edge appears in both rows).

All generators use numpy's PCG64 ``default_rng``; results are identical on
x86_64 and aarch64.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "edges_to_csr",
    "csr_to_edges",
    "random_regular_graph",
    "erdos_renyi_graph",
    "bfs_induced_subgraph",
    "lambda_linspace",
    "lambda_geomspace",
    "seeded_params",
    "seeded_adam_state",
    "seeded_P",
    "param_layout",
]


def edges_to_csr(N: int, ei: np.ndarray, ej: np.ndarray):
    """Undirected edge list (each edge once, ei != ej) -> symmetric sorted CSR."""
    ei = np.asarray(ei, dtype=np.int64)
    ej = np.asarray(ej, dtype=np.int64)
    src = np.concatenate([ei, ej])
    dst = np.concatenate([ej, ei])
    order = np.lexsort((dst, src))
    src = src[order]
    dst = dst[order]
    counts = np.bincount(src, minlength=N).astype(np.int64)
    rowptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return rowptr, dst.astype(np.int32)


def csr_to_edges(rowptr: np.ndarray, col: np.ndarray):
    """Symmetric CSR -> undirected edges (i < j), each once."""
    N = len(rowptr) - 1
    rows = np.repeat(np.arange(N, dtype=np.int64), np.diff(rowptr))
    c = col.astype(np.int64)
    keep = rows < c
    return rows[keep], c[keep]


def _pair_keys(u, v, N):
    a = np.minimum(u, v)
    b = np.maximum(u, v)
    return a * N + b


def random_regular_graph(N: int, d: int, seed: int):
    """Random d-regular simple graph on N nodes (configuration model).

    Stubs are paired by a seeded shuffle; self-loops and repeated pairs are
    then removed by random double-edge switches until the multigraph is
    simple.  The RRGs of the paper's MIS experiments (Experiments section,
    penalty- and variation-diversified MIS) have this shape.
    """
    if (N * d) % 2 != 0 or d >= N:
        raise ValueError("N*d must be even and d < N")
    rng = np.random.default_rng(seed)
    stubs = np.repeat(np.arange(N, dtype=np.int64), d)
    rng.shuffle(stubs)
    pairs = stubs.reshape(-1, 2).copy()
    E = pairs.shape[0]
    for _ in range(10000):
        u, v = pairs[:, 0], pairs[:, 1]
        keys = _pair_keys(u, v, N)
        order = np.argsort(keys, kind="stable")
        dup = np.zeros(E, dtype=bool)
        ks = keys[order]
        dup_sorted = np.zeros(E, dtype=bool)
        dup_sorted[1:] = ks[1:] == ks[:-1]
        dup[order] = dup_sorted
        bad = np.nonzero((u == v) | dup)[0]
        if bad.size == 0:
            break
        partners = rng.integers(0, E, size=bad.size)
        for b, o in zip(bad.tolist(), partners.tolist()):
            if b == o:
                continue
            ub, vb = pairs[b]
            uo, vo = pairs[o]
            if rng.integers(0, 2):
                pairs[b] = (ub, uo)
                pairs[o] = (vb, vo)
            else:
                pairs[b] = (ub, vo)
                pairs[o] = (vb, uo)
    else:  # pragma: no cover - practically unreachable
        raise RuntimeError("random_regular_graph: switching did not converge")
    return edges_to_csr(N, pairs[:, 0], pairs[:, 1])


def erdos_renyi_graph(N: int, p: float, seed: int):
    """G(N, p): edge count drawn Binomial(N(N-1)/2, p), then that many
    distinct uniform pairs (equal in law to G(N, p)).  Isolated nodes occur."""
    rng = np.random.default_rng(seed)
    total = N * (N - 1) // 2
    M = int(rng.binomial(total, p))
    keys = np.empty(0, dtype=np.int64)
    while keys.size < M:
        need = M - keys.size
        k = max(int(need * 1.1) + 16, 16)
        a = rng.integers(0, N, size=k, dtype=np.int64)
        b = rng.integers(0, N, size=k, dtype=np.int64)
        ok = a != b
        a, b = a[ok], b[ok]
        nk = _pair_keys(a, b, N)
        keys = np.unique(np.concatenate([keys, nk]))
    if keys.size > M:
        keys = rng.permutation(keys)[:M]
    ei = keys // N
    ej = keys % N
    return edges_to_csr(N, ei, ej)


def bfs_induced_subgraph(rowptr, col, n_keep: int, root: int = 0):
    """Induced subgraph on the first ``n_keep`` nodes reached by BFS from
    ``root`` (relabelled 0..n_keep-1 in BFS order)."""
    N = len(rowptr) - 1
    seen = -np.ones(N, dtype=np.int64)
    order = [root]
    seen[root] = 0
    head = 0
    while head < len(order) and len(order) < n_keep:
        u = order[head]
        head += 1
        for v in col[rowptr[u]:rowptr[u + 1]]:
            if seen[v] < 0 and len(order) < n_keep:
                seen[v] = len(order)
                order.append(int(v))
    ei, ej = csr_to_edges(rowptr, col)
    keep = (seen[ei] >= 0) & (seen[ej] >= 0)
    return edges_to_csr(len(order), seen[ei[keep]], seen[ej[keep]])


def seeded_edge_weights(rowptr, col, seed: int, kind: str = "uniform") -> np.ndarray:
    """Symmetric edge weights per CSR entry (w_ij = w_ji), float32: "uniform"
    draws U(0.5, 2) per undirected edge, "pm1" draws +1 or -1 (the signed
    unit weights of some Gset max-cut instances)."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    N = len(rowptr) - 1
    rows = np.repeat(np.arange(N, dtype=np.int64), np.diff(rowptr))
    lo, hi = np.minimum(rows, col), np.maximum(rows, col)
    keys = lo * N + hi
    uniq, inv = np.unique(keys, return_inverse=True)
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        per_edge = rng.uniform(0.5, 2.0, size=len(uniq))
    elif kind == "pm1":
        per_edge = rng.choice(np.array([-1.0, 1.0]), size=len(uniq))
    else:
        raise ValueError("kind")
    return per_edge[inv].astype(np.float32)


def lambda_linspace(lo: float, hi: float, S: int) -> np.ndarray:
    return np.linspace(lo, hi, S).astype(np.float32)


def lambda_geomspace(lo: float, hi: float, S: int) -> np.ndarray:
    return np.geomspace(lo, hi, S).astype(np.float32)


def param_layout(H0: int, H1: int, S: int):
    """Offsets of the flat parameter vector theta (float32), in order:
    Wcat1 = [B1 | W1] (H1 x 2H0, row-major), b1 (H1),
    Wcat2 = [B2 | W2] (S x 2H1, row-major), b2 (S).
    Returns a dict name -> (offset, shape)."""
    out = {}
    off = 0
    for name, shape in (("Wcat1", (H1, 2 * H0)), ("b1", (H1,)),
                        ("Wcat2", (S, 2 * H1)), ("b2", (S,))):
        out[name] = (off, shape)
        off += int(np.prod(shape))
    out["_total"] = (off, ())
    return out


def seeded_params(N: int, H0: int, H1: int, S: int, seed: int,
                  weight_scale: float = 1.0, emb_scale: float = 1.0):
    """Seeded float32 parameters: node embeddings X0 ~ N(0, emb_scale^2)
    (N x H0) and layer weights ~ U(+-weight_scale/sqrt(fan_in)).
    Returns (theta_flat float32, X0 float32)."""
    rng = np.random.default_rng(seed)
    lay = param_layout(H0, H1, S)
    theta = np.empty(lay["_total"][0], dtype=np.float32)
    for name, fan_in in (("Wcat1", H0), ("b1", H0), ("Wcat2", H1), ("b2", H1)):
        off, shape = lay[name]
        n = int(np.prod(shape))
        bound = weight_scale / np.sqrt(fan_in)
        theta[off:off + n] = rng.uniform(-bound, bound, size=n).astype(np.float32)
    X0 = (rng.standard_normal((N, H0)) * emb_scale).astype(np.float32)
    return theta, X0


def seeded_adam_state(n: int, seed: int, scale: float = 1e-2):
    """Seeded Adam moments (m ~ N(0, scale^2), v ~ |N(0, scale^2)|^2 ...)."""
    rng = np.random.default_rng(seed)
    m = (rng.standard_normal(n) * scale).astype(np.float32)
    v = (rng.standard_normal(n) * scale).astype(np.float32) ** 2
    return m, v.astype(np.float32)


def seeded_P(N: int, S: int, seed: int, special: bool = True) -> np.ndarray:
    """Seeded relaxed solutions P in [0, 1]^{N x S} (float32).

    With ``special``, plants exact 0, 1 and 0.5 entries, values one ulp
    either side of 0.5, and constant rows (zero variance across shots)."""
    rng = np.random.default_rng(seed)
    P = rng.uniform(0.0, 1.0, size=(N, S)).astype(np.float32)
    if special and N >= 8:
        flat = P.reshape(-1)
        k = max(1, flat.size // 50)
        idx = rng.choice(flat.size, size=5 * k, replace=False)
        half = np.float32(0.5)
        flat[idx[0:k]] = 0.0
        flat[idx[k:2 * k]] = 1.0
        flat[idx[2 * k:3 * k]] = half
        flat[idx[3 * k:4 * k]] = np.nextafter(half, np.float32(1.0))
        flat[idx[4 * k:5 * k]] = np.nextafter(half, np.float32(0.0))
        P[1, :] = np.float32(0.25)          # constant row: VAR == 0
        P[3, :] = np.float32(0.5)           # constant row at the threshold
    return P


# ------------------------------------------------------------ warm start
def ws_param_count(F: int, H: int, S: int) -> int:
    """Flat size of the warm-start network: three Eq. GCN layers F -> H -> H -> S."""
    return 2 * H * F + H + 2 * H * H + H + 2 * S * H + S


def seeded_ws_params(F: int, H: int, S: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """U(+-scale/sqrt(fan_in)) per block, float32, in the flat layout."""
    rng = np.random.default_rng(seed)
    out = []
    for fan, n in ((2 * F, 2 * H * F), (2 * F, H), (2 * H, 2 * H * H), (2 * H, H),
                   (2 * H, 2 * S * H), (2 * H, S)):
        b = scale / np.sqrt(fan)
        out.append(rng.uniform(-b, b, size=n))
    return np.concatenate(out).astype(np.float32)


def seeded_ws_features(rowptr, F: int, seed: int) -> np.ndarray:
    """Host stand-in for the network's node features: 1, deg/8, then N(0,1)."""
    rowptr = np.asarray(rowptr)
    N = len(rowptr) - 1
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(N, F))
    X[:, 0] = 1.0
    X[:, 1] = np.diff(rowptr) / 8.0
    return X.astype(np.float32)


def seeded_bits(N: int, S: int, seed: int, p: float = 0.3) -> np.ndarray:
    """Random 0/1 targets [N, S] packed as uint32 [N, ceil(S/32)] (bit s % 32 of word s // 32)."""
    rng = np.random.default_rng(seed)
    Y = (rng.random((N, S)) < p).astype(np.uint8)
    W = (S + 31) // 32
    out = np.zeros((N, W), dtype=np.uint32)
    for s in range(S):
        out[:, s // 32] |= (Y[:, s].astype(np.uint32) << np.uint32(s % 32))
    return out


def unpack_bits(bits, S: int) -> np.ndarray:
    """uint32 [N, ceil(S/32)] -> 0/1 uint8 [N, S]."""
    bits = np.asarray(bits, dtype=np.uint32)
    N = bits.shape[0]
    out = np.zeros((N, S), dtype=np.uint8)
    for s in range(S):
        out[:, s] = (bits[:, s // 32] >> np.uint32(s % 32)) & np.uint32(1)
    return out


# ------------------------------------------------------------ diverse bipartite matching
def dbm_graph(N1: int, N2: int):
    """GNN graph of an N1 x N2 matching problem: the node of x_ij (index
    i*N2 + j) is adjacent to every x_ik (same row) and x_kj (same column), the
    variables that share one of its constraints.  Symmetric CSR, sorted rows."""
    rows = []
    for i in range(N1):
        for j in range(N2):
            nb = [i * N2 + k for k in range(N2) if k != j] + [k * N2 + j for k in range(N1) if k != i]
            rows.append(sorted(nb))
    rowptr = np.zeros(N1 * N2 + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([v for r in rows for v in r], dtype=np.int32)
    return rowptr, col


def dbm_instance(N1: int, N2: int, seed: int, n_fields: int = 7, p: float = 0.25, q: float = 0.25):
    """Seeded stand-in for one CORA-derived matching instance: rewards C_ij
    (link likelihoods, skewed towards 0) and M_ij = 1 when the two papers'
    fields differ (fields drawn uniformly), flattened to node order i*N2 + j.
    Returns (C [N], M [N], p, q)."""
    rng = np.random.default_rng(seed)
    C = rng.random((N1, N2)) ** 3
    f1 = rng.integers(0, n_fields, size=N1)
    f2 = rng.integers(0, n_fields, size=N2)
    M = (f1[:, None] != f2[None, :]).astype(np.float64)
    return C.ravel().astype(np.float32), M.ravel().astype(np.float32), p, q


def dbm_lambda_grid(n: int = 11):
    """The penalty grid of the DBM experiment: lambda_s = (a, a, b, b) with
    a, b in {2^0, ..., 2^(n-1)}; returns [n*n, 4]."""
    v = 2.0 ** np.arange(n)
    return np.array([(a, a, b, b) for a in v for b in v], dtype=np.float32)


def dbm_shots(N1: int, N2: int, instances, lam4, pq):
    """Per-shot arrays of a DBM run from a list of instances (C, M) [N] each
    and per-shot penalties lam4 [S, 4] and shares pq [S, 2]: shot s uses
    instance s mod len(instances).  Returns C [N, S], M [N, S], lam4, pq."""
    lam4 = np.asarray(lam4, dtype=np.float32)
    S = lam4.shape[0]
    C = np.stack([instances[s % len(instances)][0] for s in range(S)], axis=1)
    M = np.stack([instances[s % len(instances)][1] for s in range(S)], axis=1)
    return (C.astype(np.float32), M.astype(np.float32), lam4,
            np.broadcast_to(np.asarray(pq, dtype=np.float32), (S, 2)).copy())
