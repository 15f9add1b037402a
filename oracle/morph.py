"""The paper's matrix formulation of a stencil step, written out literally (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain numpy and Python loops,
no blocking or reordering beyond what the paper states, so each function can be read
against the paper by eye.  Shares no code with the product planner.

Notation follows Sec. 3: k is the stencil width (2r+1), (r1, r2[, r3]) the crush factors,
g = k + r1 - 1 the block size of the local staircase, m' = r1*r2, k' = (k+r1-1)(k+r2-1).
"""
from __future__ import annotations

import itertools

import numpy as np

ZERO = -1  # marker for an inserted zero column (the zeta nodes of Algorithm 1)


# --------------------------------------------------------------------------------------
# Stencil flattening (Sec. 3.1, "Stencil Flattening")
# --------------------------------------------------------------------------------------
def flatten(u: np.ndarray, w: np.ndarray):
    """Kernel vector A (1 x k^2) and input matrix B (k^2 x outputs) of a 2D valid stencil.

    Column (i, j) of B (row-major over the (m-k+1) x (n-k+1) outputs) is the window
    u[i:i+k, j:j+k] read row by row, so A @ B is the stencil applied at every output
    whose window lies inside u.  Row (a, b) of B belongs to sub-matrix B_a, the rows of
    B that come from the a-th window row.
    """
    k = w.shape[0]
    m, n = u.shape
    A = w.reshape(1, k * k).astype(np.float64)
    outs = [(i, j) for i in range(m - k + 1) for j in range(n - k + 1)]
    B = np.zeros((k * k, len(outs)))
    for col, (i, j) in enumerate(outs):
        for a in range(k):
            for b in range(k):
                B[a * k + b, col] = u[i + a, j + b]
    return A, B


# --------------------------------------------------------------------------------------
# Duplicates crush (Sec. 3.1): horizontal (r1) then vertical (r2)
# --------------------------------------------------------------------------------------
def local_staircase(wrow: np.ndarray, r1: int) -> np.ndarray:
    """Horizontal crush of one kernel row: r1 x (k+r1-1) block, row tau holds the
    weights shifted right by tau (the local staircase)."""
    k = wrow.shape[0]
    W = np.zeros((r1, k + r1 - 1))
    for tau in range(r1):
        W[tau, tau:tau + k] = wrow
    return W


def crushed_weights(w: np.ndarray, r1: int, r2: int) -> np.ndarray:
    """A' (m' x k') after horizontal and vertical duplicate crush.

    Rows rho = s*r1 + tau: output (s, tau) of an r2 x r1 patch.  Columns kappa = u*g + c:
    input (u, c) of the patch's (k+r2-1) x (k+r1-1) window.  Block (s, u) is the local
    staircase of kernel row u-s when 0 <= u-s < k, else zero (the global staircase).
    """
    k = w.shape[0]
    g = k + r1 - 1
    mb = k + r2 - 1
    A = np.zeros((r1 * r2, g * mb))
    for s in range(r2):
        for u in range(mb):
            d = u - s
            if 0 <= d < k:
                A[s * r1:(s + 1) * r1, u * g:(u + 1) * g] = local_staircase(w[d], r1)
    return A


def crushed_inputs(u: np.ndarray, k: int, r1: int, r2: int) -> np.ndarray:
    """B' (k' x n'): one column per r2 x r1 output patch (patches row-major), holding the
    deduplicated window of the patch, rows kappa = u*g + c (valid outputs only; the output
    extents (m-k+1, n-k+1) must be multiples of (r2, r1))."""
    m, n = u.shape
    oy, ox = m - k + 1, n - k + 1
    assert oy % r2 == 0 and ox % r1 == 0
    g, mb = k + r1 - 1, k + r2 - 1
    cols = []
    for py in range(oy // r2):
        for px in range(ox // r1):
            cols.append(u[py * r2:py * r2 + mb, px * r1:px * r1 + g].reshape(-1))
    return np.stack(cols, axis=1)


def morph_dims(k: int, r1: int, r2: int, m: int, n: int):
    """(m', k', n') of the morphed product for an m x n input (Sec. 3.3, Compute Evaluation)."""
    return r1 * r2, (k + r1 - 1) * (k + r2 - 1), (m - k + 1) * (n - k + 1) // (r1 * r2)


def crushed_weights_3d(w: np.ndarray, r1: int, r2: int, r3: int) -> np.ndarray:
    """3D extension (reading): a third crush along z.  Rows rho = (q*r2 + s)*r1 + tau,
    columns kappa = (v*mb + u)*g + c; entry w[v-q][u-s][c-tau] when all three lie in
    [0, k)."""
    k = w.shape[0]
    g, mb, mz = k + r1 - 1, k + r2 - 1, k + r3 - 1
    A = np.zeros((r1 * r2 * r3, g * mb * mz))
    for q in range(r3):
        for s in range(r2):
            for tau in range(r1):
                rho = (q * r2 + s) * r1 + tau
                for dz in range(k):
                    for dy in range(k):
                        for dx in range(k):
                            kappa = ((q + dz) * mb + (s + dy)) * g + (tau + dx)
                            A[rho, kappa] = w[dz, dy, dx]
    return A


# --------------------------------------------------------------------------------------
# Structured sparsity conversion (Sec. 3.2)
# --------------------------------------------------------------------------------------
def conflict_graph(A: np.ndarray) -> np.ndarray:
    """Def. 1: boolean adjacency; columns i != j conflict iff some row has both nonzero."""
    nz = (A != 0)
    n = A.shape[1]
    E = np.zeros((n, n), dtype=bool)
    for i in range(n):
        for j in range(i + 1, n):
            if np.any(nz[:, i] & nz[:, j]):
                E[i, j] = E[j, i] = True
    return E


def is_valid_matching(pairs, E: np.ndarray, n: int) -> bool:
    """Def. 3: every real column covered exactly once, no pair is a conflict edge."""
    seen = np.zeros(n, dtype=int)
    for a, b in pairs:
        for v in (a, b):
            if v != ZERO:
                seen[v] += 1
        if a != ZERO and b != ZERO and E[a, b]:
            return False
    return bool(np.all(seen == 1))


def min_zero_columns_bruteforce(E: np.ndarray) -> int:
    """Problem 1 by exhaustive search: p* = |V| - 2*nu, nu the maximum matching of the
    non-conflict graph.  Exponential; for |V| <= ~24."""
    n = E.shape[0]
    ok = [[(i != j) and not E[i, j] for j in range(n)] for i in range(n)]
    memo = {}

    def best(mask):  # max number of pairs among the vertices in mask
        if mask == 0:
            return 0
        if mask in memo:
            return memo[mask]
        i = (mask & -mask).bit_length() - 1
        rest = mask & ~(1 << i)
        res = best(rest)  # i stays unpaired
        m = rest
        while m:
            j = (m & -m).bit_length() - 1
            m &= m - 1
            if ok[i][j]:
                res = max(res, 1 + best(rest & ~(1 << j)))
        memo[mask] = res
        return res

    return n - 2 * best((1 << n) - 1)


def max_matching_pairs(A: np.ndarray):
    """Problem 1 on the actual support of A (the maximum-matching pairing used when a stencil's
    support is smaller than the box): the nonzero columns of A, two of them compatible when no
    row has both nonzero (Def. 1), paired by a maximum-cardinality matching (networkx's
    implementation of Edmonds' algorithm, a library primitive); every unmatched nonzero column
    gets a zero partner.  Returns (pairs, zero columns); all-zero columns of A take no part."""
    import networkx as nx
    nz = np.where(np.any(A != 0, axis=0))[0]
    S = (A[:, nz] != 0).astype(np.int64)
    G = nx.Graph()
    G.add_nodes_from(range(len(nz)))
    ii, jj = np.where(np.triu((S.T @ S) == 0, 1))
    G.add_edges_from(zip(ii.tolist(), jj.tolist()))
    M = nx.max_weight_matching(G, maxcardinality=True)
    pairs = [(int(nz[a]), int(nz[b])) for a, b in M]
    matched = {v for a, b in M for v in (a, b)}
    pairs += [(int(nz[i]), ZERO) for i in range(len(nz)) if i not in matched]
    return pairs, len(nz) - 2 * len(M)


def hierarchical_matching(n: int, g: int, k: int):
    """Algorithm 1 (hierarchical two-level matching), literally.

    Input: a global conflict graph with n nodes in m = n/g sub-graphs G_0..G_{m-1} of g
    nodes each; k the stencil width.  Node t of G_x is column x*g + t.
    Returns (M1, M2, M):
      M1 — block pairs (p, q) with q - p = s1 = max(floor(m/2), k);
      M2 — pairs inside each unmatched block at distance s2 = max(floor(g/2), k), or with a
           new zero node (ZERO) when the partner index falls outside the block;
      M  — the element pairs of M1 (block p ascending, t ascending) followed by M2 (block
           ascending, u ascending).
    Reading: the block test also requires G_{i+s1} to be unmatched (the listing only tests
    G_i; with s1 >= m/2 the extra test never fires).
    """
    assert n % g == 0
    m = n // g
    s1 = max(m // 2, k)
    block_matched = [False] * m
    M1 = []
    for i in range(m):
        if not block_matched[i] and i + s1 < m and not block_matched[i + s1]:
            M1.append((i, i + s1))
            block_matched[i] = block_matched[i + s1] = True
    s2 = max(g // 2, k)
    M2 = []
    for x in range(m):
        if block_matched[x]:
            continue
        node_matched = [False] * g
        for u in range(g):
            v = u + s2
            if not node_matched[u]:
                if v < g:
                    M2.append((x * g + u, x * g + v))
                    node_matched[u] = node_matched[v] = True
                else:
                    M2.append((x * g + u, ZERO))
                    node_matched[u] = True
    M = []
    for (p, q) in M1:
        for t in range(g):
            M.append((p * g + t, q * g + t))
    M.extend(M2)
    return M1, M2, M


def hierarchical_matching_nd(sizes, k: int):
    """Reading for 3D (the paper describes 2D only): apply the block-level step of
    Algorithm 1 at the outermost level (stride max(floor(m/2), k) over the sizes[0] blocks),
    pair matched blocks elementwise, and recurse into each unmatched block with the
    remaining sizes.  For sizes = [mb, g] this is Algorithm 1 exactly."""
    sizes = list(sizes)
    if len(sizes) == 2:
        return hierarchical_matching(sizes[0] * sizes[1], sizes[1], k)[2]
    m = sizes[0]
    inner = int(np.prod(sizes[1:]))
    s0 = max(m // 2, k)
    matched = [False] * m
    top = []
    for i in range(m):
        if not matched[i] and i + s0 < m and not matched[i + s0]:
            top.append((i, i + s0))
            matched[i] = matched[i + s0] = True
    M = []
    for (p, q) in top:
        for t in range(inner):
            M.append((p * inner + t, q * inner + t))
    sub = hierarchical_matching_nd(sizes[1:], k)
    for x in range(m):
        if matched[x]:
            continue
        for (a, b) in sub:
            M.append((x * inner + a, ZERO if b == ZERO else x * inner + b))
    return M


def permutation_from_pairs(M):
    """K order after PIT: the pairs concatenated, each as (first, second); ZERO = zero column."""
    order = []
    for a, b in M:
        order.extend([a, b])
    return order


def apply_permutation(A: np.ndarray, order) -> np.ndarray:
    """A'' = columns of A' in the given K order, zero columns where order has ZERO (PIT)."""
    out = np.zeros((A.shape[0], len(order)))
    for j, c in enumerate(order):
        if c != ZERO:
            out[:, j] = A[:, c]
    return out


def satisfies_2_4(A: np.ndarray) -> bool:
    """Eq. 2 with the sub-2:4 relaxation of Sec. 2.1: every group of 4 consecutive
    entries of every row holds at most 2 nonzeros (K a multiple of 4)."""
    if A.shape[1] % 4:
        return False
    nz = (A != 0).reshape(A.shape[0], -1, 4).sum(axis=2)
    return bool(np.all(nz <= 2))


def decompress_2_4(values: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """Dense M x K from the compressed M x K/2 values and their in-group positions
    (idx[r, 2q], idx[r, 2q+1] in 0..3 for group q), per Eq. 1's mask semantics."""
    M, half = values.shape
    out = np.zeros((M, 2 * half))
    for r in range(M):
        for q in range(half // 2):
            for e in range(2):
                pos = 4 * q + int(idx[r, 2 * q + e])
                out[r, pos] += values[r, 2 * q + e]
    return out


# --------------------------------------------------------------------------------------
# Dense stencil matrix (for brute force on tiny grids)
# --------------------------------------------------------------------------------------
def dense_stencil_matrix(dims, w: np.ndarray, bc: str) -> np.ndarray:
    """S with vec(u_{s+1}) = S vec(u_s) for the stencil definition of Sec. 2.2
    (correlation: u_{s+1}[x] = sum_o w[o] u_s[x+o]); bc 'dirichlet' or 'periodic'."""
    dims = tuple(int(d) for d in dims)
    nd = len(dims)
    r = (w.shape[0] - 1) // 2
    N = int(np.prod(dims))
    S = np.zeros((N, N))
    offsets = list(itertools.product(range(-r, r + 1), repeat=nd))
    for x in itertools.product(*[range(d) for d in dims]):
        row = np.ravel_multi_index(x, dims)
        for o in offsets:
            wv = w[tuple(oi + r for oi in o)]
            if wv == 0:
                continue
            y = [x[i] + o[i] for i in range(nd)]
            if bc == "periodic":
                y = [y[i] % dims[i] for i in range(nd)]
            elif any(y[i] < 0 or y[i] >= dims[i] for i in range(nd)):
                continue
            S[row, np.ravel_multi_index(tuple(y), dims)] += wv
    return S
