"""Pins for the oracle's literal restatement of the paper's matrix formulation (Sec. 3.1-3.2):
flattening, duplicate identities (Eq. 3, Eq. 4), crush, morph dimensions, Theorem 1,
Algorithm 1 (hand-computed case, Theorem 2 validity and minimality vs brute force), PIT
invariance and the 2:4 rule."""
import itertools

import numpy as np
import pytest
import scipy.ndimage
import scipy.signal

from oracle import morph
from oracle.morph import ZERO
from paper_2506_22969_gb300 import inputs


def _ints(seed, shape, lo=-4, hi=5):
    return np.random.default_rng(seed).integers(lo, hi, size=shape).astype(np.float64)


def test_flatten_is_valid_correlation():
    u = _ints(1, (7, 8))
    w = _ints(2, (3, 3))
    A, B = morph.flatten(u, w)
    ref = scipy.signal.correlate2d(u, w, mode="valid")
    np.testing.assert_array_equal((A @ B).reshape(ref.shape), ref)


def test_duplicate_identities_eq3_eq4():
    """Eq. 3 (horizontal, inside sub-matrix B_a): B_a[b+1, (i,j)] = B_a[b, (i,j+1)].
    Eq. 4 (vertical, between sub-matrices): block (a+1, output row i) = block (a, row i+1)."""
    k, m, n = 3, 6, 7
    u = _ints(3, (m, n))
    _, B = morph.flatten(u, np.ones((k, k)))
    ox = n - k + 1
    for a in range(k):
        for b in range(k - 1):
            for i in range(m - k + 1):
                for j in range(ox - 1):
                    assert B[a * k + b + 1, i * ox + j] == B[a * k + b, i * ox + j + 1]
    for a in range(k - 1):
        for i in range(m - k):
            blk_a1_i = B[(a + 1) * k:(a + 2) * k, i * ox:(i + 1) * ox]
            blk_a_i1 = B[a * k:(a + 1) * k, (i + 1) * ox:(i + 2) * ox]
            np.testing.assert_array_equal(blk_a1_i, blk_a_i1)


@pytest.mark.parametrize("k,r1,r2", [(3, 1, 1), (3, 2, 2), (3, 4, 2), (5, 3, 2), (3, 16, 8), (7, 16, 8), (5, 8, 4)])
def test_crush_reproduces_stencil_and_dims(k, r1, r2):
    oy, ox = 2 * r2, 3 * r1
    m, n = oy + k - 1, ox + k - 1
    u = _ints(k + r1, (m, n))
    w = _ints(r2 + 7, (k, k))
    A = morph.crushed_weights(w, r1, r2)
    B = morph.crushed_inputs(u, k, r1, r2)
    mp, kp, np_ = morph.morph_dims(k, r1, r2, m, n)
    assert A.shape == (mp, kp) and B.shape == (kp, np_)
    D = A @ B
    ref = scipy.signal.correlate2d(u, w, mode="valid")
    for py in range(oy // r2):
        for px in range(ox // r1):
            col = py * (ox // r1) + px
            for s in range(r2):
                for tau in range(r1):
                    assert D[s * r1 + tau, col] == ref[py * r2 + s, px * r1 + tau]


def test_staircase_structure():
    """Global staircase: block (s, u) is nonzero iff 0 <= u - s < k; local staircase: row
    tau of a nonzero block has its k nonzeros at columns tau..tau+k-1 (reading of the
    k-staircase definition with an inclusive upper end)."""
    k, r1, r2 = 3, 4, 3
    w = np.arange(1, 10, dtype=np.float64).reshape(3, 3)
    A = morph.crushed_weights(w, r1, r2)
    g = k + r1 - 1
    for s in range(r2):
        for u in range(k + r2 - 1):
            blk = A[s * r1:(s + 1) * r1, u * g:(u + 1) * g]
            assert np.any(blk) == (0 <= u - s < k)
            if np.any(blk):
                for tau in range(r1):
                    assert list(np.nonzero(blk[tau])[0]) == list(range(tau, tau + k))


def test_theorem1_non_conflict():
    """Thm 1: in a k-staircase, columns (and block columns) at distance >= k never conflict."""
    for k, r1, r2 in [(3, 4, 3), (5, 6, 4)]:
        A = morph.crushed_weights(np.ones((k, k)), r1, r2)
        E = morph.conflict_graph(A)
        g, mb = k + r1 - 1, k + r2 - 1
        for u in range(mb):
            for c in range(g):
                for c2 in range(c + k, g):
                    assert not E[u * g + c, u * g + c2]
        for u in range(mb):
            for u2 in range(u + k, mb):
                assert not E[u * g:(u + 1) * g, u2 * g:(u2 + 1) * g].any()


def test_algorithm1_hand_case():
    """n = 20 nodes in m = 4 blocks of g = 5, k = 3.  s1 = max(2, 3) = 3: only (G0, G3).
    s2 = max(2, 3) = 3: in G1 and G2, u=0->3, u=1->4, u=2 -> zero node."""
    M1, M2, M = morph.hierarchical_matching(20, 5, 3)
    assert M1 == [(0, 3)]
    assert M2 == [(5, 8), (6, 9), (7, ZERO), (10, 13), (11, 14), (12, ZERO)]
    assert M[:5] == [(0, 15), (1, 16), (2, 17), (3, 18), (4, 19)]
    assert len(M) == 11


def test_algorithm1_hand_case_even():
    """m = 10 blocks of g = 18 (k=3, r1=16, r2=8): s1 = 5 pairs every block."""
    M1, M2, M = morph.hierarchical_matching(180, 18, 3)
    assert M1 == [(i, i + 5) for i in range(5)] and M2 == []
    assert M[18] == (18, 108) and len(M) == 90


@pytest.mark.parametrize("k,r1,r2,alg1,brute", [
    (3, 1, 1, 9, 9), (3, 2, 1, 6, 6), (3, 1, 2, 6, 6), (3, 2, 2, 4, 4), (3, 3, 1, 3, 3), (3, 4, 1, 0, 0),
    (3, 3, 2, 2, 2), (3, 6, 1, 0, 0), (3, 1, 3, 3, 3), (3, 2, 3, 2, 2), (3, 4, 2, 0, 0),
    # Theorem 2's minimality argument analyses one sub-graph at a time; when several blocks stay
    # unmatched with an odd leftover, pairing leftovers across blocks beats it (reading: the
    # claim holds among two-level matchings only).
    (3, 5, 1, 3, 1), (3, 1, 5, 3, 1)])
def test_theorem2_validity_and_minimality(k, r1, r2, alg1, brute):
    """Thm 2: Algorithm 1's matching is valid (Def. 3) on the box staircase's conflict graph;
    its zero-column count is compared with the brute-force optimum of Problem 1."""
    A = morph.crushed_weights(np.ones((k, k)), r1, r2)
    E = morph.conflict_graph(A)
    g, mb = k + r1 - 1, k + r2 - 1
    _, _, M = morph.hierarchical_matching(g * mb, g, k)
    assert morph.is_valid_matching(M, E, g * mb)
    for a, b in M:
        if b != ZERO:
            same_block = (a // g) == (b // g)
            dist = (b - a) if same_block else (b // g - a // g)
            assert dist >= k
    zeros = sum(1 for a, b in M if b == ZERO)
    assert zeros == alg1
    assert morph.min_zero_columns_bruteforce(E) == brute


@pytest.mark.parametrize("mask,r1,r2", [
    ("box3", 1, 1), ("box3", 3, 2), ("box3", 5, 1), ("box3", 1, 5), ("star3", 2, 2), ("star3", 4, 1),
    ("star5", 1, 1), ("star5", 2, 1), ("cross3", 2, 2)])
def test_max_matching_pairing_is_minimal(mask, r1, r2):
    """The maximum-matching pairing (Problem 1 on the actual support) is valid (Def. 3) and
    reaches the brute-force optimum; for box masks where Algorithm 1 pads more (r1 = 5) it
    pads less."""
    pytest.importorskip("networkx")
    k = int(mask[-1])
    w = np.ones((k, k))
    if mask.startswith("star"):
        w = np.zeros((k, k))
        w[k // 2, :] = 1.0
        w[:, k // 2] = 1.0
    elif mask.startswith("cross"):  # an asymmetric support: centre, right and lower neighbour
        w = np.zeros((k, k))
        w[1, 1] = w[1, 2] = w[2, 1] = 1.0
    A = morph.crushed_weights(w, r1, r2)
    E = morph.conflict_graph(A)
    pairs, zeros = morph.max_matching_pairs(A)
    nz = np.any(A != 0, axis=0)
    # restricted to the nonzero columns the pairing covers each exactly once, without conflicts
    cols = [v for pr in pairs for v in pr if v != ZERO]
    assert sorted(cols) == sorted(np.where(nz)[0].tolist())
    assert all(b == ZERO or not E[a, b] for a, b in pairs)
    assert zeros == sum(1 for a, b in pairs if b == ZERO)
    sub = E[np.ix_(nz, nz)]
    assert zeros == morph.min_zero_columns_bruteforce(sub)
    if mask == "box3" and (r1, r2) in ((5, 1), (1, 5)):
        _, _, M = morph.hierarchical_matching(A.shape[1], k + r1 - 1, k)
        assert zeros < sum(1 for a, b in M if b == ZERO)


@pytest.mark.parametrize("shape,k,r1,r2", [("box", 3, 16, 8), ("box", 5, 16, 8), ("box", 7, 16, 8),
                                           ("star", 7, 16, 8), ("box", 3, 8, 16), ("box", 5, 4, 3)])
def test_pit_2_4_and_invariance(shape, k, r1, r2):
    """After Algorithm 1's permutation (and zero columns padding K to a multiple of 4), A''
    satisfies 2:4 and A'' B'' = A' B' exactly (PIT, Sec. 3.2)."""
    r = (k - 1) // 2
    w = inputs.stencil_weights(shape, 2, r, "random", seed=k).astype(np.float64)
    A = morph.crushed_weights(w, r1, r2)
    g, mb = k + r1 - 1, k + r2 - 1
    _, _, M = morph.hierarchical_matching(g * mb, g, k)
    order = morph.permutation_from_pairs(M)
    while len(order) % 4:
        order.append(ZERO)
    App = morph.apply_permutation(A, order)
    assert morph.satisfies_2_4(App)
    assert not morph.satisfies_2_4(A[:, :(A.shape[1] // 4) * 4])
    u = _ints(5, (2 * r2 + k - 1, 2 * r1 + k - 1))
    B = morph.crushed_inputs(u, k, r1, r2)
    Bpp = np.zeros((len(order), B.shape[1]))
    for j, c in enumerate(order):
        if c != ZERO:
            Bpp[j] = B[c]
    np.testing.assert_array_equal(App @ Bpp, A @ B)


def test_decompress_2_4():
    vals = np.array([[1.0, 2.0, 3.0, 4.0]])
    idx = np.array([[0, 3, 1, 2]])
    np.testing.assert_array_equal(morph.decompress_2_4(vals, idx), [[1, 0, 0, 2, 0, 3, 4, 0]])


@pytest.mark.parametrize("k,r1,r2,r3", [(3, 4, 2, 2), (3, 2, 2, 3)])
def test_crush_3d_and_nd_matching(k, r1, r2, r3):
    """3D reading: the nested staircase reproduces the valid 3D correlation, and the
    level-by-level matching is valid and makes A'' 2:4."""
    g, mb, mz = k + r1 - 1, k + r2 - 1, k + r3 - 1
    w = _ints(21, (k, k, k))
    A = morph.crushed_weights_3d(w, r1, r2, r3)
    u = _ints(22, (mz, mb, g))
    ref = scipy.ndimage.correlate(u, w, mode="constant")[k // 2:k // 2 + r3, k // 2:k // 2 + r2, k // 2:k // 2 + r1]
    D = A @ u.reshape(-1)
    for q, s, tau in itertools.product(range(r3), range(r2), range(r1)):
        assert D[(q * r2 + s) * r1 + tau] == ref[q, s, tau]
    M = morph.hierarchical_matching_nd([mz, mb, g], k)
    E = morph.conflict_graph(A)
    assert morph.is_valid_matching(M, E, g * mb * mz)
    order = morph.permutation_from_pairs(M)
    while len(order) % 4:
        order.append(ZERO)
    assert morph.satisfies_2_4(morph.apply_permutation(A, order))
