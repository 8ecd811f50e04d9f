"""Pins for the CPU oracle: facts fixed by the paper and by mathematics, none of
which is the oracle's own formula typed again.  Runs on CPU (not marked gpu).

Each test names the passage it follows.  Together they are chosen so that a
plausible slip in the oracle (a dropped term, a swapped index, a transposed
operand, a wrong sign in the Jacobi rotation, a wrong window order) fails at
least one of them.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import ssa_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def paper_values():
    with open(os.path.join(GOLDEN, "paper_values.json")) as f:
        return json.load(f)


def rank_of(sigma, rel=1e-9):
    return int(np.sum(sigma > rel * sigma[0]))


# Both SVD routes of the oracle.  The paper's Step 2 goes through S = X X^T,
# so a zero singular value comes out near sqrt(eps) * sigma_1 there; the
# Jacobi route resolves it to eps * sigma_1.  Each route gets the null-space
# threshold its arithmetic allows.
ROUTES = [("jacobi", 1e-10), ("eigen", 1e-6)]


def sigmas(P, r):
    return [(O.decompose(P, r, m)[0], thr) for m, thr in ROUTES]


# ------------------------------------------------------------ embedding
def test_hankel_embedding_printed_form():
    """Eq. ssa_embedding: first row x_1..x_K, first column x_1..x_L, last row
    x_L..x_N, constant anti-diagonals."""
    N, L = 11, 4
    K = N - L + 1
    x = np.arange(1.0, N + 1)
    X = O.Problem.series(x, L).matrix()
    assert X.shape == (L, K)
    np.testing.assert_array_equal(X[0], x[:K])
    np.testing.assert_array_equal(X[:, 0], x[:L])
    np.testing.assert_array_equal(X[-1], x[L - 1:])
    for i, j in itertools.product(range(L), range(K)):
        assert X[i, j] == i + j + 1          # x_{i+j-1} with 1-based (i, j)


def test_mssa_embedding_is_stacked_hankel():
    """Eq. mssa_embedding: [X^(1) : ... : X^(s)], K = sum K_p."""
    xs = [np.arange(7.0), 100 + np.arange(9.0), -np.arange(5.0)]
    L = 3
    P = O.Problem.multi(xs, L)
    X = P.matrix()
    assert P.Ks == [5, 7, 3] and X.shape == (3, 15)
    col = 0
    for x in xs:
        for j in range(len(x) - L + 1):
            np.testing.assert_array_equal(X[:, col], x[j:j + L])
            col += 1


def test_2d_trajectory_is_hankel_block_hankel():
    """Eqs. block_hankel_cols / block_hankel_matrix: column k+(l-1)Kx is the
    vectorised window at (k, l); block (a, b) is the Hankel matrix of image
    column a+b-1."""
    rng = np.random.default_rng(0)
    nx, ny, lx, ly = 7, 6, 3, 2
    x = rng.normal(size=(nx, ny))
    P = O.Problem.image(x, lx, ly)
    X = P.matrix()
    kx, ky = nx - lx + 1, ny - ly + 1
    assert X.shape == (lx * ly, kx * ky)
    for k in range(kx):
        for l in range(ky):
            np.testing.assert_array_equal(X[:, k + l * kx],
                                          x[k:k + lx, l:l + ly].ravel(order="F"))
    for a in range(ly):
        for b in range(ky):
            H = X[a * lx:(a + 1) * lx, b * kx:(b + 1) * kx]
            col = x[:, a + b]
            for i in range(lx):
                np.testing.assert_array_equal(H[i], col[i:i + kx])


def test_mars_trajectory_sizes():
    """Sec. 4.2: the sizes the paper prints for the 258x275 Mars image."""
    for case in paper_values()["mars_trajectory_sizes"]["cases"]:
        nx, ny = case["image"]
        lx, ly = case["window"]
        obs = np.ones((nx, ny), dtype=bool)
        Lset = O.window_set(lx, ly)
        Kset = O.origin_set(obs, Lset)
        assert len(Lset) == case["L"] and len(Kset) == case["K"]


def test_origin_set_brute_force_with_holes():
    """Eq. sh_Ks by enumeration in pure Python on a shaped example: a circular
    window on an image with a hole and a ragged edge."""
    rng = np.random.default_rng(1)
    nx, ny = 13, 11
    obs = rng.uniform(size=(nx, ny)) > 0.08
    obs[4:6, 3:5] = False
    w = np.array([[0, 1, 0], [1, 1, 1], [0, 1, 1]], dtype=bool)
    Lset = O.window_set(3, 3, w)
    assert [tuple(p) for p in Lset] == [(1, 0), (0, 1), (1, 1), (2, 1), (1, 2), (2, 2)]
    brute = []
    for ky in range(ny):
        for kx in range(nx):
            if all(0 <= kx + a < nx and 0 <= ky + b < ny and obs[kx + a, ky + b]
                   for a, b in Lset):
                brute.append((kx, ky))
    assert [tuple(p) for p in O.origin_set(obs, Lset)] == brute


def test_weights_1d_closed_form():
    """Alg. hankelization, step 2: W = (1, 2, ..., L*, ..., L*, ..., 2, 1)."""
    for N, L in [(10, 3), (10, 8), (9, 5), (2, 1), (1000, 500)]:
        K = N - L + 1
        P = O.Problem.series(np.zeros(N), L)
        w = P.weights()[:, 0]
        Ls = min(L, K)
        expect = [min(k + 1, Ls, N - k) for k in range(N)]
        np.testing.assert_array_equal(w, expect)


def test_weights_count_trajectory_entries():
    """w_k = |A_k| = ||T(E_k)||_F^2 (Sec. 2.2): embed each unit element and
    count its ones, on a shaped example."""
    nx, ny = 6, 5
    obs = np.ones((nx, ny), dtype=bool)
    obs[2, 2] = False
    w = np.array([[1, 1], [0, 1]], dtype=bool)
    Lset = O.window_set(2, 2, w)
    Kset = O.origin_set(obs, Lset)
    W = O.weights((nx, ny), Lset, Kset)
    for m in range(nx):
        for n in range(ny):
            E = np.zeros((nx, ny))
            E[m, n] = 1.0
            assert O.trajectory_matrix(E, Lset, Kset).sum() == W[m, n]


# ------------------------------------------------------------ matvec
def test_matvec_brute_force():
    """u_i = sum_j x[l_i + k_j] v_j by explicit loops, both products."""
    rng = np.random.default_rng(2)
    xs = [rng.normal(size=n) for n in (9, 12)]
    P = O.Problem.multi(xs, 4)
    v = rng.normal(size=P.K)
    u = rng.normal(size=P.L)
    u_ref = np.zeros(P.L)
    v_ref = np.zeros(P.K)
    for c, x in enumerate(xs):
        for j in range(P.Ks[c]):
            for i in range(P.L):
                u_ref[i] += x[i + j] * v[P.offsets[c] + j]
                v_ref[P.offsets[c] + j] += x[i + j] * u[i]
    np.testing.assert_allclose(O.matvec(P, v), u_ref, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(O.rmatvec(P, u), v_ref, rtol=1e-13, atol=1e-13)


# ------------------------------------------------------------ SVD step
def test_jacobi_matches_lapack():
    """The one-sided Jacobi SVD reduces to the textbook SVD (LAPACK via
    numpy) on random, wide, tall and rank-deficient matrices."""
    rng = np.random.default_rng(3)
    for shape in [(7, 5), (5, 9), (12, 12), (30, 17)]:
        A = rng.normal(size=shape)
        s, U, V = O.svd_jacobi(A)
        np.testing.assert_allclose(s, np.linalg.svd(A, compute_uv=False),
                                   rtol=1e-13)
        np.testing.assert_allclose(U * s @ V.T, A, atol=1e-12)
        np.testing.assert_allclose(U.T @ U, np.eye(len(s)), atol=1e-12)
        np.testing.assert_allclose(V.T @ V, np.eye(len(s)), atol=1e-12)
    B = rng.normal(size=(10, 3)) @ rng.normal(size=(3, 8))
    s = O.svd_jacobi(B)[0]
    assert rank_of(s, 1e-12) == 3


def test_eigen_route_matches_jacobi_route():
    """Step 2 as written (S = X X^T) agrees with the Jacobi SVD of X."""
    rng = np.random.default_rng(4)
    x = np.cumsum(rng.normal(size=240))
    P = O.Problem.series(x, 60)
    s1, U1, V1 = O.decompose(P, 12, "eigen")
    s2, U2, V2 = O.decompose(P, 12, "jacobi")
    np.testing.assert_allclose(s1, s2, rtol=1e-10)
    # well separated leading triples agree as vectors (signs are normalised)
    np.testing.assert_allclose(U1[:, :3], U2[:, :3], atol=1e-8)
    np.testing.assert_allclose(V1[:, :3], V2[:, :3], atol=1e-8)


def test_transposed_eigen_route_matches_jacobi_route():
    """Step 2 on X^T (S' = X^T X, for K < L) gives the triples of the Jacobi
    SVD of X: the SVD of X^T has the same singular values with U and V
    exchanged."""
    rng = np.random.default_rng(6)
    x = np.cumsum(rng.normal(size=240))
    P = O.Problem.series(x, 200)          # L = 200 > K = 41
    s1, U1, V1 = O.decompose(P, 12, "eigen_t")
    s2, U2, V2 = O.decompose(P, 12, "jacobi")
    np.testing.assert_allclose(s1, s2, rtol=1e-10)
    np.testing.assert_allclose(U1[:, :3], U2[:, :3], atol=1e-8)
    np.testing.assert_allclose(V1[:, :3], V2[:, :3], atol=1e-8)


def test_factor_vectors_definition():
    """Eq. mmexp: X = sum sqrt(lambda_j) U_j V_j^T with orthonormal U, V."""
    rng = np.random.default_rng(5)
    P = O.Problem.image(rng.normal(size=(9, 8)), 3, 3)
    X = P.matrix()
    s, U, V = O.decompose(P, min(X.shape))
    np.testing.assert_allclose(U * s @ V.T, X, atol=1e-11)
    np.testing.assert_allclose(V.T @ V, np.eye(len(s)), atol=1e-11)


def test_rank_exponential_and_sinusoid():
    """Sec. 2.2: an exponential has rank 1, a sine wave rank 2."""
    t = np.arange(1, 201, dtype=float)
    for s, thr in sigmas(O.Problem.series(np.exp(0.01 * t), 50), 6):
        assert rank_of(s, thr) == 1
    for s, thr in sigmas(O.Problem.series(3 * np.sin(2 * np.pi * t / 17 + 0.3), 50), 6):
        assert rank_of(s, thr) == 2


def test_closed_form_sinusoid_singular_values():
    """Appendix A.1, Example ex:mssa_ev: with L*omega, K*omega integer one
    sinusoid A cos(2 pi omega k + phi) gives lambda_1 = lambda_2 = A^2 L K / 4,
    i.e. sigma = A sqrt(L K) / 2."""
    A, omega, phi = 2.5, 1 / 10, 0.7
    L, K = 40, 60                       # L*omega = 4, K*omega = 6
    N = L + K - 1
    k = np.arange(N)
    expect = A * math.sqrt(L * K) / 2
    for s, thr in sigmas(O.Problem.series(A * np.cos(2 * np.pi * omega * k + phi), L), 4):
        np.testing.assert_allclose(s[:2], [expect, expect], rtol=1e-12)
        assert s[2] < thr * expect


def test_closed_form_mssa_pair():
    """Example ex:mssa_ev: the MSSA pair has lambda_1 = lambda_2 =
    (A^2 + B^2) L K / 4 where K is each series' K (equal lengths)."""
    vals = paper_values()["mssa_equal_eigenvalues"]
    assert "A^2+B^2" in vals["cite"]
    A, B, omega = 1.5, 0.8, 1 / 8
    L, Kp = 24, 40
    N = L + Kp - 1
    k = np.arange(N)
    xs = [A * np.cos(2 * np.pi * omega * k + 0.2), B * np.cos(2 * np.pi * omega * k + 1.9)]
    expect = math.sqrt((A * A + B * B) * L * Kp / 4)
    for s, thr in sigmas(O.Problem.multi(xs, L), 4):
        np.testing.assert_allclose(s[:2], [expect, expect], rtol=1e-12)
        assert s[2] < thr * expect


def test_closed_form_2d_product_of_cosines():
    """Rank-4 product of cosines (Appendix A.2 example: a product of sines is
    two planar sines, each of 2D rank 2).  The HbH matrix of A a_m b_n is
    A T(b) kron T(a) (eq. rank_one_circ restricted to the window), so with
    integer L*omega and K*omega on both axes the four non-zero singular values
    all equal A sqrt(Lx Kx) sqrt(Ly Ky) / 4."""
    A = 1.7
    nx, ny, lx, ly = 29, 23, 10, 8          # Kx = 20, Ky = 16
    wx, wy = 1 / 10, 1 / 8                 # Lx wx = 1, Kx wx = 2; Ly wy = 1, Ky wy = 2
    m = np.arange(nx)[:, None]
    n = np.arange(ny)[None, :]
    x = A * np.cos(2 * np.pi * wx * m + 0.4) * np.cos(2 * np.pi * wy * n + 1.1)
    kx, ky = nx - lx + 1, ny - ly + 1
    expect = A * math.sqrt(lx * kx) * math.sqrt(ly * ky) / 4
    for s, thr in sigmas(O.Problem.image(x, lx, ly), 6):
        np.testing.assert_allclose(s[:4], [expect] * 4, rtol=1e-11)
        assert s[4] < thr * expect
    # off the integer grid the values split but the rank stays 4
    x = A * np.cos(2 * np.pi * 0.137 * m + 0.4) * np.cos(2 * np.pi * 0.071 * n + 1.1)
    for s, thr in sigmas(O.Problem.image(x, lx, ly), 8):
        assert rank_of(s, thr) == 4


def test_tab_dim_ranks():
    """Table tab:dim: ranks of Examples A, B, C under SSA (each series) and
    MSSA (both series)."""
    tab = paper_values()["tab_dim"]
    N = tab["N"]
    k = np.arange(1, N + 1)
    for name, ex in tab["examples"].items():
        xs = [a * np.cos(2 * np.pi * k / per + ph) for a, per, ph in (ex["h1"], ex["h2"])]
        for x in xs:
            for s, thr in sigmas(O.Problem.series(x, 24), 8):
                assert rank_of(s, thr) == ex["ssa_rank"], name
        for s, thr in sigmas(O.Problem.multi(xs, 24), 8):
            assert rank_of(s, thr) == ex["mssa_rank"], name


def test_L_and_N_minus_L_plus_1_coincide():
    """Sec. 3.2 remark 3: for one series the expansions for L and N-L+1
    coincide (the trajectory matrices are transposes)."""
    rng = np.random.default_rng(6)
    x = rng.normal(size=50)
    s1 = O.decompose(O.Problem.series(x, 13), 13)[0]
    s2 = O.decompose(O.Problem.series(x, 38), 13)[0]
    np.testing.assert_allclose(s1, s2, rtol=1e-10)


# ------------------------------------------------------------ reduction identities
def test_shaped_full_masks_equal_2d():
    """Sec. 5.1 comments: ShSSA with full rectangles coincides with 2D-SSA."""
    rng = np.random.default_rng(7)
    x = rng.normal(size=(10, 9))
    a = O.Problem.image(x, 4, 3).matrix()
    b = O.Problem.image(x, 4, 3, wmask=np.ones((4, 3), bool),
                        mask=np.ones((10, 9), bool)).matrix()
    np.testing.assert_array_equal(a, b)


def test_2d_with_ly_1_equals_mssa():
    """Sec. 4.1 comment 1: 2D-SSA with Ly = 1 is MSSA of the image columns."""
    rng = np.random.default_rng(8)
    x = rng.normal(size=(12, 5))
    a = O.Problem.image(x, 4, 1).matrix()
    b = O.Problem.multi([x[:, j] for j in range(5)], 4).matrix()
    np.testing.assert_array_equal(a, b)


def test_mssa_equals_shaped_2d_packing():
    """Sec. 5.3: MSSA of unequal series equals ShSSA of the N_max x s array,
    each series in one column, with the unused cells masked out."""
    rng = np.random.default_rng(9)
    xs = [rng.normal(size=n) for n in (15, 11, 13)]
    nmax = max(len(x) for x in xs)
    img = np.full((nmax, len(xs)), np.nan)
    for j, x in enumerate(xs):
        img[:len(x), j] = x
    a = O.Problem.multi(xs, 5).matrix()
    b = O.Problem.image(img, 5, 1).matrix()
    np.testing.assert_array_equal(a, b)


def test_ssa_equals_shaped_n_by_1():
    """Sec. 5.3: SSA is ShSSA of an N x 1 array with an L x 1 window."""
    x = np.random.default_rng(10).normal(size=30)
    np.testing.assert_array_equal(O.Problem.series(x, 7).matrix(),
                                  O.Problem.image(x.reshape(-1, 1), 7, 1).matrix())


# ------------------------------------------------------------ reconstruction
def test_sum_of_elementary_components_is_input():
    """Eq. res_decomp: the elementary components (grouping {1}, ..., {d}) sum
    to the input, for SSA, MSSA and a shaped image."""
    rng = np.random.default_rng(11)
    cases = [O.Problem.series(rng.normal(size=40), 9),
             O.Problem.multi([rng.normal(size=n) for n in (20, 26)], 6)]
    img = rng.normal(size=(11, 10))
    img[3, 4] = np.nan
    cases.append(O.Problem.image(img, 3, 3, wmask=np.array(
        [[1, 1, 0], [1, 1, 1], [0, 1, 1]], bool)))
    for P in cases:
        d = min(P.L, P.K)
        s, U, V = O.decompose(P, d)
        comps = O.reconstruct(P, s, U, V, [[i] for i in range(len(s))])
        for c, x in enumerate(P.channels):
            total = sum(comp[c] for comp in comps)
            ok = P.weights(c) > 0
            np.testing.assert_allclose(total[ok], x[ok], atol=1e-10)
            assert np.all(np.isnan(total[~ok]))


def test_reconstruction_brute_force_antidiagonals():
    """Diagonal averaging of one rank-one term, by explicit loops over the
    anti-diagonals (Sec. 2.1, Step 4)."""
    rng = np.random.default_rng(12)
    x = rng.normal(size=17)
    L = 6
    P = O.Problem.series(x, L)
    s, U, V = O.decompose(P, 3)
    rec = O.reconstruct(P, s, U, V, [[1]])[0][0][:, 0]
    K = 17 - L + 1
    Y = s[1] * np.outer(U[:, 1], V[:, 1])
    for k in range(17):
        vals = [Y[i, k - i] for i in range(L) if 0 <= k - i < K]
        assert abs(rec[k] - sum(vals) / len(vals)) < 1e-13


def test_finite_rank_signal_is_recovered_exactly():
    """Sec. 2.2: a series of finite rank r reconstructs to itself from its r
    components; an exponential + sinusoid has rank 3."""
    t = np.arange(1, 121, dtype=float)
    x = 2 * np.exp(0.01 * t) + np.sin(2 * np.pi * t / 9 + 0.5)
    P = O.Problem.series(x, 40)
    s, U, V = O.decompose(P, 5)
    assert rank_of(s, 1e-6) == 3
    rec = O.reconstruct(P, s, U, V, [[0, 1, 2]])[0][0][:, 0]
    np.testing.assert_allclose(rec, x, atol=1e-9)


def test_reconstruct_at_matches_full_reconstruction():
    """The one-element-at-a-time route (used on full-size workloads) agrees
    with the full averaging on a shaped image."""
    rng = np.random.default_rng(13)
    img = rng.normal(size=(14, 12))
    img[5:7, 4:6] = np.nan
    P = O.Problem.image(img, 4, 3)
    s, U, V = O.decompose(P, 6)
    full = O.reconstruct(P, s, U, V, [[0, 1, 2]])[0][0]
    pts = [(0, 0), (13, 11), (6, 3), (8, 7), (5, 4)]
    got = O.reconstruct_at(P, U[:, :3], pts)
    for (m, n), g in zip(pts, got):
        if np.isnan(full[m, n]):
            assert np.isnan(g)
        else:
            assert abs(g - full[m, n]) < 1e-10


# ------------------------------------------------------------ long-series entry routes
def test_series_rows_cols_geometric_closed_form():
    """x_t = q^t gives X_ij = q^i q^j (eq. ssa_embedding): every row of X v is
    q^i times the same sum, every column of X^T u q^j times another."""
    q = 0.999
    n, L = 300, 120
    K = n - L + 1
    x = q ** np.arange(n)
    rng = np.random.default_rng(3)
    v, u = rng.normal(size=K), rng.normal(size=L)
    rows, cols = [0, 7, 119], [0, 50, 180]
    sv = float(np.sum(q ** np.arange(K) * v))
    su = float(np.sum(q ** np.arange(L) * u))
    np.testing.assert_allclose(O.series_rows(x, L, rows, v), [q ** i * sv for i in rows], rtol=1e-12)
    np.testing.assert_allclose(O.series_cols(x, L, cols, u), [q ** j * su for j in cols], rtol=1e-12)


def test_series_rows_cols_match_trajectory_products():
    """Single rows / columns agree with the full products of the explicit
    trajectory matrix (pinned to the printed Hankel form above)."""
    rng = np.random.default_rng(4)
    x = rng.normal(size=97)
    L = 40
    P = O.Problem.series(x, L)
    v, u = rng.normal(size=P.K), rng.normal(size=P.L)
    np.testing.assert_allclose(O.series_rows(x, L, range(P.L), v), O.matvec(P, v), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(O.series_cols(x, L, range(P.K), u), O.rmatvec(P, u), rtol=1e-12, atol=1e-12)


def test_series_hankelize_at_full_sum_is_input_and_matches_groups():
    """All elementary components of a full decomposition sum to the series
    (Sec. 2.1, Step 4), element by element; a single group agrees with the
    full diagonal averaging."""
    rng = np.random.default_rng(5)
    n, L = 60, 25
    t = np.arange(n)
    x = np.sin(2 * np.pi * t / 9) + 0.3 * rng.normal(size=n)
    P = O.Problem.series(x, L)
    s, U, V = O.decompose(P, L, "jacobi")
    pts = list(range(n))
    np.testing.assert_allclose(O.series_hankelize_at(s, U, V, range(len(s)), pts), x, atol=1e-10)
    full = O.reconstruct(P, s, U, V, [[0, 1]])[0][0][:, 0]
    np.testing.assert_allclose(O.series_hankelize_at(s, U, V, [0, 1], pts), full, atol=1e-12)


# ---------------------------------------------------------------- w-correlations
def test_w_inner_is_frobenius_product_of_trajectory_matrices():
    """Sec. 2.2: each element y_k sits in w_k = |A_k| entries of T(Y), so
    (Y, Z)_w = <T(Y), T(Z)>_F for any Y, Z -- checked on random objects for a
    shaped image with holes and an MSSA system, the trajectory matrices built
    entry by entry."""
    rng = np.random.default_rng(3)
    x = rng.normal(size=(15, 13))
    mask = np.ones((15, 13), bool)
    mask[4:7, 5:8] = False
    wmask = np.array([[1, 1, 0], [1, 1, 1], [1, 1, 1], [0, 1, 1]], bool)
    P2 = O.Problem.image(x, 4, 3, wmask=wmask, mask=mask)
    Pm = O.Problem.multi([rng.normal(size=n) for n in (23, 31, 19)], 7)
    for P in (P2, Pm):
        ys = [rng.normal(size=c.shape) for c in P.channels]
        zs = [rng.normal(size=c.shape) for c in P.channels]
        frob = sum(float(np.sum(O.trajectory_columns(ys[c], P.Lset, P.Ksets[c])
                                * O.trajectory_columns(zs[c], P.Lset, P.Ksets[c])))
                   for c in range(len(P.channels)))
        assert abs(O.w_inner(P, ys, zs) - frob) <= 1e-12 * abs(frob) + 1e-12


def test_wcor_exactly_separable_harmonics():
    """Two harmonics with periods 8 and 4 and L, K multiples of 8 have
    orthogonal trajectory rows and columns (weak separability, Sec. 2.2): the
    reconstructions of the two rank-2 groups are the harmonics themselves, so
    their w-correlation is 0, each self-correlation 1, and the contributions
    are the harmonics' weighted energies, summing to 1."""
    L, K = 16, 32
    n = np.arange(L + K - 1, dtype=float)
    x1 = 2.0 * np.cos(2 * np.pi * n / 8 + 0.4)
    x2 = np.cos(2 * np.pi * n / 4 + 0.3)
    P = O.Problem.series(x1 + x2, L)
    sig, U, V = O.decompose(P, 4)
    rho, contrib = O.wcor(P, sig, U, V, [[0, 1], [2, 3]])
    np.testing.assert_allclose(np.diag(rho), 1.0, atol=1e-12)
    assert abs(rho[0, 1]) <= 1e-10 and rho[0, 1] == rho[1, 0]
    w = np.minimum.reduce([n + 1, np.full_like(n, L), np.full_like(n, K), len(n) - n])   # 1D weights
    xx = np.sum(w * (x1 + x2) ** 2)
    np.testing.assert_allclose(contrib, [np.sum(w * x1 ** 2) / xx, np.sum(w * x2 ** 2) / xx], rtol=1e-10)
    assert abs(contrib.sum() - 1.0) <= 1e-10


def test_wcor_invariants_on_noisy_image():
    """Elementary w-correlations of a shaped 2D decomposition: symmetric,
    unit diagonal, |rho| <= 1 (Cauchy-Schwarz in the weighted inner product);
    a component that mixes two others is correlated with both."""
    rng = np.random.default_rng(8)
    i, j = np.meshgrid(np.arange(20), np.arange(18), indexing="ij")
    x = np.cos(2 * np.pi * i / 7) * np.cos(2 * np.pi * j / 5) + 0.3 * rng.normal(size=i.shape)
    P = O.Problem.image(x, 6, 5)
    sig, U, V = O.decompose(P, 6)
    rho, contrib = O.wcor(P, sig, U, V, [[k] for k in range(6)])
    np.testing.assert_allclose(rho, rho.T, atol=0)
    np.testing.assert_allclose(np.diag(rho), 1.0, atol=1e-12)
    assert np.all(np.abs(rho) <= 1 + 1e-12)
    assert np.all(contrib > 0) and contrib.sum() < 1.0 + 1e-12
    rho2, _ = O.wcor(P, sig, U, V, [[0], [1], [0, 1]])
    assert rho2[0, 2] > 0.3 and rho2[1, 2] > 0.3


# ---------------------------------------------------------------- forecasting
def test_lrr_reproduces_last_coordinate_of_the_subspace():
    """R_L of eq. Forec:ContMSSAL is the recurrence of the subspace: for every
    vector of span(U_I), its last coordinate is R_L . (the others)."""
    rng = np.random.default_rng(4)
    Q, _ = np.linalg.qr(rng.normal(size=(15, 3)))
    R = O.lrr_column(Q)
    for j in range(3):
        assert abs(R @ Q[:-1, j] - Q[-1, j]) <= 1e-12
    y = Q @ rng.normal(size=3)
    assert abs(R @ y[:-1] - y[-1]) <= 1e-12
    e = np.zeros((15, 1))
    e[-1, 0] = 1.0
    with pytest.raises(ValueError):
        O.lrr_column(e)                      # nu^2 = 1: no recurrence


def test_recurrent_forecast_continues_a_finite_rank_series_exactly():
    """A sum of two damped / growing harmonics has rank 4 and satisfies an
    LRR; its reconstruction by the 4 leading triples is the series itself and
    the recurrent forecast is its exact continuation (Sec. 3.3)."""
    n = np.arange(75, dtype=float)
    f = 1.01 ** n * np.cos(2 * np.pi * n / 9 + 0.2) + 0.5 * 0.99 ** n * np.cos(2 * np.pi * n / 5)
    P = O.Problem.series(f[:60], 20)
    sig, U, V = O.decompose(P, 4)
    (fc,) = O.forecast_recurrent_column(P, sig, U, V, [0, 1, 2, 3], 15)
    np.testing.assert_allclose(fc, f[60:], rtol=1e-8, atol=1e-8)


def test_recurrent_column_forecast_mssa_common_recurrence():
    """Two series of one frequency (different phases, amplitudes and
    lengths) span a common rank-2 column space; one recurrence continues both
    exactly (column forecast: the same LRR, different initial data)."""
    n = np.arange(70, dtype=float)
    x1 = np.cos(2 * np.pi * n / 7)
    x2 = 2.0 * np.sin(2 * np.pi * n / 7 + 0.5)
    P = O.Problem.multi([x1[:40], x2[:50]], 12)
    sig, U, V = O.decompose(P, 2)
    f1, f2 = O.forecast_recurrent_column(P, sig, U, V, [0, 1], 10)
    np.testing.assert_allclose(f1, x1[40:50], atol=1e-9)
    np.testing.assert_allclose(f2, x2[50:60], atol=1e-9)


def test_vector_forecast_continues_finite_rank_series_exactly():
    """The vector column forecast (Sec. 3.3, eqs. PGcolumn, V_FORcolumn)
    continues a finite-rank series exactly, for one series and for an MSSA
    pair sharing its column space."""
    n = np.arange(75, dtype=float)
    f = 1.01 ** n * np.cos(2 * np.pi * n / 9 + 0.2) + 0.5 * 0.99 ** n * np.cos(2 * np.pi * n / 5)
    P = O.Problem.series(f[:60], 20)
    sig, U, V = O.decompose(P, 4)
    (fc,) = O.forecast_vector_column(P, sig, U, V, [0, 1, 2, 3], 15)
    np.testing.assert_allclose(fc, f[60:], rtol=1e-8, atol=1e-8)
    n = np.arange(70, dtype=float)
    x1 = np.cos(2 * np.pi * n / 7)
    x2 = 2.0 * np.sin(2 * np.pi * n / 7 + 0.5)
    P = O.Problem.multi([x1[:40], x2[:50]], 12)
    sig, U, V = O.decompose(P, 2)
    f1, f2 = O.forecast_vector_column(P, sig, U, V, [0, 1], 10)
    np.testing.assert_allclose(f1, x1[40:50], atol=1e-9)
    np.testing.assert_allclose(f2, x2[50:60], atol=1e-9)


@pytest.mark.parametrize("lens", [(40, 40), (40, 50)])
def test_row_forecasts_continue_an_mssa_pair_exactly(lens):
    """Recurrent and vector row forecasts (Sec. 3.3, eqs. Forec:ContMSSAK,
    PGrow, V_FORrow) continue a finite-rank MSSA pair exactly, for equal and
    unequal series lengths."""
    n = np.arange(70, dtype=float)
    x1 = np.cos(2 * np.pi * n / 7)
    x2 = 2.0 * np.sin(2 * np.pi * n / 7 + 0.5)
    P = O.Problem.multi([x1[:lens[0]], x2[:lens[1]]], 12)
    sig, U, V = O.decompose(P, 2)
    for fn in (O.forecast_recurrent_row, O.forecast_vector_row):
        f1, f2 = fn(P, sig, U, V, [0, 1], 10)
        np.testing.assert_allclose(f1, x1[lens[0]:lens[0] + 10], atol=1e-9)
        np.testing.assert_allclose(f2, x2[lens[1]:lens[1] + 10], atol=1e-9)

