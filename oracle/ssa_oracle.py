"""CPU FP64 oracle for SSA, MSSA, 2D-SSA and Shaped 2D-SSA.

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously correct
statement of what the GPU library computes.  Only the test-suite, the smoke
check and the benchmark's CPU-baseline leg may import it; the library never
does, and the library fails loudly instead of falling back to it.

It shares no code with the CUDA path: no FFT, no Lanczos, no packed spectra.
Every quantity is formed from its definition in the paper:

* shapes -- the window set (Sec. 5.1, ordered lexicographically = column-major),
  the origin set ``K = {kappa : L (+) {kappa} subset N}`` (eq. sh_Ks) by brute
  force over all origins, and the reconstructable set ``N' = L (+) K``;
* the trajectory matrix -- built entry by entry from ``X_ij = x_{l_i (+) k_j}``
  (eq. ssa_embedding for 1D, eq. mssa_embedding for stacked series, eqs.
  block_hankel_cols / qh_mat for images), using 0-based indices, so the paper's
  shifted sum ``l (+) k = l + k - 1`` becomes ``l + k``;
* the SVD step -- exactly as Step 2 of Sec. 2.1 states it: ``S = X X^T``,
  eigenvalues ``lambda_1 >= ...`` with eigenvectors ``U_j`` and factor vectors
  ``V_j = X^T U_j / sqrt(lambda_j)`` (eq. mmexp); a one-sided Jacobi SVD of the
  explicit matrix is kept beside it as an independent second route;
* reconstruction -- the projection ``Pi^(H)`` of Step 4 written out: every
  entry ``(i, j)`` of the grouped matrix is added into the data element
  ``l_i (+) k_j`` and divided by the count ``w_k = |A_k|`` of entries that map
  there (eq. res_decomp and the averaging formula above it);
* beyond the hot path -- the weighted inner product and w-correlations of
  Sec. 2.2 summed element by element, and the four MSSA forecasts of Sec. 3.3
  (recurrent and vector, column and row) with their projectors and
  recurrences formed explicitly and applied step by step.

A "problem" is a list of channels (one for 1D and 2D, ``s`` for MSSA), each an
``(Nx, Ny)`` float64 array with NaN marking missing values, sharing one window
shape.  The MSSA trajectory matrix is the horizontal stack of the channels'
matrices (eq. mssa_embedding); a 1D series of length N is the ``(N, 1)`` array.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "Problem", "window_set", "origin_set", "trajectory_matrix",
    "trajectory_columns", "weights", "svd_eigen", "svd_eigen_t", "svd_jacobi", "decompose",
    "reconstruct", "reconstruct_at", "matvec", "rmatvec",
    "series_rows", "series_cols", "series_hankelize_at", "w_inner", "wcor",
    "lrr_column", "forecast_recurrent_column", "forecast_vector_column",
    "forecast_recurrent_row", "forecast_vector_row",
]


# ---------------------------------------------------------------- shapes
def window_set(lx: int, ly: int = 1, wmask=None) -> np.ndarray:
    """Window shape as an ``(L, 2)`` int array of 0-based ``(l_x, l_y)``.

    Lexicographic order in the paper's sense (Sec. 5.1: the order in which the
    elements appear in the column-major vectorisation), i.e. sorted by
    ``l_y`` then ``l_x``.  ``wmask`` (``lx x ly`` bool) selects a sub-shape.
    """
    if wmask is None:
        wmask = np.ones((lx, ly), dtype=bool)
    wmask = np.asarray(wmask, dtype=bool)
    assert wmask.shape == (lx, ly)
    out = [(a, b) for b in range(ly) for a in range(lx) if wmask[a, b]]
    return np.array(out, dtype=np.int64).reshape(-1, 2)


def observed(x: np.ndarray, mask=None) -> np.ndarray:
    """The set N: pixels that are inside ``mask`` and not NaN (Sec. 5.2: NA
    values and the user mask are both excluded)."""
    ok = ~np.isnan(x)
    if mask is not None:
        ok &= np.asarray(mask, dtype=bool)
    return ok


def origin_set(obs: np.ndarray, Lset: np.ndarray) -> np.ndarray:
    """All origins ``kappa`` with ``L (+) {kappa}`` inside N (eq. sh_Ks).

    Every candidate origin of the grid starts admissible and is struck out as
    soon as one window element ``l + kappa`` falls on a pixel outside N (one
    shifted comparison of the whole grid per window element).  Returned as a
    ``(K, 2)`` array in lexicographic (column-major) order.
    """
    nx, ny = obs.shape
    ex = int(Lset[:, 0].max()) + 1
    ey = int(Lset[:, 1].max()) + 1
    cx, cy = nx - ex + 1, ny - ey + 1          # origins keeping the box inside
    if cx <= 0 or cy <= 0:
        return np.zeros((0, 2), dtype=np.int64)
    ok = np.ones((cx, cy), dtype=bool)
    for (lx, ly) in Lset:
        ok &= obs[lx:lx + cx, ly:ly + cy]
    kx, ky = np.nonzero(ok.T)                  # column-major order: ky outer
    return np.stack([ky, kx], axis=1).astype(np.int64)


def trajectory_columns(x: np.ndarray, Lset: np.ndarray, Kset: np.ndarray,
                       cols=None) -> np.ndarray:
    """Columns ``cols`` of the trajectory matrix: ``X_ij = x[l_i + k_j]``.

    Eq. qh_mat with 0-based indices; for a full rectangle this is the
    Hankel-block-Hankel matrix of eq. block_hankel_matrix and for a series the
    Hankel matrix of eq. ssa_embedding.
    """
    if cols is None:
        cols = np.arange(len(Kset))
    px = Lset[:, 0][:, None] + Kset[cols, 0][None, :]
    py = Lset[:, 1][:, None] + Kset[cols, 1][None, :]
    return np.asarray(x, dtype=np.float64)[px, py]


def trajectory_matrix(x: np.ndarray, Lset: np.ndarray, Kset: np.ndarray) -> np.ndarray:
    """The full ``L x K`` trajectory matrix of one channel."""
    return trajectory_columns(x, Lset, Kset)


def weights(shape, Lset: np.ndarray, Kset: np.ndarray) -> np.ndarray:
    """``w_k = |A_k|``: how many trajectory entries hold data element k.

    Counted directly: for every window element l, each origin kappa adds one
    at ``l + kappa``.  Zero outside N' (the elements that never enter the
    trajectory matrix, Sec. 5.1).
    """
    nx, ny = shape
    w = np.zeros((nx, ny), dtype=np.int64)
    ind = np.zeros((nx, ny), dtype=np.int64)
    ind[Kset[:, 0], Kset[:, 1]] = 1
    for (lx, ly) in Lset:
        w[lx:, ly:] += ind[:nx - lx, :ny - ly]
    return w


# ---------------------------------------------------------------- problem
class Problem:
    """Channels sharing one window shape; see the module docstring."""

    def __init__(self, channels, lx: int, ly: int = 1, wmask=None, masks=None):
        self.channels = [np.asarray(c, dtype=np.float64).reshape(c.shape[0], -1)
                         for c in channels]
        if masks is None:
            masks = [None] * len(self.channels)
        self.obs = [observed(c, m) for c, m in zip(self.channels, masks)]
        self.Lset = window_set(lx, ly, wmask)
        self.Ksets = [origin_set(o, self.Lset) for o in self.obs]
        self.L = len(self.Lset)
        self.Ks = [len(k) for k in self.Ksets]
        self.K = int(sum(self.Ks))
        self.offsets = np.concatenate([[0], np.cumsum(self.Ks)]).astype(np.int64)

    @classmethod
    def series(cls, x, L: int):
        """Basic SSA of one series (eq. ssa_embedding)."""
        x = np.asarray(x, dtype=np.float64)
        return cls([x.reshape(-1, 1)], L, 1)

    @classmethod
    def multi(cls, xs, L: int):
        """MSSA of a system of series of possibly unequal lengths
        (eq. mssa_embedding)."""
        return cls([np.asarray(x, dtype=np.float64).reshape(-1, 1) for x in xs], L, 1)

    @classmethod
    def image(cls, x, lx: int, ly: int, wmask=None, mask=None):
        """2D-SSA (full window and image) or Shaped 2D-SSA (wmask / mask /
        NaN pixels)."""
        return cls([np.asarray(x, dtype=np.float64)], lx, ly, wmask=wmask,
                   masks=[mask])

    def block(self, c: int, cols=None) -> np.ndarray:
        """Columns of channel c's trajectory matrix."""
        return trajectory_columns(self.channels[c], self.Lset, self.Ksets[c], cols)

    def matrix(self) -> np.ndarray:
        """The stacked ``L x K`` trajectory matrix ``[X^(1) : ... : X^(s)]``."""
        return np.hstack([self.block(c) for c in range(len(self.channels))])

    def weights(self, c: int = 0) -> np.ndarray:
        return weights(self.channels[c].shape, self.Lset, self.Ksets[c])

    def column_blocks(self, width: int = 4096):
        """Yield ``(global_col0, X_block)`` over all channels, in column order."""
        for c in range(len(self.channels)):
            for j0 in range(0, self.Ks[c], width):
                cols = np.arange(j0, min(j0 + width, self.Ks[c]))
                yield int(self.offsets[c] + j0), self.block(c, cols)


# ---------------------------------------------------------------- matvec
def matvec(P: Problem, v: np.ndarray) -> np.ndarray:
    """``u = X v`` with the explicit trajectory matrix (column blocks)."""
    u = np.zeros(P.L)
    for j0, Xb in P.column_blocks():
        u += Xb @ v[j0:j0 + Xb.shape[1]]
    return u


def rmatvec(P: Problem, u: np.ndarray) -> np.ndarray:
    """``v = X^T u`` with the explicit trajectory matrix."""
    v = np.zeros(P.K)
    for j0, Xb in P.column_blocks():
        v[j0:j0 + Xb.shape[1]] = Xb.T @ u
    return v


# ---------------------------------------------------------------- SVD step
def svd_eigen(P: Problem, r: int | None = None):
    """Step 2 of Sec. 2.1 as written: ``S = X X^T``; its eigenvalues in
    decreasing order with eigenvectors ``U_j``; ``sqrt(lambda_j)`` are the
    singular values and ``V_j = X^T U_j / sqrt(lambda_j)`` the factor vectors.

    ``S`` is summed over column blocks of X (a matrix product split by
    columns).  Returns ``sigma (r,), U (L, r), V (K, r)``.
    """
    S = np.zeros((P.L, P.L))
    for _, Xb in P.column_blocks():
        S += Xb @ Xb.T
    lam, U = np.linalg.eigh(S)
    order = np.argsort(lam)[::-1]
    lam, U = lam[order], U[:, order]
    d = int(np.sum(lam > lam[0] * 1e-28)) if lam[0] > 0 else 0
    if r is None:
        r = d
    r = min(r, d)
    lam, U = lam[:r], U[:, :r]
    sigma = np.sqrt(lam)
    V = np.zeros((P.K, r))
    for j0, Xb in P.column_blocks():
        V[j0:j0 + Xb.shape[1]] = Xb.T @ U
    V /= sigma[None, :]
    return sigma, U, V


def svd_eigen_t(P: Problem, r: int | None = None):
    """Step 2 of Sec. 2.1 applied to ``X^T`` (for ``K < L``): the singular
    triples of ``X^T`` are those of ``X`` with U and V exchanged, so
    ``S' = X^T X`` (K x K) gives ``V_j`` and ``sigma_j``, and
    ``U_j = X V_j / sigma_j``.  Forms the explicit matrix; meant for small K.
    """
    X = P.matrix()
    lam, V = np.linalg.eigh(X.T @ X)
    order = np.argsort(lam)[::-1]
    lam, V = lam[order], V[:, order]
    d = int(np.sum(lam > lam[0] * 1e-28)) if lam[0] > 0 else 0
    if r is None:
        r = d
    r = min(r, d)
    sigma = np.sqrt(lam[:r])
    V = V[:, :r]
    U = (X @ V) / sigma[None, :]
    return sigma, U, V


def _round_robin(n: int):
    """Pairings of a round-robin tournament on n (even) players: n-1 rounds of
    n/2 disjoint pairs covering every pair once."""
    players = list(range(n))
    rounds = []
    for _ in range(n - 1):
        half = n // 2
        rounds.append((np.array(players[:half]), np.array(players[half:][::-1])))
        players = [players[0]] + [players[-1]] + players[1:-1]
    return rounds


def svd_jacobi(X: np.ndarray, tol: float = 1e-15, max_sweeps: int = 80):
    """One-sided (Hestenes) Jacobi SVD of an explicit matrix.

    Columns of the (tall) working matrix are rotated pairwise until every pair
    is orthogonal to ``|a.b| <= tol |a||b|``; singular values are the final
    column norms.  Returns ``sigma (n,), U (m, n), V (q, n)`` with
    ``X = U diag(sigma) V^T`` and sigma decreasing, n = min(m, q).
    """
    X = np.asarray(X, dtype=np.float64)
    transpose = X.shape[1] > X.shape[0]
    A = (X.T if transpose else X).copy()          # tall: m >= n
    m, n = A.shape
    n2 = n + (n % 2)
    if n2 != n:
        A = np.hstack([A, np.zeros((m, 1))])
    R = np.eye(n2)
    rounds = _round_robin(n2)
    for _ in range(max_sweeps):
        rotated = False
        for p, q in rounds:
            a, b = A[:, p], A[:, q]
            alpha = np.einsum("ij,ij->j", a, a)
            beta = np.einsum("ij,ij->j", b, b)
            gamma = np.einsum("ij,ij->j", a, b)
            need = np.abs(gamma) > tol * np.sqrt(alpha * beta)
            if not np.any(need):
                continue
            rotated = True
            g = np.where(need, gamma, 1.0)
            zeta = (beta - alpha) / (2.0 * g)
            t = np.sign(zeta) / (np.abs(zeta) + np.sqrt(1.0 + zeta * zeta))
            t = np.where(zeta == 0, 1.0, t)
            t = np.where(need, t, 0.0)
            c = 1.0 / np.sqrt(1.0 + t * t)
            s = c * t
            A[:, p], A[:, q] = c * a - s * b, s * a + c * b
            rp, rq = R[:, p], R[:, q]
            R[:, p], R[:, q] = c * rp - s * rq, s * rp + c * rq
        if not rotated:
            break
    A, R = A[:, :n], R[:n, :n]
    sigma = np.linalg.norm(A, axis=0)
    order = np.argsort(sigma)[::-1]
    sigma, A, R = sigma[order], A[:, order], R[:, order]
    safe = np.where(sigma > 0, sigma, 1.0)
    W = A / safe[None, :]
    if transpose:          # X^T = W diag(sigma) R^T  =>  X = R diag(sigma) W^T
        return sigma, R, W
    return sigma, W, R


def decompose(P: Problem, r: int, method: str = "eigen"):
    """The r leading eigentriples ``(sigma, U, V)`` of the trajectory matrix,
    each pair ``(U_i, V_i)`` signed so that the largest-magnitude entry of U_i
    is positive (singular vectors are defined up to sign, Sec. 3.4)."""
    if method == "eigen":
        sigma, U, V = svd_eigen(P, r)
    elif method == "eigen_t":
        sigma, U, V = svd_eigen_t(P, r)
    elif method == "jacobi":
        sigma, U, V = svd_jacobi(P.matrix())
        sigma, U, V = sigma[:r], U[:, :r], V[:, :r]
    else:
        raise ValueError(method)
    for i in range(U.shape[1]):
        if U[np.argmax(np.abs(U[:, i])), i] < 0:
            U[:, i] *= -1
            V[:, i] *= -1
    return sigma, U, V


# ---------------------------------------------------------------- reconstruction
def reconstruct(P: Problem, sigma, U, V, groups, residual: bool = False):
    """Step 4 of Sec. 2.1: for each group I, ``X_I = sum_{i in I} sigma_i U_i
    V_i^T`` is averaged over the sets ``A_k`` (diagonal averaging).

    Returns ``out[g][c]``: an array of channel c's shape with NaN outside N'.
    With ``residual`` one more group ``x - sum_g x~_g`` (on N') is appended.
    """
    sigma = np.asarray(sigma, dtype=np.float64)
    out = []
    for g in groups:
        g = list(g)
        per_ch = []
        for c, x in enumerate(P.channels):
            nx, ny = x.shape
            Kc = P.Ksets[c]
            Vc = V[P.offsets[c]:P.offsets[c + 1]]
            Y = (U[:, g] * sigma[g][None, :]) @ Vc[:, g].T            # L x K_c
            # data element of entry (i, j): l_i + k_j, flattened column-major
            flat = ((P.Lset[:, 0][:, None] + Kc[:, 0][None, :])
                    + nx * (P.Lset[:, 1][:, None] + Kc[:, 1][None, :]))
            acc = np.bincount(flat.ravel(), weights=Y.ravel(),
                              minlength=nx * ny).reshape((nx, ny), order="F")
            cnt = np.bincount(flat.ravel(),
                              minlength=nx * ny).reshape((nx, ny), order="F")
            rec = np.full((nx, ny), np.nan)
            ok = cnt > 0
            rec[ok] = acc[ok] / cnt[ok]
            per_ch.append(rec)
        out.append(per_ch)
    if residual:
        res = []
        for c, x in enumerate(P.channels):
            r_ = x.copy()
            for g in range(len(groups)):
                r_ = r_ - out[g][c]
            res.append(r_)
        out.append(res)
    return out


def reconstruct_at(P: Problem, Ug: np.ndarray, points, c: int = 0) -> np.ndarray:
    """Reconstruction of the group spanned by the orthonormal columns ``Ug`` at
    selected data elements, one element at a time.

    Uses ``X_I = U_I U_I^T X`` (the group's matrix is the projection of X on
    its eigenvectors, since ``sigma_i V_i^T = U_i^T X``) and averages the
    entries of ``A_k`` for each requested ``k = (m, n)`` of channel c.
    """
    x = P.channels[c]
    Kc = P.Ksets[c]
    kindex = {(int(a), int(b)): j for j, (a, b) in enumerate(Kc)}
    vals = []
    for (m, n) in points:
        rows, cols = [], []
        for i, (lx, ly) in enumerate(P.Lset):
            j = kindex.get((m - int(lx), n - int(ly)))
            if j is not None:
                rows.append(i)
                cols.append(j)
        if not rows:
            vals.append(np.nan)
            continue
        Xc = trajectory_columns(x, P.Lset, Kc, np.array(cols))   # L x |A_k|
        proj = Ug @ (Ug.T @ Xc)                                   # L x |A_k|
        vals.append(float(np.mean(proj[np.array(rows), np.arange(len(rows))])))
    return np.array(vals)


# ---------------------------------------------------------------- long series, one entry at a time
# For series too long for an explicit trajectory matrix: single rows and
# columns of X, and single reconstructed elements, straight from the
# embedding X_ij = x_{i+j} (eq. ssa_embedding, 0-based) and the averaging of
# Step 4 (Sec. 2.1) over the anti-diagonal i + j = p.
def series_rows(x, L: int, rows, v) -> np.ndarray:
    """``(X v)_i`` for the listed rows i: ``sum_j x[i + j] v[j]``."""
    x = np.asarray(x, dtype=np.float64)
    K = len(x) - L + 1
    v = np.asarray(v, dtype=np.float64)
    return np.array([float(x[i:i + K] @ v) for i in rows])


def series_cols(x, L: int, cols, u) -> np.ndarray:
    """``(X^T u)_j`` for the listed columns j: ``sum_i x[i + j] u[i]``."""
    x = np.asarray(x, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    return np.array([float(x[j:j + L] @ u) for j in cols])


def series_hankelize_at(sigma, U, V, group, points) -> np.ndarray:
    """Element p of the reconstruction of ``group`` from the triples
    ``(sigma_i, U_i, V_i)``: the mean over the anti-diagonal ``i + j = p`` of
    ``sum_{c in group} sigma_c U[i, c] V[j, c]``."""
    L, K = U.shape[0], V.shape[0]
    g = list(group)
    s = np.asarray(sigma, dtype=np.float64)[g]
    out = []
    for p in points:
        i = np.arange(max(0, p - K + 1), min(p, L - 1) + 1)
        vals = (U[i][:, g] * s[None, :] * V[p - i][:, g]).sum(axis=1)
        out.append(float(vals.mean()))
    return np.array(out)


# ---------------------------------------------------------------- w-correlations
def w_inner(P: Problem, ys, zs) -> float:
    """Weighted inner product ``(Y, Z)_w = sum_k w_k y_k z_k`` (Sec. 2.2,
    paragraph Separability), summed over every channel; ``w_k = |A_k|`` is zero outside
    N', where the reconstructions hold NaN and are skipped."""
    tot = 0.0
    for c in range(len(P.channels)):
        w = P.weights(c).astype(np.float64)
        ok = w > 0
        tot += float(np.sum(w[ok] * np.asarray(ys[c])[ok] * np.asarray(zs[c])[ok]))
    return tot


def wcor(P: Problem, sigma, U, V, groups):
    """The w-correlation matrix of the reconstructed components of
    ``groups`` (Sec. 2.2): ``rho_ij = (X~_i, X~_j)_w / (||X~_i||_w ||X~_j||_w)``
    (means not subtracted; 0 when a norm is 0), and each component's
    contribution ``||X~_i||_w^2 / ||X||_w^2``.  Elementary grouping
    ``[[0], [1], ...]`` gives the w-correlation matrix of the paper."""
    rec = reconstruct(P, sigma, U, V, groups)
    n = len(groups)
    G = np.zeros((n, n))
    for i in range(n):
        for j in range(i, n):
            G[i, j] = G[j, i] = w_inner(P, rec[i], rec[j])
    xx = w_inner(P, P.channels, P.channels)
    d = np.sqrt(np.diag(G))
    rho = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if d[i] > 0 and d[j] > 0:
                rho[i, j] = G[i, j] / (d[i] * d[j])
    contrib = np.diag(G) / xx if xx > 0 else np.zeros(n)
    return rho, contrib


# ---------------------------------------------------------------- forecasting
def lrr_column(Ug: np.ndarray) -> np.ndarray:
    """The linear recurrence of the column recurrent forecast (Sec. 3.3,
    eq. Forec:ContMSSAL): with pi(U_j) the last coordinate of U_j and U_j
    without it written U_j', ``R_L = sum_j pi(U_j) U_j' / (1 - nu^2)``,
    ``nu^2 = sum_j pi(U_j)^2``; defined only when nu^2 < 1."""
    Ug = np.asarray(Ug, dtype=np.float64)
    pi = Ug[-1, :]
    nu2 = float(np.sum(pi * pi))
    if nu2 >= 1.0:
        raise ValueError("nu^2 >= 1: the subspace contains the last unit vector, no recurrence")
    return (Ug[:-1, :] @ pi) / (1.0 - nu2)


def forecast_recurrent_column(P: Problem, sigma, U, V, group, M: int):
    """M-step recurrent column forecast of every series of a 1D or MSSA
    problem (Sec. 3.3): the reconstruction of ``group`` is continued by
    ``x~_{N_p + 1} = R_L . (the last L - 1 values)`` applied M times, one
    recurrence R_L for all series.  Returns a list of M-vectors, one per
    series."""
    assert all(c.shape[1] == 1 for c in P.channels) and P.Lset[:, 1].max() == 0, "series problems only"
    L = P.L
    R = lrr_column(np.asarray(U)[:, list(group)])
    rec = reconstruct(P, sigma, U, V, [list(group)])[0]
    out = []
    for c in range(len(P.channels)):
        y = list(rec[c][:, 0])
        for _ in range(M):
            y.append(float(np.dot(R, y[len(y) - (L - 1):])))
        out.append(np.array(y[len(y) - M:]))
    return out


def forecast_vector_column(P: Problem, sigma, U, V, group, M: int):
    """M-step vector column forecast of every series of a 1D or MSSA problem
    (Sec. 3.3, vector forecasting, eqs. PGcolumn and V_FORcolumn).

    For series p the columns of the reconstructed matrix X^ = U_I U_I^T X^(p)
    (the lagged vectors projected on the group's column space) are continued
    by Z_j = [Pi Z_{j-1}' ; R_L . Z_{j-1}'] for j = K_p + 1 .. K_p + M + L - 1,
    where Z' drops the first coordinate, Pi projects R^{L-1} orthogonally on
    the span of the vectors U_i without their last coordinate, and R_L is the
    recurrence of ``lrr_column``.  The extended L x (K_p + M + L - 1) matrix
    is diagonally averaged and its values N_p + 1 .. N_p + M are the
    forecast.  Returns a list of M-vectors, one per series."""
    assert all(c.shape[1] == 1 for c in P.channels) and P.Lset[:, 1].max() == 0, "series problems only"
    L = P.L
    Ug = np.asarray(U, dtype=np.float64)[:, list(group)]
    R = lrr_column(Ug)
    Ub = Ug[:-1, :]                                   # U_i without the last coordinate
    Pi = Ub @ np.linalg.solve(Ub.T @ Ub, Ub.T)        # orthogonal projector on span(Ub)
    out = []
    for c in range(len(P.channels)):
        X = P.block(c)                                # L x K_p trajectory matrix
        Kp = X.shape[1]
        Z = np.zeros((L, Kp + M + L - 1))
        Z[:, :Kp] = Ug @ (Ug.T @ X)
        for j in range(Kp, Kp + M + L - 1):
            y = Z[1:, j - 1]
            Z[:-1, j] = Pi @ y
            Z[-1, j] = R @ y
        # diagonal averaging of the L x Kz matrix: element n collects Z[i, j], i + j = n
        Kz = Z.shape[1]
        acc = np.zeros(L + Kz - 1)
        cnt = np.zeros(L + Kz - 1)
        for i in range(L):
            acc[i:i + Kz] += Z[i]
            cnt[i:i + Kz] += 1
        z = acc / cnt
        Np = len(P.channels[c])
        out.append(z[Np:Np + M])
    return out


def _row_parts(P: Problem, V, group):
    """For the row forecasts: the blocks of V_I per series, S = [mu(V_j)] (the
    last coordinate of every series' block, s x r), V_I with those rows
    removed ((K - s) x r), and R_K = (I_s - S S^T)^-1 S Vbar^T (Sec. 3.3,
    eq. Forec:ContMSSAK)."""
    Vg = np.asarray(V, dtype=np.float64)[:, list(group)]
    s_ = len(P.channels)
    last = [P.offsets[c + 1] - 1 for c in range(s_)]
    keep = np.ones(P.K, bool)
    keep[last] = False
    S = Vg[last, :]
    Vbar = Vg[keep, :]
    RK = np.linalg.solve(np.eye(s_) - S @ S.T, S @ Vbar.T)
    return Vg, S, Vbar, RK, keep


def forecast_recurrent_row(P: Problem, sigma, U, V, group, M: int):
    """M-step recurrent row forecast of an MSSA system (Sec. 3.3, eq.
    Forec:ContMSSAK): every step the next value of each series is R_K Z, Z the
    stacked last K_p - 1 reconstructed values of all series -- a different
    relation per series, the same data for all.  Returns one M-vector per
    series."""
    assert all(c.shape[1] == 1 for c in P.channels) and P.Lset[:, 1].max() == 0, "series problems only"
    _, _, _, RK, _ = _row_parts(P, V, group)
    rec = reconstruct(P, sigma, U, V, [list(group)])[0]
    ys = [list(rec[c][:, 0]) for c in range(len(P.channels))]
    for _ in range(M):
        Z = np.concatenate([ys[c][len(ys[c]) - (P.Ks[c] - 1):] for c in range(len(P.channels))])
        nxt = RK @ Z
        for c in range(len(P.channels)):
            ys[c].append(float(nxt[c]))
    return [np.array(y[len(y) - M:]) for y in ys]


def forecast_vector_row(P: Problem, sigma, U, V, group, M: int):
    """M-step vector row forecast of an MSSA system (Sec. 3.3, eqs. PGrow and
    V_FORrow).  The rows of the reconstructed matrix X^ = X V_I V_I^T are
    continued by A = P(Z): with Z' the row without the first coordinate of
    each series' block, A without the last coordinate of each block is the
    orthogonal projection of Z' on span(Vbar_I), and the last coordinates are
    R_K Z'.  The (L + M + K* - 1) x K matrix of rows is averaged along each
    series' anti-diagonals (the MSSA reconstruction step) and the values
    N_p + 1 .. N_p + M of series p are its forecast."""
    assert all(c.shape[1] == 1 for c in P.channels) and P.Lset[:, 1].max() == 0, "series problems only"
    Vg, S, Vbar, RK, keep = _row_parts(P, V, group)
    Pi = Vbar @ np.linalg.solve(Vbar.T @ Vbar, Vbar.T)      # projector on span(Vbar) in R^(K - s)
    X = P.matrix()
    L = P.L
    s_ = len(P.channels)
    Kstar = max(P.Ks)
    rows = L + M + Kstar - 1
    Z = np.zeros((rows, P.K))
    Z[:L] = (X @ Vg) @ Vg.T
    first = np.ones(P.K, bool)                              # drop the first coordinate of each block
    first[P.offsets[:-1]] = False
    last_idx = [P.offsets[c + 1] - 1 for c in range(s_)]
    for i in range(L, rows):
        zp = Z[i - 1, first]
        Z[i, keep] = Pi @ zp
        Z[i, last_idx] = RK @ zp
    out = []
    for c in range(s_):
        blk = Z[:, P.offsets[c]:P.offsets[c + 1]]           # rows x K_c; element (i, j) is series index i + j
        Kc = blk.shape[1]
        acc = np.zeros(rows + Kc - 1)
        cnt = np.zeros(rows + Kc - 1)
        for j in range(Kc):
            acc[j:j + rows] += blk[:, j]
            cnt[j:j + rows] += 1
        z = acc / cnt
        Np = len(P.channels[c])
        out.append(z[Np:Np + M])
    return out

