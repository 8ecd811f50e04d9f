"""Planted mistakes: the oracle's pins catch plausible slips.

Each case replaces one oracle function by a copy with one deliberate mistake
(on the CPU, for the duration of the case) and runs a few pins from
test_oracle_pins.py; at least one of them must fail.  This shows that the pins
constrain the oracle beyond restating its own formulas.
"""
import contextlib

import numpy as np
import pytest

from oracle import ssa_oracle as O
from tests import test_oracle_pins as pins


@contextlib.contextmanager
def planted(name, fn):
    keep = getattr(O, name)
    setattr(O, name, fn)
    try:
        yield
    finally:
        setattr(O, name, keep)


def fails(*tests):
    """True when at least one of the pins raises (fails) under the plant."""
    for t in tests:
        try:
            t()
        except Exception:
            return True
    return False


# ---------------------------------------------------------------- the plants
def traj_transposed(x, Lset, Kset, cols=None):
    """X_ij = x[l_j + k_i]: window and origin roles swapped."""
    if cols is None:
        cols = np.arange(len(Kset))
    n = min(len(Lset), len(cols))
    px = Lset[:n, 0][None, :] + Kset[cols[:n], 0][:, None]
    py = Lset[:n, 1][None, :] + Kset[cols[:n], 1][:, None]
    out = np.zeros((len(Lset), len(cols)))
    out[:n, :n] = np.asarray(x, dtype=np.float64)[px, py]
    return out


def traj_off_by_one(x, Lset, Kset, cols=None):
    """X_ij = x[l_i + k_j + 1] (the paper's 1-based shift kept)."""
    if cols is None:
        cols = np.arange(len(Kset))
    px = Lset[:, 0][:, None] + Kset[cols, 0][None, :]
    py = Lset[:, 1][:, None] + Kset[cols, 1][None, :]
    xx = np.asarray(x, dtype=np.float64)
    return xx[np.minimum(px + 1, xx.shape[0] - 1), py]


def origins_short(obs, Lset):
    """The last admissible origin dropped (range nx - ex instead of nx - ex + 1)."""
    K = O.__dict__["_planted_origin_keep"](obs, Lset)
    nx = obs.shape[0]
    ex = int(Lset[:, 0].max()) + 1
    return K[K[:, 0] < nx - ex]


def window_row_major(lx, ly=1, wmask=None):
    """Window listed row by row (l_x outer) instead of column-major."""
    if wmask is None:
        wmask = np.ones((lx, ly), dtype=bool)
    out = [(a, b) for a in range(lx) for b in range(ly) if wmask[a, b]]
    return np.array(out, dtype=np.int64).reshape(-1, 2)


def weights_one_short(shape, Lset, Kset):
    """Counts that skip the last window element."""
    return O.__dict__["_planted_weights_keep"](shape, Lset[:-1], Kset)


def svd_eigen_no_sqrt(P, r=None):
    """sigma = lambda instead of sqrt(lambda)."""
    s, U, V = O.__dict__["_planted_eigen_keep"](P, r)
    return s ** 2, U, V * s[None, :]


def svd_eigen_doubled_block(P, r=None):
    """The first column block of S = X X^T added twice."""
    S = np.zeros((P.L, P.L))
    first = True
    for _, Xb in P.column_blocks(width=16):
        S += (2.0 if first else 1.0) * (Xb @ Xb.T)
        first = False
    lam, U = np.linalg.eigh(S)
    o = np.argsort(lam)[::-1]
    lam, U = lam[o], U[:, o]
    r = r or P.L
    r = min(r, int(np.sum(lam > lam[0] * 1e-28)))
    sig = np.sqrt(lam[:r])
    V = O.rmatvec_block(P, U[:, :r]) / sig[None, :] if hasattr(O, "rmatvec_block") else \
        np.column_stack([O.rmatvec(P, U[:, i]) for i in range(r)]) / sig[None, :]
    return sig, U[:, :r], V


def jacobi_wrong_sign(X, tol=1e-15, max_sweeps=80):
    """One-sided Jacobi whose rotation has the sine's sign flipped."""
    A = np.asarray(X, dtype=np.float64)
    transpose = A.shape[1] > A.shape[0]
    A = (A.T if transpose else A).copy()
    m, n = A.shape
    R = np.eye(n)
    for _ in range(max_sweeps):
        for p in range(n - 1):
            for q in range(p + 1, n):
                a, b = A[:, p], A[:, q]
                al, be, ga = a @ a, b @ b, a @ b
                if abs(ga) <= tol * np.sqrt(al * be):
                    continue
                z = (be - al) / (2 * ga)
                t = np.sign(z) / (abs(z) + np.sqrt(1 + z * z)) if z != 0 else 1.0
                c = 1 / np.sqrt(1 + t * t)
                s = -c * t
                A[:, p], A[:, q] = c * a - s * b, s * a + c * b
                R[:, p], R[:, q] = c * R[:, p] - s * R[:, q], s * R[:, p] + c * R[:, q]
    sig = np.linalg.norm(A, axis=0)
    o = np.argsort(sig)[::-1]
    sig = sig[o]
    W = A[:, o] / np.where(sig > 0, sig, 1)[None, :]
    return (sig, R[:, o], W) if transpose else (sig, W, R[:, o])


def reconstruct_wrong_divisor(P, sigma, U, V, groups, residual=False):
    """Diagonal averaging divided by the window length instead of |A_k|."""
    out = O.__dict__["_planted_rec_keep"](P, sigma, U, V, groups, residual=False)
    for g in out:
        for c, rec in enumerate(g):
            w = P.weights(c)
            ok = w > 0
            rec[ok] = rec[ok] * w[ok] / P.L
    if residual:
        res = []
        for c, x in enumerate(P.channels):
            r_ = x.copy()
            for g in out:
                r_ = r_ - g[c]
            res.append(r_)
        out.append(res)
    return out


CASES = [
    ("trajectory_columns", traj_transposed, None,
     [pins.test_hankel_embedding_printed_form, pins.test_matvec_brute_force]),
    ("trajectory_columns", traj_off_by_one, None,
     [pins.test_hankel_embedding_printed_form, pins.test_2d_trajectory_is_hankel_block_hankel]),
    ("origin_set", origins_short, "_planted_origin_keep",
     [pins.test_origin_set_brute_force_with_holes, pins.test_mars_trajectory_sizes]),
    ("window_set", window_row_major, None,
     [pins.test_2d_trajectory_is_hankel_block_hankel, pins.test_2d_with_ly_1_equals_mssa]),
    ("weights", weights_one_short, "_planted_weights_keep",
     [pins.test_weights_1d_closed_form, pins.test_weights_count_trajectory_entries]),
    ("svd_eigen", svd_eigen_no_sqrt, "_planted_eigen_keep",
     [pins.test_closed_form_sinusoid_singular_values, pins.test_eigen_route_matches_jacobi_route]),
    ("svd_eigen", svd_eigen_doubled_block, None,
     [pins.test_eigen_route_matches_jacobi_route, pins.test_closed_form_mssa_pair]),
    ("svd_jacobi", jacobi_wrong_sign, None,
     [pins.test_jacobi_matches_lapack, pins.test_closed_form_sinusoid_singular_values]),
    ("reconstruct", reconstruct_wrong_divisor, "_planted_rec_keep",
     [pins.test_sum_of_elementary_components_is_input, pins.test_reconstruction_brute_force_antidiagonals]),
]


@pytest.mark.parametrize("name,fn,keep,tests", CASES,
                         ids=[f"{c[0]}:{c[1].__name__}" for c in CASES])
def test_planted_mistake_fails_a_pin(name, fn, keep, tests):
    assert not fails(*tests), "the pins must pass on the unplanted oracle"
    if keep:
        setattr(O, keep, getattr(O, name))
    try:
        with planted(name, fn):
            assert fails(*tests), f"planted mistake in {name} ({fn.__name__}) passed every pin"
    finally:
        if keep:
            delattr(O, keep)
