"""Exact-rank inputs with the rank asked above the signal rank, both forms.

The Lanczos process meets an invariant subspace on these inputs: a series of
finite rank (Sec. 2.2, Appendix A) leaves a residual at the rounding level
once the Krylov space holds its whole column space, and a multiple singular
value (Appendix A.1 Example ex:mssa_ev: equal sigma for a sinusoid with
integer L omega, K omega and for the MSSA pair; four equal values for a 2D
product of cosines) cannot be resolved from one start vector at all.  The
library must still return the r leading triples: the closed-form values, zeros
beyond the rank, orthonormal vectors for the non-zero values and the input
back from the signal components.

Tolerances: |s - s*| <= rtol s* + atol s_1 with rtol as in the parity tests
(1e-5 FP32 form, 1e-9 FP64 form) and atol the noise floor of one product
(5e-6 FP32, 1e-11 FP64: zero singular values come back at that level);
reconstructions 1e-4 / 1e-9 of max|x|.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1309_5050_gb300 as pkg  # noqa: E402
from oracle import ssa_oracle as O  # noqa: E402

RTOL = {"fp32": 1e-5, "fp64": 1e-9}
ATOL = {"fp32": 5e-6, "fp64": 1e-11}
TOL_REC = {"fp32": 1e-4, "fp64": 1e-9}
PRECS = ["fp32", "fp64"]


def sinusoid_pair():
    """A cos(2 pi omega k + phi) with L omega = 4, K omega = 6: sigma_1 =
    sigma_2 = A sqrt(L K) / 2, rank 2."""
    A, omega, L, K = 2.5, 1 / 10, 40, 60
    k = np.arange(L + K - 1)
    x = A * np.cos(2 * np.pi * omega * k + 0.7)
    e = A * math.sqrt(L * K) / 2
    return pkg.SSA.series(x, L), O.Problem.series(x, L), [x], [e, e]


def exponential():
    """exp(0.01 k): rank 1."""
    k = np.arange(120)
    x = np.exp(0.01 * k)
    P = O.Problem.series(x, 50)
    return pkg.SSA.series(x, 50), P, [x], [float(np.linalg.norm(P.matrix(), 2))]


def product_of_cosines():
    """A cos(2 pi wx m + a) cos(2 pi wy n + b) on a 29 x 23 image, window
    10 x 8: four equal values A sqrt(Lx Kx) sqrt(Ly Ky) / 4, 2D rank 4."""
    A, nx, ny, lx, ly = 1.7, 29, 23, 10, 8
    m = np.arange(nx)[:, None]
    n = np.arange(ny)[None, :]
    x = A * np.cos(2 * np.pi * m / 10 + 0.4) * np.cos(2 * np.pi * n / 8 + 1.1)
    e = A * math.sqrt(lx * (nx - lx + 1)) * math.sqrt(ly * (ny - ly + 1)) / 4
    return pkg.SSA.image(x, lx, ly), O.Problem.image(x, lx, ly), [x], [e] * 4


def mssa_pair():
    """(A cos(2 pi k / 8 + 0.2), B cos(2 pi k / 8 + 1.9)), L = 24, K_p = 40:
    sigma_1 = sigma_2 = sqrt((A^2 + B^2) L K_p / 4), MSSA rank 2."""
    A, B, L, Kp = 1.5, 0.8, 24, 40
    k = np.arange(L + Kp - 1)
    xs = [A * np.cos(2 * np.pi * k / 8 + 0.2), B * np.cos(2 * np.pi * k / 8 + 1.9)]
    e = math.sqrt((A * A + B * B) * L * Kp / 4)
    return pkg.SSA.multi(xs, L, dtype=np.float64), O.Problem.multi(xs, L), xs, [e, e]


def damped_pair_series():
    """Two damped / growing harmonics, N = 60, L = 20: rank 4, distinct values
    (the Krylov dimension min(2r + 16, L) = 20 spans the whole window space)."""
    n = np.arange(60, dtype=float)
    x = 1.01 ** n * np.cos(2 * np.pi * n / 9 + 0.2) + 0.5 * 0.99 ** n * np.cos(2 * np.pi * n / 5)
    P = O.Problem.series(x, 20)
    return pkg.SSA.series(x, 20), P, [x], list(np.linalg.svd(P.matrix(), compute_uv=False)[:4])


CASES = [("sinusoid_pair", sinusoid_pair, 4), ("exponential", exponential, 3),
         ("product_of_cosines", product_of_cosines, 7), ("mssa_pair", mssa_pair, 4),
         ("damped_pair_series", damped_pair_series, 6)]


def check_sigma(sig, expect, r, prec):
    want = np.zeros(r)
    want[:len(expect)] = expect
    s1 = max(expect)
    err = np.abs(sig - want)
    assert np.all(err <= RTOL[prec] * want + ATOL[prec] * s1), (sig, want)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name,make,r", CASES, ids=[c[0] for c in CASES])
def test_exact_rank_triples(name, make, r, prec):
    s, P, xs, expect = make()
    rank = len(expect)
    s.decompose(r, prec)
    sig = s.sigma()
    check_sigma(sig, expect, r, prec)
    assert s.info()["converged"] == 1
    U, V = s.vectors()
    Ur, Vr = U[:, :rank], V[:, :rank]
    # The FP32 form returns its vectors in FP32: rounding each entry of unit
    # vectors moves an entry of U^T U by at most 2 * 2^-24 (Cauchy-Schwarz),
    # on top of the 1e-10 cosines its small SVD stops at.  V (the long side,
    # not re-orthogonalised) is stored in FP32 in that form.
    tol_u = 2.0 ** -23 + 1e-9 if prec == "fp32" else 1e-10
    tol_o = 1e-4 if prec == "fp32" else 1e-10
    np.testing.assert_allclose(Ur.T @ Ur, np.eye(rank), atol=tol_u)
    np.testing.assert_allclose(Vr.T @ Vr, np.eye(rank), atol=tol_o)
    for i in range(rank):
        np.testing.assert_allclose(O.matvec(P, Vr[:, i]), sig[i] * Ur[:, i], atol=10 * tol_o * sig[0])
    s.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name,make,r", CASES, ids=[c[0] for c in CASES])
def test_exact_rank_reconstruction(name, make, r, prec):
    """The signal components give the input back (a structured matrix of rank
    below r reconstructs to itself, Sec. 2.1 Step 4); the components past the
    rank give zero; both agree with the oracle's reconstruction."""
    s, P, xs, expect = make()
    rank = len(expect)
    s.decompose(r, prec)
    sig = s.sigma()
    groups = [list(range(rank)), list(range(rank, r))]
    rec = s.reconstruct(groups, residual=True)
    so, Uo, Vo = O.decompose(P, rank)
    ref = O.reconstruct(P, so, Uo, Vo, [list(range(rank))])
    xmax = max(float(np.max(np.abs(x))) for x in xs)
    tol = TOL_REC[prec] * xmax
    for c, x in enumerate(xs):
        sig_c = rec[0][c] if isinstance(rec[0], list) else rec[0]
        sig_c = np.asarray(sig_c).reshape(np.shape(x), order="F")
        assert np.max(np.abs(sig_c - x)) <= tol
        assert np.max(np.abs(sig_c - ref[0][c].reshape(np.shape(x)))) <= tol
        # a component's value is an average of sigma_i U_i V_j^T entries,
        # so the ones past the rank stay below the sum of their values
        rest = rec[1][c] if isinstance(rec[1], list) else rec[1]
        assert np.max(np.abs(rest)) <= tol + float(np.sum(sig[rank:]))
        resid = rec[2][c] if isinstance(rec[2], list) else rec[2]
        assert np.max(np.abs(resid)) <= tol + float(np.sum(sig[rank:]))
    s.close()


def test_fp64_breakdown_path_is_taken():
    """The FP64 form meets its breakdown level on a rank-2 series asked for
    rank 4 (the replacement path runs and is counted) and stays exact."""
    s, P, xs, expect = sinusoid_pair()
    s.decompose(4, "fp64")
    assert s.info()["breakdowns"] >= 1
    check_sigma(s.sigma(), expect, 4, "fp64")
    s.close()


@pytest.mark.parametrize("prec", PRECS)
def test_wide_dynamic_range_is_not_a_breakdown(prec):
    """A steep trend with small noise (x = t + N(0, 0.05^2), N = 4000, L =
    2000): the noise part's Lanczos coefficients sit near 5e-7 sigma_1, far
    below any fixed fraction of sigma_1 one would call rounding, but well above
    the products' own rounding (4 eps log2 M ||x||).  No breakdown may be
    declared there, and the leading values keep the form's accuracy."""
    rng = np.random.default_rng(21)
    t = np.arange(1, 4001, dtype=float)
    x = t + rng.normal(0, 0.05, t.size)
    s = pkg.SSA.series(x, 2000)
    s.decompose(6, prec)
    assert s.info()["breakdowns"] == 0
    so, _, _ = O.decompose(O.Problem.series(x, 2000), 6)
    sig = s.sigma()
    # the two trend values only: at sigma_1 / sigma_3 ~ 1e6 the noise values
    # are resolved to ~eps (sigma_1 / sigma_3)^2 relative by the oracle's
    # S = X X^T route and by a one-sided bidiagonalisation alike
    np.testing.assert_allclose(sig[:2], so[:2], rtol=RTOL[prec], atol=0)
    s.close()
