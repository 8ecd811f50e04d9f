"""GPU parity of the column forecasts (Sec. 3.3): recurrent (eq. Forec:ContMSSAL)
and vector (eqs. PGcolumn, V_FORcolumn).

ssa_forecast reconstructs the component on the device, forms the recurrence
from the window-side vectors and continues every series.  Checked against the
continuation of a finite-rank series and against the oracle on noisy series
and an MSSA system (groups bounded by spectral gaps).

Tolerances: FP64 form 1e-8 of max|x|; FP32 form 2e-4 of max|x|.  The
starting values carry the reconstruction error (FP32 form: bounded by 1e-4
of max|x|, about 1e-6 at these sizes) and the recurrence feeds on itself
over 8-12 steps, so the error grows with the steps.  Measured on a GB300: FP32 2.6e-5, FP64 3.7e-10 of max|x|
at most -- the bounds sit more than seven and twenty times above them.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1309_5050_gb300 as pkg  # noqa: E402
from oracle import ssa_oracle as O  # noqa: E402
from paper_1309_5050_gb300 import _lib as LL  # noqa: E402

TOL = {"fp32": 2e-4, "fp64": 1e-8}


def noisy_series(n, seed):
    rng = np.random.default_rng(seed)
    t = np.arange(n, dtype=float)
    return 0.02 * t + 3 * np.sin(2 * np.pi * t / 11.3) + 1.5 * np.cos(2 * np.pi * t / 4.7 + 0.3) + rng.normal(0, 0.3, n)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_forecast_continues_finite_rank_series(prec):
    """A rank-4 series (two damped / growing harmonics) with 1e-6 noise: the
    forecast of the four leading components continues the noiseless series
    to the noise level."""
    n = np.arange(80, dtype=float)
    f = 1.01 ** n * np.cos(2 * np.pi * n / 9 + 0.2) + 0.5 * 0.99 ** n * np.cos(2 * np.pi * n / 5)
    x = f[:60] + 1e-6 * np.random.default_rng(0).normal(size=60)
    s = pkg.SSA.series(x, 20)
    s.decompose(4, prec)
    fc = s.forecast([0, 1, 2, 3], 20)
    assert np.max(np.abs(fc - f[60:])) <= 1e-5 * np.max(np.abs(f))
    s.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_forecast_matches_oracle(prec):
    x = noisy_series(600, 5)
    s = pkg.SSA.series(x, 200)
    P = O.Problem.series(x, 200)
    s.decompose(6, prec)
    so, Uo, Vo = O.decompose(P, 6)
    # the trend and the two harmonic pairs: ranks 1 + 2 + 2 lead the spectrum
    grp = [0, 1, 2, 3, 4]
    assert so[4] / so[5] > 1.5
    (ref,) = O.forecast_recurrent_column(P, so, Uo, Vo, grp, 12)
    got = s.forecast(grp, 12)
    print(f"forecast {prec}: {np.max(np.abs(got - ref)) / np.max(np.abs(x)):.3e} of max|x|")
    assert np.max(np.abs(got - ref)) <= TOL[prec] * np.max(np.abs(x))
    s.close()
    xs = [noisy_series(n, 20 + i) for i, n in enumerate((300, 350, 280))]
    xs32 = [np.asarray(v, np.float32).astype(np.float64) for v in xs]
    m = pkg.SSA.multi(xs, 100)
    Pm = O.Problem.multi(xs32, 100)
    m.decompose(6, prec)
    so, Uo, Vo = O.decompose(Pm, 6)
    assert so[4] / so[5] > 1.5
    refs = O.forecast_recurrent_column(Pm, so, Uo, Vo, grp, 8)
    gots = m.forecast(grp, 8)
    for g, r_ in zip(gots, refs):
        print(f"forecast {prec}: {np.max(np.abs(g - r_)) / max(np.max(np.abs(v)) for v in xs32):.3e} of max|x|")
        assert np.max(np.abs(g - r_)) <= TOL[prec] * max(np.max(np.abs(v)) for v in xs32)
    m.close()


def test_forecast_errors():
    x = noisy_series(300, 1)
    s = pkg.SSA.series(x, 100)
    with pytest.raises(pkg.SSAError) as e:
        s.forecast([0], 5)
    assert e.value.code == LL.SSA_ESTATE
    s.decompose(4, "fp32")
    with pytest.raises(pkg.SSAError) as e:
        s.forecast([7], 5)
    assert e.value.code == LL.SSA_EINVAL
    s.close()
    img = np.random.default_rng(2).normal(size=(20, 20))
    g = pkg.SSA.image(img, 5, 5)
    g.decompose(3, "fp32")
    with pytest.raises(pkg.SSAError) as e:
        g.forecast([0], 5)
    assert e.value.code == LL.SSA_EINVAL
    g.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_vector_forecast_continues_finite_rank_series(prec):
    """The vector column forecast (eqs. PGcolumn, V_FORcolumn) of a rank-4
    series with 1e-6 noise continues the noiseless series to the noise level."""
    n = np.arange(80, dtype=float)
    f = 1.01 ** n * np.cos(2 * np.pi * n / 9 + 0.2) + 0.5 * 0.99 ** n * np.cos(2 * np.pi * n / 5)
    x = f[:60] + 1e-6 * np.random.default_rng(0).normal(size=60)
    s = pkg.SSA.series(x, 20)
    s.decompose(4, prec)
    fc = s.forecast([0, 1, 2, 3], 20, method="vector")
    assert np.max(np.abs(fc - f[60:])) <= 1e-5 * np.max(np.abs(f))
    s.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_vector_forecast_matches_oracle(prec):
    """ssa_forecast_vector (shift-matrix recursion in the window space's
    coefficients) against the oracle's explicit projector form."""
    grp = [0, 1, 2, 3, 4]
    x = noisy_series(600, 5)
    s = pkg.SSA.series(x, 200)
    P = O.Problem.series(x, 200)
    s.decompose(6, prec)
    so, Uo, Vo = O.decompose(P, 6)
    (ref,) = O.forecast_vector_column(P, so, Uo, Vo, grp, 12)
    got = s.forecast(grp, 12, method="vector")
    print(f"forecast {prec}: {np.max(np.abs(got - ref)) / np.max(np.abs(x)):.3e} of max|x|")
    assert np.max(np.abs(got - ref)) <= TOL[prec] * np.max(np.abs(x))
    s.close()
    xs = [noisy_series(n, 20 + i) for i, n in enumerate((300, 350, 280))]
    xs32 = [np.asarray(v, np.float32).astype(np.float64) for v in xs]
    m = pkg.SSA.multi(xs, 100)
    Pm = O.Problem.multi(xs32, 100)
    m.decompose(6, prec)
    so, Uo, Vo = O.decompose(Pm, 6)
    refs = O.forecast_vector_column(Pm, so, Uo, Vo, grp, 8)
    gots = m.forecast(grp, 8, method="vector")
    for g, r_ in zip(gots, refs):
        print(f"forecast {prec}: {np.max(np.abs(g - r_)) / max(np.max(np.abs(v)) for v in xs32):.3e} of max|x|")
        assert np.max(np.abs(g - r_)) <= TOL[prec] * max(np.max(np.abs(v)) for v in xs32)
    m.close()
    img = np.random.default_rng(2).normal(size=(20, 20))
    im = pkg.SSA.image(img, 5, 5)
    im.decompose(3, "fp32")
    with pytest.raises(pkg.SSAError) as e:
        im.forecast([0], 5, method="vector")
    assert e.value.code == LL.SSA_EINVAL
    im.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("method", ["recurrent_row", "vector_row"])
def test_row_forecasts_match_oracle(method, prec):
    """ssa_forecast_row (eqs. Forec:ContMSSAK, PGrow, V_FORrow) against the
    oracle on an MSSA system of unequal lengths, and the continuation of a
    finite-rank pair (1e-6 noise)."""
    ref_fn = {"recurrent_row": O.forecast_recurrent_row, "vector_row": O.forecast_vector_row}[method]
    grp = [0, 1, 2, 3, 4]
    xs = [noisy_series(n, 20 + i) for i, n in enumerate((300, 350, 280))]
    xs32 = [np.asarray(v, np.float32).astype(np.float64) for v in xs]
    m = pkg.SSA.multi(xs, 100)
    Pm = O.Problem.multi(xs32, 100)
    m.decompose(6, prec)
    so, Uo, Vo = O.decompose(Pm, 6)
    refs = ref_fn(Pm, so, Uo, Vo, grp, 8)
    gots = m.forecast(grp, 8, method=method)
    for g, r_ in zip(gots, refs):
        print(f"forecast {prec}: {np.max(np.abs(g - r_)) / max(np.max(np.abs(v)) for v in xs32):.3e} of max|x|")
        assert np.max(np.abs(g - r_)) <= TOL[prec] * max(np.max(np.abs(v)) for v in xs32)
    m.close()
    n = np.arange(80, dtype=float)
    x1 = np.cos(2 * np.pi * n / 7)
    x2 = 2.0 * np.sin(2 * np.pi * n / 7 + 0.5)
    rng = np.random.default_rng(1)
    a1 = x1[:40] + 1e-6 * rng.normal(size=40)
    a2 = x2[:50] + 1e-6 * rng.normal(size=50)
    pair = pkg.SSA.multi([a1, a2], 12)
    pair.decompose(2, prec)
    f1, f2 = pair.forecast([0, 1], 10, method=method)
    assert np.max(np.abs(f1 - x1[40:50])) <= 1e-4 and np.max(np.abs(f2 - x2[50:60])) <= 1e-4
    pair.close()


def test_fp64_exact_rank_series_decomposition():
    """A noiseless rank-4 series whose Krylov dimension spans the window
    space: the FP64 form meets a breakdown after four steps and must go on
    from a random vector instead of normalising rounding noise."""
    n = np.arange(60, dtype=float)
    f = 1.01 ** n * np.cos(2 * np.pi * n / 9 + 0.2) + 0.5 * 0.99 ** n * np.cos(2 * np.pi * n / 5)
    s = pkg.SSA.series(f, 20)
    s.decompose(4, "fp64")
    so = np.linalg.svd(O.Problem.series(f, 20).matrix(), compute_uv=False)[:4]
    np.testing.assert_allclose(s.sigma(), so, rtol=1e-9, atol=0)
    s.close()
