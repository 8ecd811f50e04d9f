"""GPU parity of the w-correlations (Sec. 2.2, paragraph Separability).

ssa_wcor reconstructs the components on the device and sums the weighted
Gram matrix there; these tests compare it with the oracle's definition on
groups whose boundaries sit in spectral gaps (a group that splits a cluster
of near-equal singular values has no unique answer), and with the closed
form of two exactly separable harmonics.

Tolerances: FP64 form 1e-11 on rho and relative on the contributions; FP32
form 1e-5.  rho and the contributions are ratios of weighted inner products
of the components, so the components' relative error (FP32 form: a few
FP32 roundings per product and per diagonal average, about 1e-6 of their
norms at these sizes) enters once, not amplified.  Measured on a GB300: FP32
rho 2.9e-8, contributions 7.9e-7; FP64 rho 1.4e-14, contributions 1.8e-14
-- the bounds sit more than ten times above them.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1309_5050_gb300 as pkg  # noqa: E402
import workloads as W  # noqa: E402
from oracle import ssa_oracle as O  # noqa: E402
from paper_1309_5050_gb300 import _lib as LL  # noqa: E402

TOL = {"fp32": 1e-5, "fp64": 1e-11}


def gap_groups(sig, min_gap=1.1):
    groups, cur = [], [0]
    for i in range(1, len(sig)):
        if sig[i - 1] / sig[i] >= min_gap:
            groups.append(cur)
            cur = []
        cur.append(i)
    return groups


def noisy_series(n, seed):
    rng = np.random.default_rng(seed)
    t = np.arange(n, dtype=float)
    return 0.02 * t + 3 * np.sin(2 * np.pi * t / 11.3) + 1.5 * np.cos(2 * np.pi * t / 4.7 + 0.3) + rng.normal(0, 0.3, n)


def cases():
    x = noisy_series(700, 1)
    yield "1d_700_250", pkg.SSA.series(x, 250), O.Problem.series(x, 250)
    xs = [noisy_series(n, 10 + i) for i, n in enumerate((300, 411, 377))]
    xs32 = [np.asarray(v, np.float32).astype(np.float64) for v in xs]
    yield "mssa_3x", pkg.SSA.multi(xs, 90), O.Problem.multi(xs32, 90)
    img = W.harmonic_image(40, 36, n_harm=2, seed=4, noise=0.2, trend=True, dtype=np.float64)
    mask = np.ones(img.shape, bool)
    mask[10:14, 20:25] = False
    wm = pkg.window_circle(4)
    yield "shaped_40x36_circle4", pkg.SSA.image(img, 9, 9, wmask=wm, mask=mask), O.Problem.image(img, 9, 9, wmask=wm, mask=mask)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_wcor_matches_oracle(prec):
    for name, s, P in cases():
        r = 8
        so, Uo, Vo = O.decompose(P, r + 1)
        s.decompose(r, prec)
        groups = [g for g in gap_groups(so[:r + 1]) if max(g) < r]
        assert len(groups) >= 2, name
        rho, contrib = s.wcor(groups)
        rho_o, contrib_o = O.wcor(P, so, Uo, Vo, groups)
        print(f"wcor {name} {prec}: rho {np.max(np.abs(rho - rho_o)):.3e}, "
              f"contributions {np.max(np.abs(contrib - contrib_o) / np.abs(contrib_o)):.3e}")
        assert np.max(np.abs(rho - rho_o)) <= TOL[prec], (name, rho, rho_o)
        np.testing.assert_allclose(contrib, contrib_o, rtol=TOL[prec], atol=0, err_msg=name)
        np.testing.assert_array_equal(rho, rho.T)
        s.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_wcor_separable_harmonics_closed_form(prec):
    L, K = 16, 32
    n = np.arange(L + K - 1, dtype=float)
    x1 = 2.0 * np.cos(2 * np.pi * n / 8 + 0.4)
    x2 = np.cos(2 * np.pi * n / 4 + 0.3)
    s = pkg.SSA.series(x1 + x2, L)
    s.decompose(4, prec)
    rho, contrib = s.wcor([[0, 1], [2, 3]])
    w = np.minimum.reduce([n + 1, np.full_like(n, L), np.full_like(n, K), len(n) - n])
    xx = np.sum(w * (x1 + x2) ** 2)
    tol = 1e-5 if prec == "fp32" else 1e-10
    assert abs(rho[0, 1]) <= tol and rho[0, 0] == 1.0 and rho[1, 1] == 1.0
    np.testing.assert_allclose(contrib, [np.sum(w * x1 ** 2) / xx, np.sum(w * x2 ** 2) / xx], rtol=tol)
    s.close()


def test_wcor_elementary_default_and_errors():
    x = noisy_series(500, 3)
    s = pkg.SSA.series(x, 200)
    with pytest.raises(pkg.SSAError) as e:
        s.wcor([[0]])
    assert e.value.code == LL.SSA_ESTATE
    s.decompose(6, "fp32")
    rho, contrib = s.wcor()
    assert rho.shape == (6, 6) and contrib.shape == (6,)
    np.testing.assert_array_equal(np.diag(rho), 1.0)
    assert np.all(np.abs(rho) <= 1.0 + 1e-12) and np.all(contrib > 0) and contrib.sum() <= 1.0 + 1e-9
    with pytest.raises(pkg.SSAError) as e:
        s.wcor([])
    assert e.value.code == LL.SSA_EINVAL
    s.close()
