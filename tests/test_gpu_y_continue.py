"""Continuation of a decomposition to a larger rank (ssa_continue; the
auto-continuation of Sec. 2.4): the previous Ritz triples seed the new Krylov
space.  The continued triples must be those of a fresh decomposition and of
the oracle (same tolerances as the parity tests)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1309_5050_gb300 as pkg  # noqa: E402
from oracle import ssa_oracle as O  # noqa: E402
from paper_1309_5050_gb300 import _lib as LL  # noqa: E402

TOL_SIG = {"fp32": 1e-5, "fp64": 1e-9}


def noisy_series(n, seed):
    rng = np.random.default_rng(seed)
    t = np.arange(n, dtype=float)
    return 0.02 * t + 3 * np.sin(2 * np.pi * t / 11.3) + 1.5 * np.cos(2 * np.pi * t / 4.7 + 0.3) + rng.normal(0, 0.3, n)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_continued_triples_equal_a_fresh_decomposition(prec):
    x = noisy_series(700, 3)
    s = pkg.SSA.series(x, 250)
    s.decompose(4, prec)
    s.extend(9, prec)
    assert s.info()["rank"] == 9
    so, Uo, Vo = O.decompose(O.Problem.series(x, 250), 9)
    np.testing.assert_allclose(s.sigma(), so, rtol=TOL_SIG[prec], atol=0)
    # the continued vectors satisfy the SVD relations of the explicit matrix
    U, V = s.vectors()
    X = O.Problem.series(x, 250).matrix()
    for i in range(5):                       # the leading, gap-separated ones
        assert np.max(np.abs(X @ V[:, i] - so[i] * U[:, i])) <= 1e-4 * so[0]
    rec = s.reconstruct([[0], [1, 2]])
    ref = O.reconstruct(O.Problem.series(x, 250), so, Uo, Vo, [[0], [1, 2]])
    assert np.max(np.abs(rec[0] - ref[0][0][:, 0])) <= 1e-4 * np.max(np.abs(x))
    s.close()
    xs = [noisy_series(n, 30 + i) for i, n in enumerate((300, 350, 280))]
    xs32 = [np.asarray(v, np.float32).astype(np.float64) for v in xs]
    m = pkg.SSA.multi(xs, 100)
    m.decompose(3, prec)
    m.extend(7, prec)
    so, _, _ = O.decompose(O.Problem.multi(xs32, 100), 7)
    np.testing.assert_allclose(m.sigma(), so, rtol=TOL_SIG[prec], atol=0)
    m.close()


def test_continue_errors():
    x = noisy_series(400, 4)
    s = pkg.SSA.series(x, 150)
    with pytest.raises(pkg.SSAError) as e:
        s.extend(5)
    assert e.value.code == LL.SSA_ESTATE
    s.decompose(5, "fp32")
    with pytest.raises(pkg.SSAError) as e:
        s.extend(5)
    assert e.value.code == LL.SSA_ERANK
    s.close()


def test_continue_rank_rule_holds_on_the_fresh_run_fallback():
    """A previous run in the other precision form is redone from a new start
    vector; the rank must still grow (equal or lower rank: SSA_ERANK), and a
    valid larger rank gives the oracle's triples."""
    x = noisy_series(500, 6)
    s = pkg.SSA.series(x, 180)
    s.decompose(5, "fp32")
    for r in (5, 3):
        with pytest.raises(pkg.SSAError) as e:
            s.extend(r, "fp64")
        assert e.value.code == LL.SSA_ERANK
    s.extend(8, "fp64")
    so, _, _ = O.decompose(O.Problem.series(x, 180), 8)
    np.testing.assert_allclose(s.sigma(), so, rtol=TOL_SIG["fp64"], atol=0)
    s.close()
