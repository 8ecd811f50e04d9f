"""The plan autotuner (ssa_autotune): it times Krylov dimensions and, on 2D
grids, y-pass tiles on a real problem, records the fastest for the problem's
size class, and later decompositions of that class use it -- with the same
results as the oracle.  The plan table is process-wide, so this file uses
size classes no other test shares."""
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


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp64", 1e-9)])
def test_autotune_image_plan_is_used_and_exact(prec, tol):
    x = W.harmonic_image(77, 83, n_harm=2, seed=31, noise=0.2, dtype=np.float64)
    s = pkg.SSA.image(x, 13, 11)
    res = s.autotune(6, prec)
    assert res["n_tried"] >= 2
    assert res["ytk"] >= 1 and 1 <= res["krylov_dim"] <= 112
    assert res["ms_best"] <= res["ms_default"] * 1.0001
    so = O.decompose(O.Problem.image(x, 13, 11), 6)[0]
    np.testing.assert_allclose(s.sigma(), so, rtol=tol, atol=0)
    text = LL.plans_export()
    assert f"kdim p{1 if prec == 'fp64' else 0}.k2.L143." in text and "ytk e" in text
    # a new problem of the same class takes the tuned Krylov dimension
    y = W.harmonic_image(77, 83, n_harm=2, seed=32, noise=0.2, dtype=np.float64)
    t = pkg.SSA.image(y, 13, 11)
    t.decompose(6, prec)
    assert t.info()["krylov_dim"] == res["krylov_dim"]
    np.testing.assert_allclose(t.sigma(), O.decompose(O.Problem.image(y, 13, 11), 6)[0], rtol=tol, atol=0)
    s.close()
    t.close()


def test_plans_round_trip_and_reject_garbage(tmp_path):
    x = W.series_1d(1500, seed=33)
    s = pkg.SSA.series(x, 371)
    s.autotune(5, "fp32")
    path = tmp_path / "plans.txt"
    pkg.save_plans(str(path))
    before = LL.plans_export()
    pkg.load_plans(str(path))
    assert LL.plans_export() == before
    assert "L371." in before
    with pytest.raises(pkg.SSAError):
        LL.plans_import("kdim only-two-fields\n")
    with pytest.raises(pkg.SSAError):
        LL.plans_import("color x.y 3\n")
    s.close()


def test_every_tile_width_gives_the_same_results():
    """Whatever y-pass tile width a plan names (tuned or imported), every launch
    that uses it -- products, spectra, the reconstruction's passes -- must size
    its staging buffers for it, and the results must not depend on it (each
    x-frequency's column transform is computed alone)."""
    x = W.harmonic_image(45, 100, n_harm=2, seed=41, noise=0.1, dtype=np.float64)
    before = set(LL.plans_export().splitlines())
    s = pkg.SSA.image(x, 9, 12)
    s.autotune(4, "fp32")
    s.close()
    new = [ln for ln in LL.plans_export().splitlines() if ln.startswith("ytk ") and ln not in before]
    assert len(new) == 1, new
    key = new[0].split()[1]
    ref = None
    for tk in (1, 2, 4, 8, 16, 32, 64):
        LL.plans_import(f"ytk {key} {tk}\n")
        t = pkg.SSA.image(x, 9, 12)
        t.decompose(4, "fp32", seed=7)
        got = (t.sigma(), t.reconstruct([[0, 1], [2, 3]], residual=True))
        t.close()
        if ref is None:
            ref = got
            continue
        np.testing.assert_allclose(got[0], ref[0], rtol=1e-6, atol=0)
        scale = float(np.nanmax(np.abs(x)))
        for a, b in zip(got[1], ref[1]):
            np.testing.assert_allclose(a, b, rtol=0, atol=1e-5 * scale)
