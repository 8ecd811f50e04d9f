"""The allocation-free series product against the regular one.

ssa_matvec_series_noalloc serves callers that cannot allocate device memory
when they call (captured graph regions, fixed-budget or plug-in hosts); it
keeps its intermediates in a fixed device array.  It must give what
ssa_matvec gives, call after call, since every call reuses that array.  This
file is collected last so a failure here leaves every other test already run.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1309_5050_gb300 as pkg  # noqa: E402
from paper_1309_5050_gb300 import _lib  # noqa: E402

TOL_MV = 5e-6   # FP32 FFT product: |u - u*|_inf <= TOL ||x||_2 ||v||_2 (as in the parity tests)


def series(n, seed):
    rng = np.random.default_rng(seed)
    t = np.arange(n)
    return (0.01 * t + np.sin(2 * np.pi * t / 12.5) + rng.normal(0, 0.2, n)).astype(np.float32)


@pytest.mark.parametrize("n,L", [(1000, 500), (4097, 1500), (16384, 7000)])
def test_noalloc_matches_regular_product_twice(n, L):
    x = series(n, n)
    K = n - L + 1
    ref = pkg.SSA.series(x.astype(np.float64), L)
    xd = torch.from_numpy(x).cuda()
    rng = np.random.default_rng(1)
    xn = float(np.linalg.norm(x.astype(np.float64)))
    for call in range(2):                          # two calls in a row share the scratch array
        for transpose in (False, True):
            nin, nout = (L, K) if transpose else (K, L)
            v = rng.normal(size=nin)
            vd = torch.from_numpy(v.astype(np.float32)).cuda()
            out = torch.full((nout,), float("nan"), dtype=torch.float32, device="cuda")
            _lib.matvec_series_noalloc(xd, L, vd, out, transpose)
            torch.cuda.synchronize()
            got = out.cpu().numpy().astype(np.float64)
            want = ref.matvec(v.astype(np.float32).astype(np.float64), transpose, "fp32")
            err = np.max(np.abs(got - want))
            assert err <= TOL_MV * xn * np.linalg.norm(v), (call, transpose, err)
    ref.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    x = torch.zeros(16385, dtype=torch.float32, device="cuda")
    v = torch.zeros(16385, dtype=torch.float32, device="cuda")
    with pytest.raises(RuntimeError, match="scratch limit"):
        _lib.matvec_series_noalloc(x, 100, v, v, False)
    assert math.isfinite(0.0)
