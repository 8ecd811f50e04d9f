"""The allocation-free series product against the oracle and the regular one.

ssa_matvec_series_noalloc serves callers that cannot allocate device memory
when they call (captured graph regions, fixed-budget or plug-in hosts); it
keeps its intermediates in one fixed device array that every call reuses.  So
each call must give what the explicit trajectory-matrix product of the oracle
gives, and what ssa_matvec gives, even when the previous call left another
series' spectrum of another size in that array.  This file is collected last
so a failure here leaves every other test already run.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1309_5050_gb300 as pkg  # noqa: E402
from oracle import ssa_oracle as O  # noqa: E402
from paper_1309_5050_gb300 import _lib  # noqa: E402

TOL_MV = 5e-6   # FP32 FFT product: |u - u*|_inf <= TOL ||x||_2 ||v||_2 (as in the parity tests)


def series(n, seed):
    rng = np.random.default_rng(seed)
    t = np.arange(n)
    return (0.01 * t + np.sin(2 * np.pi * t / 12.5) + rng.normal(0, 0.2, n)).astype(np.float32)


class Case:
    """One series on the device with its oracle problem and regular context."""

    def __init__(self, n, L, seed):
        self.x = series(n, seed)
        self.n, self.L, self.K = n, L, n - L + 1
        self.xd = torch.from_numpy(self.x).cuda()
        x64 = self.x.astype(np.float64)
        self.P = O.Problem.series(x64, L)
        self.ref = pkg.SSA.series(x64, L)
        self.xn = float(np.linalg.norm(x64))

    def check(self, transpose, rng, tag):
        nin, nout = (self.L, self.K) if transpose else (self.K, self.L)
        v = rng.normal(size=nin).astype(np.float32).astype(np.float64)
        vd = torch.from_numpy(v.astype(np.float32)).cuda()
        out = torch.full((nout,), float("nan"), dtype=torch.float32, device="cuda")
        _lib.matvec_series_noalloc(self.xd, self.L, vd, out, transpose)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        bound = TOL_MV * self.xn * np.linalg.norm(v)
        want = O.rmatvec(self.P, v) if transpose else O.matvec(self.P, v)
        err_oracle = np.max(np.abs(got - want))
        assert err_oracle <= bound, (tag, transpose, err_oracle, bound)
        regular = self.ref.matvec(v, transpose, "fp32")
        err_regular = np.max(np.abs(got - regular))
        assert err_regular <= bound, (tag, transpose, err_regular, bound)

    def close(self):
        self.ref.close()


@pytest.mark.parametrize("sizes", [((1000, 500), (4097, 1500)), ((16384, 7000), (300, 41))],
                         ids=["1000_then_4097", "16384_then_300"])
def test_noalloc_alternating_series_match_oracle_and_regular_product(sizes):
    """Two series of different lengths take turns, two rounds, both
    directions: every call overwrites the shared spectrum and grid size."""
    a, b = Case(*sizes[0], seed=11), Case(*sizes[1], seed=12)
    rng = np.random.default_rng(1)
    for rnd in range(2):
        for transpose in (False, True):
            a.check(transpose, rng, f"a round {rnd}")
            b.check(transpose, rng, f"b round {rnd}")
    a.close()
    b.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    x = torch.zeros(16385, dtype=torch.float32, device="cuda")
    v = torch.zeros(16385, dtype=torch.float32, device="cuda")
    with pytest.raises(RuntimeError, match="scratch limit"):
        _lib.matvec_series_noalloc(x, 100, v, v, False)
    out = torch.full((16385,), 7.0, dtype=torch.float32, device="cuda")
    with pytest.raises(RuntimeError, match="1 < L < n"):
        _lib.matvec_series_noalloc(x[:10], 10, v, out, False)
    torch.cuda.synchronize()
    assert bool(torch.all(out == 7.0)), "a rejected call wrote its output"
