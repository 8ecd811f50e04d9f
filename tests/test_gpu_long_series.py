"""GPU parity for series longer than the single-CTA FFT grid (segment form).

Series above 16384 samples run as the Hankel-block-Hankel matrix of a segment
image (block length 4096) on a 2D grid.  These tests compare that path with
the CPU oracle: products and decompositions element by element at sizes the
oracle handles in seconds (several segments, ragged last blocks, both
orientations, MSSA systems), and at the longest serving size (N = 200000,
L = 100000) through sampled rows, columns and reconstructed elements that the
oracle computes one at a time.

Tolerances as in the other parity tests: sigma 1e-5 / 1e-9 relative
(FP32 / FP64 form), reconstructions 1e-4 / 1e-9 of max|x|, one product
5e-6 / 1e-13 of ||x|| ||v||.
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

TOL_SIG = {"fp32": 1e-5, "fp64": 1e-9}
TOL_REC = {"fp32": 1e-4, "fp64": 1e-9}
TOL_MV = {"fp32": 5e-6, "fp64": 1e-13}


def noisy_series(n, seed):
    rng = np.random.default_rng(seed)
    t = np.arange(n, dtype=float)
    return (0.0005 * t + 3 * np.sin(2 * np.pi * t / 113.3) + 1.5 * np.cos(2 * np.pi * t / 37.7 + 0.3)
            + rng.normal(0, 0.3, n))


def gap_groups(sig, min_gap=1.1):
    groups, cur = [], [0]
    for i in range(1, len(sig)):
        if sig[i - 1] / sig[i] >= min_gap:
            groups.append(cur)
            cur = []
        cur.append(i)
    return groups


MV_CASES = [
    ("1d_16385_4097", [16385], 4097),       # just past the limit: 1-sample tails in both blocks
    ("1d_30000_1500", [30000], 1500),
    ("1d_20000_17000", [20000], 17000),     # L > K
    ("mssa_20000_17500_9000", [20000, 17500, 9000], 1000),
]


def build(lengths, L, seed):
    xs = [noisy_series(n, seed + i) for i, n in enumerate(lengths)]
    if len(xs) == 1:
        return pkg.SSA.series(xs[0], L), O.Problem.series(xs[0], L), xs
    xs32 = [np.asarray(v, np.float32).astype(np.float64) for v in xs]
    return pkg.SSA.multi(xs, L), O.Problem.multi(xs32, L), xs32


@pytest.mark.parametrize("name,lengths,L", MV_CASES, ids=[c[0] for c in MV_CASES])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_long_matvec(name, lengths, L, prec):
    g, P, xs = build(lengths, L, 11)
    inf = g.info()
    assert inf["fft_mx"] == 8192 and inf["fft_my"] > 1      # segment form
    assert (inf["L"], inf["K"]) == (P.L, P.K)
    rng = np.random.default_rng(7)
    xn = np.sqrt(sum(float(np.sum(np.asarray(x) ** 2)) for x in xs))
    v = rng.normal(size=P.K)
    u = g.matvec(v, transpose=False, prec=prec)
    ref = O.matvec(P, v)
    assert np.max(np.abs(u - ref)) <= TOL_MV[prec] * xn * np.linalg.norm(v)
    w = rng.normal(size=P.L)
    vt = g.matvec(w, transpose=True, prec=prec)
    ref_t = O.rmatvec(P, w)
    assert np.max(np.abs(vt - ref_t)) <= TOL_MV[prec] * xn * np.linalg.norm(w)
    g.close()


DEC_CASES = [
    ("1d_30000_1500_fp32", [30000], 1500, 8, "fp32"),
    ("1d_30000_1500_fp64", [30000], 1500, 8, "fp64"),
    ("1d_20000_17000_fp32", [20000], 17000, 6, "fp32"),
    ("mssa_20000_17500_9000_fp32", [20000, 17500, 9000], 1000, 6, "fp32"),
]


@pytest.mark.parametrize("name,lengths,L,r,prec", DEC_CASES, ids=[c[0] for c in DEC_CASES])
def test_long_decompose_and_reconstruct(name, lengths, L, r, prec):
    g, P, xs = build(lengths, L, 21)
    g.decompose(r, prec=prec, seed=3)
    sig = g.sigma()
    # Step 2 on the short side: S = X X^T when L <= K, else S' = X^T X
    s_ref, U, V = O.decompose(P, r, "eigen" if P.L <= P.K else "eigen_t")
    np.testing.assert_allclose(sig, s_ref, rtol=TOL_SIG[prec], atol=0)
    groups = gap_groups(s_ref)[:3]
    assert groups, "no spectral gap to test reconstruction on"
    got = g.reconstruct(groups, residual=True)
    ref = O.reconstruct(P, s_ref, U, V, groups, residual=True)
    scale = max(float(np.nanmax(np.abs(x))) for x in xs)
    for gi in range(len(groups) + 1):
        gg = got[gi] if isinstance(got[gi], list) else [got[gi]]
        for c, rc in enumerate(ref[gi]):
            rc = rc[:, 0]
            ok = ~np.isnan(rc)
            assert np.array_equal(ok, ~np.isnan(gg[c]))
            assert np.max(np.abs(gg[c][ok] - rc[ok])) <= TOL_REC[prec] * scale, (gi, c)
    g.close()


def test_longest_serving_size_sampled():
    """N = 200000, L = 100000: the products, the singular triples and the
    reconstruction checked on sampled rows, columns and elements."""
    n, L, r = 200000, 100000, 10
    x = noisy_series(n, 99)
    K = n - L + 1
    g = pkg.SSA.series(x, L)
    rng = np.random.default_rng(1)
    rows = np.sort(rng.choice(L, 48, replace=False))
    cols = np.sort(rng.choice(K, 48, replace=False))
    xn = float(np.linalg.norm(x))
    # one product each way, sampled
    v = rng.normal(size=K)
    u = g.matvec(v, prec="fp32")
    assert np.max(np.abs(u[rows] - O.series_rows(x, L, rows, v))) <= TOL_MV["fp32"] * xn * np.linalg.norm(v)
    w = rng.normal(size=L)
    vt = g.matvec(w, transpose=True, prec="fp32")
    assert np.max(np.abs(vt[cols] - O.series_cols(x, L, cols, w))) <= TOL_MV["fp32"] * xn * np.linalg.norm(w)
    # singular triples: X V_i = sigma_i U_i and X^T U_i = sigma_i V_i on the samples
    g.decompose(r, prec="fp32", seed=5)
    sig = g.sigma()
    U, V = g.vectors()
    for i in range(r):
        res_r = O.series_rows(x, L, rows, V[:, i]) - sig[i] * U[rows, i]
        res_c = O.series_cols(x, L, cols, U[:, i]) - sig[i] * V[cols, i]
        assert np.max(np.abs(res_r)) <= 1e-5 * sig[0], i
        assert np.max(np.abs(res_c)) <= 1e-5 * sig[0], i
    # the FP64 form finds the same leading values
    g64 = pkg.SSA.series(x, L)
    g64.decompose(r, prec="fp64", seed=5)
    np.testing.assert_allclose(sig, g64.sigma(), rtol=TOL_SIG["fp32"], atol=0)
    g64.close()
    # reconstruction of the leading groups at sampled elements, from the
    # decomposition's own triples
    groups = gap_groups(sig)[:3]
    got = g.reconstruct(groups)
    pts = np.concatenate([[0, 1, n - 1, n - 2, L - 1, L, K - 1, K], rng.choice(n, 40, replace=False)])
    scale = float(np.max(np.abs(x)))
    for gi, grp in enumerate(groups):
        ref = O.series_hankelize_at(sig, U, V, grp, pts)
        assert np.max(np.abs(got[gi][pts] - ref)) <= TOL_REC["fp32"] * scale, gi
    g.close()


def test_long_series_with_missing_values_is_refused():
    x = noisy_series(20000, 5)
    x[1234] = np.nan
    with pytest.raises(pkg.SSAError) as e:
        pkg.SSA.series(x, 5000)
    assert e.value.code == LL.SSA_EUNSUPPORTED


def test_long_and_short_series_share_a_batch():
    """A batch (and a server) may hold series of both forms; each result is
    the one it gets alone."""
    xa, xb = noisy_series(24000, 1), noisy_series(3000, 2)
    alone = []
    for x, L in ((xa, 2000), (xb, 1000)):
        s = pkg.SSA.series(x, L)
        s.decompose(6, seed=9)
        alone.append((s.sigma(), s.reconstruct([[0], [1, 2]])))
        s.close()
    srv = pkg.Server()
    ta = srv.submit_series(xa, 2000, 6, groups=[[0], [1, 2]], seed=9)
    tb = srv.submit_series(xb, 1000, 6, groups=[[0], [1, 2]], seed=9)
    srv.drain()
    for t, (s_ref, rec_ref) in zip((ta, tb), alone):
        r = srv.take(t)
        assert r["status"] == 0
        np.testing.assert_allclose(r["sigma"], s_ref, rtol=1e-6, atol=0)
        for a, b in zip(r["outputs"], rec_ref):
            assert np.max(np.abs(a - b)) <= 1e-5 * float(np.max(np.abs(b)))
    srv.close()
