"""GPU parity: the CUDA path through the C ABI against the CPU FP64 oracle.

Tolerances (FP32-FFT form / FP64 form):
  * singular values: |s - s*| <= 1e-5 s* / 1e-10 s* (per value);
  * reconstructions: max |x~ - x~*| <= 1e-4 max|x| / 1e-9 max|x| over N',
    for groups whose boundaries sit in spectral gaps (a group that splits a
    cluster of near-equal singular values has no unique answer);
  * one FFT product: |u - u*|_inf <= 5e-6 ||x||_2 ||v||_2 / 1e-13 ||x||_2 ||v||_2
    (FP32 FFT convolution error grows like eps log2(M) ||x|| ||v||, M <= 2^14);
  * shapes and weights: bit-exact (integers).
"""
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1309_5050_gb300 as pkg  # noqa: E402
import workloads as W  # noqa: E402
from oracle import ssa_oracle as O  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TOL_SIG = {"fp32": 1e-5, "fp64": 1e-9}
TOL_REC = {"fp32": 1e-4, "fp64": 1e-9}
TOL_MV = {"fp32": 5e-6, "fp64": 1e-13}


def gap_groups(sig, min_gap=1.1):
    """Split 0..len-1 at the boundaries where sigma drops by >= min_gap."""
    groups, cur = [], [0]
    for i in range(1, len(sig)):
        if sig[i - 1] / sig[i] >= min_gap:
            groups.append(cur)
            cur = []
        cur.append(i)
    return groups  # the last (open) cluster is left out: its end is not a gap


def noisy_series(n, seed):
    rng = np.random.default_rng(seed)
    t = np.arange(n, dtype=float)
    return (0.02 * t + 3 * np.sin(2 * np.pi * t / 11.3) + 1.5 * np.cos(2 * np.pi * t / 4.7 + 0.3)
            + rng.normal(0, 0.3, n))


def noisy_image(nx, ny, seed):
    return W.harmonic_image(nx, ny, n_harm=2, seed=seed, noise=0.2, trend=True, dtype=np.float64)


# ------------------------------------------------------------------ cases
def case_1d(n, L, seed):
    x = noisy_series(n, seed)
    return pkg.SSA.series(x, L), O.Problem.series(x, L), x


def case_1d_gaps(n, L, seed, gaps):
    """A series with missing stretches: the origin set has holes (bit-mapped)."""
    x = noisy_series(n, seed)
    for a, b in gaps:
        x[a:b] = np.nan
    return pkg.SSA.series(x, L), O.Problem.series(x, L), x


def case_mssa_gaps(lengths, L, seed):
    xs = [noisy_series(n, seed + i) for i, n in enumerate(lengths)]
    xs[1][7:9] = np.nan
    xs32 = [np.asarray(v, np.float32).astype(np.float64) for v in xs]
    return pkg.SSA.multi(xs, L), O.Problem.multi(xs32, L), xs32


def case_mssa(lengths, L, seed):
    xs = [noisy_series(n, seed + i) for i, n in enumerate(lengths)]
    xs32 = [np.asarray(v, np.float32).astype(np.float64) for v in xs]
    return pkg.SSA.multi(xs, L), O.Problem.multi(xs32, L), xs32


def case_2d(nx, ny, lx, ly, seed, wmask=None, holes=False):
    x = noisy_image(nx, ny, seed)
    mask = None
    if holes:
        rng = np.random.default_rng(seed)
        mask = np.ones((nx, ny), bool)
        for _ in range(3):
            cx, cy = rng.integers(0, nx), rng.integers(0, ny)
            mask[max(0, cx - 2):cx + 2, max(0, cy - 3):cy + 2] = False
        x = x.copy()
        x[rng.integers(0, nx), rng.integers(0, ny)] = np.nan
    return (pkg.SSA.image(x, lx, ly, wmask=wmask, mask=mask),
            O.Problem.image(x, lx, ly, wmask=wmask, mask=mask), x)


SMALL = [
    ("1d_37_11", lambda: case_1d(37, 11, 1)),
    ("1d_1000_500", lambda: case_1d(1000, 500, 2)),
    ("1d_1000_700_swapped", lambda: case_1d(1000, 700, 3)),
    ("1d_4097_1500", lambda: case_1d(4097, 1500, 4)),
    ("1d_gaps_600_80", lambda: case_1d_gaps(600, 80, 11, [(130, 133), (400, 401)])),
    ("mssa_3x_gaps", lambda: case_mssa_gaps([120, 173, 161], 30, 12)),
    ("mssa_3x_ragged", lambda: case_mssa([50, 73, 61], 20, 5)),
    ("mssa_5x_300_700", lambda: case_mssa([300, 701, 455, 512, 333], 100, 6)),
    ("2d_30x27_w7x5", lambda: case_2d(30, 27, 7, 5, 7)),
    ("2d_100x130_w20x30", lambda: case_2d(100, 130, 20, 30, 8)),
    ("shaped_40x35_circle4_holes", lambda: case_2d(40, 35, 9, 9, 9, wmask=pkg.window_circle(4), holes=True)),
    ("shaped_64x50_triangle6", lambda: case_2d(64, 50, 6, 6, 10, wmask=pkg.window_triangle(6), holes=True)),
]


def flat(P, arrs):
    """oracle per-channel arrays -> the library's flat layout"""
    return np.concatenate([np.asarray(a).ravel(order="F") for a in arrs])


@pytest.mark.parametrize("name,make", SMALL, ids=[s[0] for s in SMALL])
def test_shapes_exact(name, make):
    s, P, _ = make()
    L, K, om, w = s.shape()
    assert L == P.L and K == P.K
    om_ref, w_ref = [], []
    for c in range(len(P.channels)):
        shp = P.channels[c].shape
        m = np.zeros(shp, np.uint8)
        if len(P.Ksets[c]):
            m[P.Ksets[c][:, 0], P.Ksets[c][:, 1]] = 1
        om_ref.append(m)
        w_ref.append(P.weights(c))
    np.testing.assert_array_equal(np.ravel(om, order="F") if not isinstance(om, list) else np.concatenate(om),
                                  flat(P, om_ref))
    np.testing.assert_array_equal(np.ravel(w, order="F") if not isinstance(w, list) else np.concatenate(w),
                                  flat(P, w_ref))


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("name,make", SMALL, ids=[s[0] for s in SMALL])
def test_matvec(name, make, prec):
    s, P, _ = make()
    rng = np.random.default_rng(0)
    xnorm = math.sqrt(sum(np.nansum(np.where(o, c, 0.0) ** 2) for c, o in zip(P.channels, P.obs)))
    v = rng.normal(size=P.K)
    u = rng.normal(size=P.L)
    got = s.matvec(v, False, prec)
    ref = O.matvec(P, v)
    assert np.max(np.abs(got - ref)) <= TOL_MV[prec] * xnorm * np.linalg.norm(v)
    got = s.matvec(u, True, prec)
    ref = O.rmatvec(P, u)
    assert np.max(np.abs(got - ref)) <= TOL_MV[prec] * xnorm * np.linalg.norm(u)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("name,make", SMALL, ids=[s[0] for s in SMALL])
def test_decompose_and_reconstruct(name, make, prec):
    s, P, x = make()
    r = min(8, min(P.L, P.K) - 1)
    so, Uo, Vo = O.decompose(P, r + 1)
    s.decompose(r, prec)
    sig = s.sigma()
    rel = np.abs(sig - so[:r]) / so[:r]
    assert rel.max() <= TOL_SIG[prec], (rel, sig, so)
    groups = gap_groups(so[:r + 1])
    groups = [g for g in groups if max(g) < r]
    if not groups:
        return
    rec = s.reconstruct(groups, residual=True)
    ref = O.reconstruct(P, so, Uo, Vo, groups, residual=True)
    xmax = max(np.nanmax(np.abs(np.where(o, c, np.nan))) for c, o in zip(P.channels, P.obs))
    for g in range(len(groups) + 1):
        got = rec[g]
        got = [got] if not isinstance(got, list) else got
        for c in range(len(P.channels)):
            a = np.asarray(got[c]).reshape(P.channels[c].shape, order="F")
            b = ref[g][c]
            np.testing.assert_array_equal(np.isnan(a), np.isnan(b))
            err = np.nanmax(np.abs(a - b)) / xmax
            assert err <= TOL_REC[prec], (g, err)


def test_vectors_satisfy_svd_relations():
    """U, V returned by the C ABI: orthonormal and X V_i = sigma_i U_i."""
    s, P, _ = case_2d(48, 40, 9, 7, 11)
    s.decompose(6, "fp64")
    sig = s.sigma()
    U, V = s.vectors()
    np.testing.assert_allclose(U.T @ U, np.eye(6), atol=1e-9)
    np.testing.assert_allclose(V.T @ V, np.eye(6), atol=1e-9)
    for i in range(6):
        np.testing.assert_allclose(O.matvec(P, V[:, i]), sig[i] * U[:, i], atol=1e-8 * sig[0])
        k = np.argmax(np.abs(U[:, i]))
        assert U[k, i] > 0


def test_fp32_vectors_satisfy_svd_relations():
    """FP32 form: the long-side Ritz vectors come from the tensor-core
    contraction (3xTF32 split, FP32 accumulation in TMEM) at every restart and
    at the end; they stay orthonormal to FP32 level and satisfy
    X V_i = sigma_i U_i to the form's accuracy on an MSSA problem that
    restarts several times."""
    s, P, _ = case_mssa([300, 701, 455, 512, 333], 100, 6)
    s.decompose(12, "fp32", krylov_dim=30)
    assert s.info()["restarts"] >= 2
    sig = s.sigma()
    U, V = s.vectors()
    np.testing.assert_allclose(V.T @ V, np.eye(12), atol=2e-5)
    for i in range(12):
        np.testing.assert_allclose(O.matvec(P, V[:, i]), sig[i] * U[:, i], atol=2e-5 * sig[0])
    so = O.decompose(P, 12)[0]
    np.testing.assert_allclose(sig, so, rtol=TOL_SIG["fp32"], atol=0)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_small_svd_fp32_rotations_fp64_polish(prec):
    """The small SVD finds its rotations in FP32 and polishes them in a few
    FP64 sweeps; the triples keep the accuracy of the form."""
    x = W.series_1d(3000, seed=17)
    s = pkg.SSA.series(x, 1200)
    s.decompose(12, prec, seed=4)
    inf = s.info()
    assert inf["jacobi_sweeps_fp32"] >= 1
    assert 1 <= inf["jacobi_sweeps"] <= 4, inf["jacobi_sweeps"]
    so, _, _ = O.decompose(O.Problem.series(x, 1200), 12)
    np.testing.assert_allclose(s.sigma(), so, rtol=TOL_SIG[prec], atol=0)
    s.close()


def test_batch_equals_single():
    """ssa_decompose_batch gives each problem the result it gets alone."""
    cases = [case_mssa([300, 400, 350], 80, 20 + i)[0] for i in range(3)]
    singles = []
    for s in cases:
        s.decompose(6, "fp32")
        singles.append(s.sigma())
    pkg.decompose_batch(cases, 6, "fp32")
    for s, ref in zip(cases, singles):
        np.testing.assert_allclose(s.sigma(), ref, rtol=1e-6)


def test_batch_images_of_different_heights():
    """One y-pass launch serves images whose y-grids differ: each item keeps
    the tile width that fits its own column length, and the launch's staging
    buffer is sized for the largest tile x column among them (a wide tile of
    a short image times the column of a tall one overflowed shared memory)."""
    def image(nx, ny, seed):
        rng = np.random.default_rng(seed)
        m, n = np.arange(nx)[:, None], np.arange(ny)[None, :]
        return (np.cos(2 * np.pi * m / 9 + 0.3) * np.cos(2 * np.pi * n / 13 + 0.7)
                + 0.5 * np.cos(2 * np.pi * m / 5) * np.sin(2 * np.pi * n / 31) + 0.05 * rng.standard_normal((nx, ny)))
    specs = [(40, 10, 6, 4, 1), (48, 700, 8, 40, 2), (36, 24, 5, 6, 3)]
    singles = []
    for nx, ny, lx, ly, sd in specs:
        s = pkg.SSA.image(image(nx, ny, sd), lx, ly)
        s.decompose(4, "fp32")
        singles.append(s.sigma())
        s.close()
    batch = [pkg.SSA.image(image(nx, ny, sd), lx, ly) for nx, ny, lx, ly, sd in specs]
    pkg.decompose_batch(batch, 4, "fp32")
    for s, ref in zip(batch, singles):
        np.testing.assert_allclose(s.sigma(), ref, rtol=1e-6)
        s.close()


def test_shared_u_transform_batch_equals_single():
    """Engines of 32 problems or more transform u_j once per problem and grid
    size (k_uspec, compile-time sizes for grids of 2^11..2^13 points) and the
    X^T u products read it; alone, a problem transforms u_j inside each
    product.  Both give the same triples and components."""
    cases = [pkg.SSA.multi(W.mssa_series(3, seed=60 + i), 1000) for i in range(34)]
    ref = []
    for s in cases[:3] + cases[-2:]:
        s.decompose(6, "fp32", seed=4)
        ref.append((s.sigma(), s.reconstruct([[0], [1, 2]])))
    pkg.decompose_batch(cases, 6, "fp32", seed=4)
    for s, (sig, rec) in zip(cases[:3] + cases[-2:], ref):
        np.testing.assert_allclose(s.sigma(), sig, rtol=1e-5, atol=0)
        got = s.reconstruct([[0], [1, 2]])
        for ga, gb in zip(got, rec):          # groups, then the system's series
            for a, b in zip(ga, gb):
                np.testing.assert_allclose(a, b, rtol=0, atol=1e-4 * float(np.nanmax(np.abs(b))))
    for s in cases:
        s.close()


def test_large_batch_runs_in_two_halves_with_single_results():
    """Batches of 64 problems or more run as two interleaved halves on two
    streams; every problem still gets the result it gets alone."""
    cases = [case_1d(300 + 7 * i, 90, 40 + i)[0] for i in range(70)]
    singles = []
    for s in cases[:6] + cases[-6:]:
        s.decompose(5, "fp32", seed=3)
        singles.append((s.sigma(), s.reconstruct([[0], [1, 2]])))
    pkg.decompose_batch(cases, 5, "fp32", seed=3)
    for s, (ref, rec) in zip(cases[:6] + cases[-6:], singles):
        np.testing.assert_allclose(s.sigma(), ref, rtol=1e-12, atol=0)
        got = s.reconstruct([[0], [1, 2]])
        for a, b in zip(got, rec):
            np.testing.assert_allclose(a, b, rtol=0, atol=1e-12 * float(np.max(np.abs(b))))


# ------------------------------------------------------------------ errors
def test_error_codes():
    lib = pkg.load()
    x = noisy_series(50, 1)
    with pytest.raises(pkg.SSAError) as e:
        pkg.SSA.series(x, 50)
    assert e.value.code == -1
    y = x.copy()
    y[3] = np.inf
    with pytest.raises(pkg.SSAError) as e:
        pkg.SSA.series(y, 10)
    assert e.value.code == -1
    img = np.full((20, 20), np.nan)
    img[:5, :5] = 1.0
    with pytest.raises(pkg.SSAError) as e:
        pkg.SSA.image(img, 8, 8)
    assert e.value.code == -2
    s = pkg.SSA.series(x, 10)
    with pytest.raises(pkg.SSAError) as e:
        s.decompose(11)
    assert e.value.code == -3
    with pytest.raises(pkg.SSAError) as e:
        s.reconstruct([[0]])
    assert e.value.code == -8
    del lib


def test_rank_edge_cases():
    """r = 1, r = min(L, K) and L = 2."""
    x = noisy_series(60, 3)
    for L, r in [(2, 1), (2, 2), (30, 30), (12, 1)]:
        s = pkg.SSA.series(x, L)
        P = O.Problem.series(x, L)
        s.decompose(r, "fp64")
        so = O.decompose(P, r)[0]
        np.testing.assert_allclose(s.sigma(), so, rtol=1e-9)


def test_empty_groups_and_skipped_components():
    x = noisy_series(200, 4)
    s = pkg.SSA.series(x, 60)
    s.decompose(6)
    rec = s.reconstruct([[], [0]], residual=False)
    ok = ~np.isnan(rec[0])
    assert np.all(rec[0][ok] == 0.0)


# ------------------------------------------------------------------ full-size workloads
def golden(name):
    d = np.load(os.path.join(GOLDEN, name + ".npz"))
    return d["sigma"], d["U"], int(d["L"]), int(d["K"])


def check_sigma(sig, ref, prec="fp32"):
    rel = np.abs(sig - ref) / ref
    assert rel.max() <= TOL_SIG[prec], rel


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_workload_series_1d_n1000(prec):
    cfg = W.CONFIGS["series_1d_n1000"]
    x = W.series_1d(cfg["n"], seed=cfg["seed"])
    ref, Ug, L, K = golden("series_1d_n1000")
    s = pkg.SSA.series(x, cfg["L"])
    s.decompose(cfg["rank"], prec)
    check_sigma(s.sigma(), ref, prec)
    P = O.Problem.series(x, cfg["L"])
    so, Uo, Vo = O.decompose(P, cfg["rank"])
    xmax = np.abs(x).max()
    # gap-bounded groups, then the groups of the workload ({1,2},{3,4},rest);
    # every element of every group and of the residual
    for groups in ([[0], [1, 2], [3], [4, 5]], cfg["groups"]):
        rec = s.reconstruct(groups, residual=True)
        refr = O.reconstruct(P, so, Uo, Vo, groups, residual=True)
        for g in range(len(groups) + 1):
            err = np.nanmax(np.abs(rec[g] - refr[g][0][:, 0])) / xmax
            assert err <= TOL_REC[prec], (groups, g, err)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_workload_mssa_16_series(prec):
    """The MSSA workload at full size (16 series of 2000..8000 samples, L =
    1000, r = 20): singular values against the stored oracle values, and every
    reconstructed element of all 16 series -- each group and the residual --
    against the oracle's diagonal averaging."""
    cfg = W.CONFIGS["mssa_16x2000-8000_L1000"]
    xs = W.mssa_series(cfg["s"], seed=cfg["seed"])
    ref, Ug, L, K = golden("mssa_16x2000-8000_L1000")
    s = pkg.SSA.multi(xs, cfg["L"])
    assert s.info()["K"] == K
    s.decompose(cfg["rank"], prec)
    check_sigma(s.sigma(), ref, prec)
    groups = [[0], [1, 2], [3, 4]]
    rec = s.reconstruct(groups, residual=True)
    P = O.Problem.multi([np.asarray(v, np.float64) for v in xs], cfg["L"])
    so, Uo, Vo = O.decompose(P, 5)
    refr = O.reconstruct(P, so, Uo, Vo, groups, residual=True)
    xmax = max(np.abs(v).max() for v in xs)
    for g in range(len(groups) + 1):
        for c in range(cfg["s"]):
            got = rec[g][c]
            want = refr[g][c][:, 0]
            assert got.shape == want.shape
            err = np.max(np.abs(got - want)) / xmax
            assert err <= TOL_REC[prec], (g, c, err)


def image_points(w, n_low, n_any, seed):
    """Sample points of an image for element-wise checks: n_low among the
    elements with 0 < w < 64 (borders, corners, rims of holes: there the
    reconstruction divides by a small count, which amplifies FFT error),
    n_any among all elements of N', plus the four corners of the grid."""
    rng = np.random.default_rng(seed)
    nx, ny = w.shape
    low = np.argwhere((w > 0) & (w < 64))
    anyw = np.argwhere(w > 0)
    pts = [(0, 0), (nx - 1, ny - 1), (0, ny - 1), (nx - 1, 0)]
    for src, n in ((low, n_low), (anyw, n_any)):
        if len(src):
            for i in rng.choice(len(src), size=min(n, len(src)), replace=False):
                pts.append((int(src[i][0]), int(src[i][1])))
    return pts


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("name", ["image_1024x1024_w64", "shaped_2048x2048_disc40holes_w32"])
def test_workload_images(name, prec):
    """The 2D-SSA (1024^2, window 64^2, r = 30) and Shaped 2D-SSA (2048^2 disc
    with 40 holes, window 32^2, r = 20) workloads at full size: singular
    values against the stored oracle values, and each gap-bounded group at
    more than 200 elements, most of them where the weight is below 64."""
    cfg = W.CONFIGS[name]
    if cfg["kind"] == "2d":
        x = W.harmonic_image(cfg["nx"], cfg["ny"], seed=cfg["seed"])
    else:
        x, mask, _ = W.shaped_image(cfg["nx"], cfg["ny"], seed=cfg["seed"])
    ref, Ug, L, K = golden(name)
    s = pkg.SSA.image(x, cfg["lx"], cfg["ly"])
    assert s.info()["L"] == L and s.info()["K"] == K
    s.decompose(cfg["rank"], prec)
    check_sigma(s.sigma(), ref, prec)
    groups = gap_groups(ref)
    rec = s.reconstruct(groups)
    _, _, _, w = s.shape()
    w = np.asarray(w).reshape(cfg["nx"], cfg["ny"], order="F") if np.ndim(w) == 1 else np.asarray(w)
    pts = image_points(w, 170, 30, 1)
    P = O.Problem.image(x, cfg["lx"], cfg["ly"])
    xmax = np.nanmax(np.abs(x))
    for gi, g in enumerate(groups):
        want = O.reconstruct_at(P, Ug[:, g], pts)
        got = np.array([rec[gi][m, n] for m, n in pts])
        np.testing.assert_array_equal(np.isnan(got), np.isnan(want))
        err = np.nanmax(np.abs(got - want)) / xmax
        assert err <= TOL_REC[prec], (g, err)
    # elements outside N' are NaN in every group
    outside = np.argwhere(w == 0)
    if len(outside):
        sel = outside[np.random.default_rng(2).choice(len(outside), size=min(50, len(outside)), replace=False)]
        for gi in range(len(groups)):
            assert np.all(np.isnan(rec[gi][sel[:, 0], sel[:, 1]]))
