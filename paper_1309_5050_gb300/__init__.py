"""GB300-native Singular Spectrum Analysis (SSA, MSSA, 2D-SSA, Shaped 2D-SSA).

Python face of ``libssa.so``; see ``include/ssa.h`` for the C ABI.  Inputs may
be numpy arrays (host) or CUDA torch tensors (device, used in place).  All
computation happens in the library's sm_103a kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L
from ._lib import (SSA_1D, SSA_2D, SSA_F32, SSA_F64, SSA_MSSA,  # noqa: F401
                   SSA_PREC_FP32FFT_FP64REORTH, SSA_PREC_FP64, SSAError)

__all__ = ["SSA", "Server", "embed_multi_batch", "embed_series_batch", "decompose_batch", "reconstruct_batch", "window_circle", "window_triangle",
           "load", "SSAError", "PREC", "save_plans", "load_plans"]

PREC = {"fp32": SSA_PREC_FP32FFT_FP64REORTH, "fp64": SSA_PREC_FP64}


def load():
    """Load (building if needed) the CUDA library."""
    return L.load()


def window_circle(R: int) -> np.ndarray:
    """Circular window of radius R (bounding box (2R+1)^2, (i-R)^2+(j-R)^2 <= R^2)."""
    i = np.arange(2 * R + 1)[:, None]
    j = np.arange(2 * R + 1)[None, :]
    return (i - R) ** 2 + (j - R) ** 2 <= R * R


def window_triangle(side: int) -> np.ndarray:
    """Right isosceles triangle, right angle top-left: i + j <= side - 1."""
    i = np.arange(side)[:, None]
    j = np.arange(side)[None, :]
    return i + j <= side - 1


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _buf(x, dtype=None):
    """(pointer, on_device, keepalive, dtype_code) for a numpy array or a torch tensor."""
    if _is_torch(x):
        if not x.is_contiguous():
            x = x.contiguous()
        code = {"torch.float32": SSA_F32, "torch.float64": SSA_F64}.get(str(x.dtype))
        return x.data_ptr(), 1 if x.is_cuda else 0, x, code
    a = np.ascontiguousarray(x) if dtype is None else np.ascontiguousarray(x, dtype=dtype)
    code = {np.dtype(np.float32): SSA_F32, np.dtype(np.float64): SSA_F64}.get(a.dtype)
    return a.ctypes.data, 0, a, code


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


class SSA:
    """One SSA problem held on the GPU (a library context)."""

    def __init__(self, inp: L.ssa_input, win: L.ssa_window, keep, stream=None, layout=None):
        lib = L.load()
        ctx = C.c_void_p()
        L.check(lib.ssa_embed(C.byref(inp), C.byref(win), _stream_ptr(stream), C.byref(ctx)), "ssa_embed")
        self._lib = lib
        self.ctx = ctx
        self.layout = layout            # ("1d", n) | ("mssa", lengths) | ("2d", nx, ny)
        self.rank = 0
        del keep

    @classmethod
    def _wrap(cls, ctx, layout):
        obj = cls.__new__(cls)
        obj._lib = L.load()
        obj.ctx = ctx
        obj.layout = layout
        obj.rank = 0
        return obj

    # ----------------------------------------------------------- builders
    @classmethod
    def series(cls, x, L_: int, stream=None):
        if not _is_torch(x):
            x = np.asarray(x)
            if x.dtype not in (np.float32, np.float64):
                x = x.astype(np.float64)
        ptr, dev, keep, code = _buf(x)
        n = int(x.shape[0])
        inp = L.ssa_input(kind=SSA_1D, dtype=code, on_device=dev, n_series=1, data=ptr, n=n)
        win = L.ssa_window(L=L_)
        return cls(inp, win, keep, stream, ("1d", n))

    @classmethod
    def multi(cls, xs, L_: int, stream=None, dtype=np.float32):
        """MSSA of a list of series (host arrays) or of one concatenated
        device tensor with ``lengths``."""
        if isinstance(xs, (list, tuple)):
            lengths = np.array([len(v) for v in xs], dtype=np.int64)
            cat = np.concatenate([np.asarray(v, dtype=dtype) for v in xs])
            ptr, dev, keep, code = _buf(cat)
        else:
            raise TypeError("multi() takes a list of series; use multi_concat for a flat buffer")
        return cls._multi_flat(ptr, dev, keep, code, lengths, L_, stream)

    @classmethod
    def multi_concat(cls, flat, lengths, L_: int, stream=None):
        ptr, dev, keep, code = _buf(flat)
        return cls._multi_flat(ptr, dev, keep, code, np.asarray(lengths, dtype=np.int64), L_, stream)

    @classmethod
    def _multi_flat(cls, ptr, dev, keep, code, lengths, L_, stream):
        lens = np.ascontiguousarray(lengths, dtype=np.int64)
        inp = L.ssa_input(kind=SSA_MSSA, dtype=code, on_device=dev, n_series=len(lens), data=ptr,
                          lengths=lens.ctypes.data_as(C.POINTER(C.c_int64)))
        win = L.ssa_window(L=L_)
        obj = cls(inp, win, (keep, lens), stream, ("mssa", lens.copy()))
        return obj

    @classmethod
    def image(cls, x, lx: int, ly: int, wmask=None, mask=None, stream=None):
        """2D-SSA / Shaped 2D-SSA of an (nx, ny) image (x down, y right).
        Host arrays are passed column-major; a device tensor must already be
        laid out column-major (i.e. be the transpose-contiguous view)."""
        if _is_torch(x):
            nx, ny = int(x.shape[0]), int(x.shape[1])
            xt = x.t().contiguous()          # column-major bytes
            ptr, dev, keep, code = _buf(xt)
        else:
            a = np.asarray(x)
            if a.dtype not in (np.float32, np.float64):
                a = a.astype(np.float64)
            nx, ny = a.shape
            af = np.asfortranarray(a)
            ptr, dev, keep, code = af.ctypes.data, 0, af, {np.dtype(np.float32): SSA_F32,
                                                            np.dtype(np.float64): SSA_F64}[af.dtype]
        mptr, mkeep = None, None
        if mask is not None:
            if _is_torch(mask):
                mkeep = mask.t().contiguous().to(dtype=__import__("torch").uint8)
                mptr = mkeep.data_ptr()
            else:
                if dev:
                    raise TypeError("a device image needs a device mask")
                m = np.asfortranarray(np.asarray(mask, dtype=np.uint8))
                mptr, mkeep = m.ctypes.data, m
        wptr, wkeep = None, None
        if wmask is not None:
            w = np.asfortranarray(np.asarray(wmask, dtype=np.uint8))
            wptr, wkeep = w.ctypes.data, w
            lx, ly = w.shape
        inp = L.ssa_input(kind=SSA_2D, dtype=code, on_device=dev, n_series=1, data=ptr, nx=nx, ny=ny, mask=mptr)
        win = L.ssa_window(lx=lx, ly=ly, wmask=wptr)
        return cls(inp, win, (keep, mkeep, wkeep), stream, ("2d", nx, ny))

    # ----------------------------------------------------------- calls
    def decompose(self, rank: int, prec: str = "fp32", krylov_dim: int = 0, tol: float = 0.0,
                  seed: int = 0, max_restarts: int = 0, check: bool = True) -> int:
        p = L.ssa_params(rank=rank, krylov_dim=krylov_dim, max_restarts=max_restarts,
                         prec=PREC[prec], tol=tol, seed=seed)
        rc = self._lib.ssa_decompose(self.ctx, C.byref(p))
        if check:
            L.check(rc, "ssa_decompose")
        self.rank = rank
        return rc

    def extend(self, rank: int, prec: str = "fp32", krylov_dim: int = 0, tol: float = 0.0,
               max_restarts: int = 0) -> int:
        """Continue the decomposition to a larger rank (ssa_continue): the
        previous Ritz triples and residual direction seed the new Krylov
        space instead of a new start vector."""
        p = L.ssa_params(rank=rank, krylov_dim=krylov_dim, max_restarts=max_restarts,
                         prec=PREC[prec], tol=tol, seed=0)
        L.check(self._lib.ssa_continue(self.ctx, C.byref(p)), "ssa_continue")
        self.rank = rank
        return 0

    def autotune(self, rank: int, prec: str = "fp32", seed: int = 0) -> dict:
        """Time the candidate plans on this problem (ssa_autotune), record
        the fastest for its size class and leave the problem decomposed."""
        p = L.ssa_params(rank=rank, krylov_dim=0, max_restarts=0, prec=PREC[prec], tol=0.0, seed=seed)
        res = L.ssa_tune_result()
        L.check(self._lib.ssa_autotune(self.ctx, C.byref(p), C.byref(res)), "ssa_autotune")
        self.rank = rank
        return {f: getattr(res, f) for f, _ in L.ssa_tune_result._fields_ if f != "pad_"}

    def info(self) -> dict:
        i = L.ssa_info()
        L.check(self._lib.ssa_get_info(self.ctx, C.byref(i)), "ssa_get_info")
        return {f: getattr(i, f) for f, _ in L.ssa_info._fields_}

    def sigma(self, r: int | None = None) -> np.ndarray:
        r = self.rank if r is None else r
        out = np.zeros(r)
        L.check(self._lib.ssa_get_sigma(self.ctx, out.ctypes.data_as(C.POINTER(C.c_double)), r), "ssa_get_sigma")
        return out

    def vectors(self):
        inf = self.info()
        U = np.zeros((inf["L"], self.rank), order="F")
        V = np.zeros((inf["K"], self.rank), order="F")
        L.check(self._lib.ssa_get_vectors(self.ctx, U.ctypes.data, V.ctypes.data, 0), "ssa_get_vectors")
        return U, V

    def _total(self):
        if self.layout[0] == "1d":
            return self.layout[1]
        if self.layout[0] == "mssa":
            return int(np.sum(self.layout[1]))
        return self.layout[1] * self.layout[2]

    def _split(self, flat):
        return _split_layout(self.layout, flat)

    def reconstruct(self, groups, residual: bool = False):
        """groups: list of lists of 0-based component indices.  Returns one
        array per group (plus the residual) in the input's shape; NaN outside N'."""
        gof = _group_of(groups, self.rank)
        nout = len(groups) + (1 if residual else 0)
        total = self._total()
        out = np.zeros(total * nout)
        L.check(self._lib.ssa_reconstruct(self.ctx, gof.ctypes.data_as(C.POINTER(C.c_int32)), len(groups),
                                          1 if residual else 0, out.ctypes.data, 0), "ssa_reconstruct")
        return [self._split(out[g * total:(g + 1) * total]) for g in range(nout)]

    def wcor(self, groups=None):
        """w-correlation matrix (n x n) and contributions (n) of the
        reconstructed components of ``groups`` (default: the elementary
        components 0..r-1), Sec. 2.2; computed by ssa_wcor on the device."""
        if groups is None:
            groups = [[i] for i in range(self.rank)]
        gof = _group_of(groups, self.rank)
        n = len(groups)
        rho = np.zeros(n * n)
        contrib = np.zeros(n)
        L.check(self._lib.ssa_wcor(self.ctx, gof.ctypes.data_as(C.POINTER(C.c_int32)), n, rho.ctypes.data,
                                   contrib.ctypes.data), "ssa_wcor")
        return rho.reshape(n, n), contrib

    def forecast(self, group, M: int, method: str = "recurrent"):
        """M-step forecast of the component ``group`` (0-based indices),
        Sec. 3.3: ``method`` "recurrent" or "vector" (column forecasts,
        ssa_forecast / ssa_forecast_vector), "recurrent_row" or "vector_row"
        (row forecasts, ssa_forecast_row).  One array of M values for a
        series, a list of them for an MSSA system."""
        idx = np.ascontiguousarray(list(group), dtype=np.int32)
        multi = self.layout[0] == "mssa"
        ns = len(self.layout[1]) if multi else 1
        out = np.zeros(ns * M)
        ip = idx.ctypes.data_as(C.POINTER(C.c_int32))
        if method in ("recurrent_row", "vector_row"):
            L.check(self._lib.ssa_forecast_row(self.ctx, ip, len(idx), int(M), 1 if method == "vector_row" else 0,
                                               out.ctypes.data), "ssa_forecast_row")
        else:
            fn = {"recurrent": "ssa_forecast", "vector": "ssa_forecast_vector"}[method]
            L.check(getattr(self._lib, fn)(self.ctx, ip, len(idx), int(M), out.ctypes.data), fn)
        parts = [out[p * M:(p + 1) * M] for p in range(ns)]
        return parts if multi else parts[0]

    def shape(self):
        """(L, K, origin_mask, weights) in the input's layout."""
        total = self._total()
        Lc, Kc = C.c_int64(), C.c_int64()
        om = np.zeros(total, dtype=np.uint8)
        w = np.zeros(total, dtype=np.int32)
        L.check(self._lib.ssa_get_shape(self.ctx, C.byref(Lc), C.byref(Kc), om.ctypes.data, w.ctypes.data),
                "ssa_get_shape")
        return Lc.value, Kc.value, self._split(om), self._split(w)

    def matvec(self, v, transpose: bool = False, prec: str = "fp32") -> np.ndarray:
        inf = self.info()
        nin, nout = (inf["L"], inf["K"]) if transpose else (inf["K"], inf["L"])
        a = np.ascontiguousarray(v, dtype=np.float64)
        assert a.shape == (nin,)
        out = np.zeros(nout)
        L.check(self._lib.ssa_matvec(self.ctx, 1 if transpose else 0, PREC[prec], a.ctypes.data, out.ctypes.data, 0),
                "ssa_matvec")
        return out

    def synchronize(self):
        L.check(self._lib.ssa_synchronize(self.ctx), "ssa_synchronize")

    def close(self):
        if self.ctx:
            self._lib.ssa_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _split_layout(layout, flat):
    """One flat output (the library's element order) in the input's shape."""
    kind = layout[0]
    if kind == "1d":
        return flat
    if kind == "mssa":
        offs = np.concatenate([[0], np.cumsum(layout[1])])
        return [flat[offs[i]:offs[i + 1]] for i in range(len(layout[1]))]
    return flat.reshape((layout[1], layout[2]), order="F")


def _group_of(groups, rank):
    need = max([rank] + [i + 1 for g in groups for i in g])
    gof = np.full(max(need, 1), -1, dtype=np.int32)
    for g, idx in enumerate(groups):
        for i in idx:
            gof[i] = g
    return gof


class Server:
    """Many SSA requests in flight on one GPU (continuous batching at
    restart-cycle granularity, admission by a device-memory budget); the C
    side is ssa_server_* in include/ssa.h.  Requests take host data."""

    def __init__(self, memory_budget: int = 40 << 30, max_live: int = 512, prec: str = "fp32", stream=None):
        self._lib = L.load()
        cfg = L.ssa_server_config(memory_budget=int(memory_budget), max_live=int(max_live), prec=PREC[prec])
        h = C.c_void_p()
        L.check(self._lib.ssa_server_create(C.byref(cfg), _stream_ptr(stream), C.byref(h)), "ssa_server_create")
        self.h = h
        self._meta = {}

    def _submit(self, inp, win, layout, total, rank, groups, residual, seed, tol, krylov_dim, max_restarts):
        groups = [] if groups is None else groups
        p = L.ssa_params(rank=rank, krylov_dim=krylov_dim, max_restarts=max_restarts, prec=0, tol=tol, seed=seed)
        gof = _group_of(groups, rank)
        t = C.c_int64()
        L.check(self._lib.ssa_server_submit(self.h, C.byref(inp), C.byref(win), C.byref(p),
                                            gof.ctypes.data if groups else None, len(groups),
                                            1 if residual else 0, C.byref(t)), "ssa_server_submit")
        self._meta[t.value] = (layout, total, rank, len(groups) + (1 if residual else 0))
        return t.value

    def submit_series(self, x, L_: int, rank: int, groups=None, residual: bool = False, seed: int = 0,
                      tol: float = 0.0, krylov_dim: int = 0, max_restarts: int = 0) -> int:
        a = np.ascontiguousarray(x)
        if a.dtype not in (np.float32, np.float64):
            a = a.astype(np.float64)
        code = SSA_F32 if a.dtype == np.float32 else SSA_F64
        n = int(a.shape[0])
        inp = L.ssa_input(kind=SSA_1D, dtype=code, on_device=0, n_series=1, data=a.ctypes.data, n=n)
        return self._submit(inp, L.ssa_window(L=L_), ("1d", n), n, rank, groups, residual, seed, tol,
                            krylov_dim, max_restarts)

    def submit_multi(self, xs, L_: int, rank: int, groups=None, residual: bool = False, seed: int = 0,
                     tol: float = 0.0, krylov_dim: int = 0, max_restarts: int = 0, dtype=np.float32) -> int:
        lens = np.array([len(v) for v in xs], dtype=np.int64)
        cat = np.ascontiguousarray(np.concatenate([np.asarray(v, dtype=dtype) for v in xs]))
        code = SSA_F32 if cat.dtype == np.float32 else SSA_F64
        inp = L.ssa_input(kind=SSA_MSSA, dtype=code, on_device=0, n_series=len(lens), data=cat.ctypes.data,
                          lengths=lens.ctypes.data_as(C.POINTER(C.c_int64)))
        return self._submit(inp, L.ssa_window(L=L_), ("mssa", lens.copy()), int(lens.sum()), rank, groups,
                            residual, seed, tol, krylov_dim, max_restarts)

    def submit_image(self, x, lx: int, ly: int, rank: int, wmask=None, mask=None, groups=None,
                     residual: bool = False, seed: int = 0, tol: float = 0.0, krylov_dim: int = 0,
                     max_restarts: int = 0) -> int:
        a = np.asarray(x)
        if a.dtype not in (np.float32, np.float64):
            a = a.astype(np.float64)
        nx, ny = a.shape
        af = np.asfortranarray(a)
        code = SSA_F32 if af.dtype == np.float32 else SSA_F64
        mptr = None
        if mask is not None:
            m = np.asfortranarray(np.asarray(mask, dtype=np.uint8))
            mptr = m.ctypes.data
        wptr = None
        if wmask is not None:
            w = np.asfortranarray(np.asarray(wmask, dtype=np.uint8))
            wptr = w.ctypes.data
            lx, ly = w.shape
        inp = L.ssa_input(kind=SSA_2D, dtype=code, on_device=0, n_series=1, data=af.ctypes.data, nx=nx, ny=ny,
                          mask=mptr)
        win = L.ssa_window(lx=lx, ly=ly, wmask=wptr)
        return self._submit(inp, win, ("2d", nx, ny), nx * ny, rank, groups, residual, seed, tol, krylov_dim,
                            max_restarts)

    def step(self) -> int:
        """Admit, run one restart cycle for every live request, retire the
        converged ones; returns how many finished."""
        n = C.c_int32()
        L.check(self._lib.ssa_server_step(self.h, C.byref(n)), "ssa_server_step")
        return n.value

    def stats(self) -> dict:
        q, lv, f, b = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        L.check(self._lib.ssa_server_stats(self.h, C.byref(q), C.byref(lv), C.byref(f), C.byref(b)),
                "ssa_server_stats")
        return {"queued": q.value, "live": lv.value, "finished": f.value, "bytes_live": b.value}

    def finished(self, cap: int = 4096) -> list:
        """Tickets of finished requests not taken yet."""
        buf = (C.c_int64 * cap)()
        n = C.c_int32()
        L.check(self._lib.ssa_server_finished(self.h, buf, cap, C.byref(n)), "ssa_server_finished")
        return [buf[i] for i in range(n.value)]

    def take(self, ticket: int) -> dict:
        """Result of a finished request: status, sigma, outputs (one per group,
        plus the residual, in the input's shape) and its timestamps."""
        if ticket not in self._meta:        # unknown or already taken: the library says which
            L.check(self._lib.ssa_server_take(self.h, ticket, None, None, None), "ssa_server_take")
        layout, total, rank, nout = self._meta[ticket]
        res = L.ssa_server_result()
        sig = np.zeros(max(rank, 1))
        out = np.zeros(max(total * nout, 1))
        L.check(self._lib.ssa_server_take(self.h, ticket, C.byref(res), sig.ctypes.data, out.ctypes.data),
                "ssa_server_take")
        del self._meta[ticket]
        d = {f: getattr(res, f) for f, _ in L.ssa_server_result._fields_ if f != "pad_"}
        d["sigma"] = sig[:rank]
        d["outputs"] = [_split_layout(layout, out[g * total:(g + 1) * total]) for g in range(nout)] \
            if res.out_len else []
        return d

    def clock(self) -> float:
        return float(self._lib.ssa_server_clock(self.h))

    def drain(self, max_steps: int = 1_000_000) -> int:
        """Step until nothing is queued or live; returns the steps taken."""
        steps = 0
        while steps < max_steps:
            s = self.stats()
            if s["queued"] == 0 and s["live"] == 0:
                break
            self.step()
            steps += 1
        return steps

    def close(self):
        if getattr(self, "h", None):
            self._lib.ssa_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def embed_multi_batch(flats, lengths, L_: int, stream=None):
    """Batched MSSA embed of n problems: flats[i] holds problem i's series
    concatenated (numpy array or torch tensor, host or device), lengths[i]
    their lengths.  Returns n SSA objects."""
    lib = L.load()
    n = len(flats)
    ins = (L.ssa_input * n)()
    wins = (L.ssa_window * n)()
    keep = []
    for i, (f, ln) in enumerate(zip(flats, lengths)):
        ptr, dev, kp, code = _buf(f)
        lens = np.ascontiguousarray(ln, dtype=np.int64)
        keep.append((kp, lens))
        ins[i] = L.ssa_input(kind=SSA_MSSA, dtype=code, on_device=dev, n_series=len(lens), data=ptr,
                             lengths=lens.ctypes.data_as(C.POINTER(C.c_int64)))
        wins[i] = L.ssa_window(L=L_)
    outs = (C.c_void_p * n)()
    st = (C.c_int32 * n)()
    L.check(lib.ssa_embed_batch(ins, wins, n, _stream_ptr(stream), outs, st), "ssa_embed_batch")
    return [SSA._wrap(C.c_void_p(outs[i]), ("mssa", np.asarray(lengths[i], dtype=np.int64).copy()))
            for i in range(n)]


def embed_series_batch(xs, L_: int, stream=None):
    """Batched 1D embed of n series (numpy arrays or torch tensors, host or
    device) with one window length: ssa_embed_batch.  Returns n SSA objects."""
    lib = L.load()
    n = len(xs)
    ins = (L.ssa_input * n)()
    wins = (L.ssa_window * n)()
    keep = []
    for i, x in enumerate(xs):
        ptr, dev, kp, code = _buf(x)
        keep.append(kp)
        ins[i] = L.ssa_input(kind=SSA_1D, dtype=code, on_device=dev, n_series=1, data=ptr, n=int(x.shape[0]))
        wins[i] = L.ssa_window(L=L_)
    outs = (C.c_void_p * n)()
    st = (C.c_int32 * n)()
    L.check(lib.ssa_embed_batch(ins, wins, n, _stream_ptr(stream), outs, st), "ssa_embed_batch")
    return [SSA._wrap(C.c_void_p(outs[i]), ("1d", int(xs[i].shape[0]))) for i in range(n)]


def decompose_batch(problems, rank, prec: str = "fp32", krylov_dim: int = 0, tol: float = 0.0, seed: int = 0,
                    max_restarts: int = 0, check: bool = True):
    """Decompose many SSA objects in one batched run (lock-step Lanczos)."""
    lib = L.load()
    n = len(problems)
    ranks = rank if isinstance(rank, (list, tuple)) else [rank] * n
    arr = (C.c_void_p * n)(*[p.ctx for p in problems])
    ps = (L.ssa_params * n)(*[L.ssa_params(rank=r, krylov_dim=krylov_dim, max_restarts=max_restarts,
                                           prec=PREC[prec], tol=tol, seed=seed) for r in ranks])
    st = (C.c_int32 * n)()
    rc = lib.ssa_decompose_batch(arr, n, ps, st)
    for p, r in zip(problems, ranks):
        p.rank = r
    if check:
        L.check(rc, "ssa_decompose_batch")
    return rc, list(st)


def reconstruct_batch(problems, groups, residual: bool = False, outs=None):
    """Reconstruct many decomposed problems at once.  With ``outs`` (one CUDA
    tensor of float64 per problem, (n_groups + residual) * total elements) the
    results stay on the device and the tensors are returned; otherwise host
    arrays split per group are returned."""
    lib = L.load()
    n = len(problems)
    r = problems[0].rank
    gof = np.full(r, -1, dtype=np.int32)
    for g, idx in enumerate(groups):
        for i in idx:
            gof[i] = g
    nout = len(groups) + (1 if residual else 0)
    on_device = outs is not None
    if outs is None:
        outs = [np.zeros(p._total() * nout) for p in problems]
        ptrs = (C.c_void_p * n)(*[o.ctypes.data for o in outs])
    else:
        ptrs = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
    arr = (C.c_void_p * n)(*[p.ctx for p in problems])
    L.check(lib.ssa_reconstruct_batch(arr, n, gof.ctypes.data_as(C.POINTER(C.c_int32)), len(groups),
                                      1 if residual else 0, ptrs, 1 if on_device else 0), "ssa_reconstruct_batch")
    if on_device:
        return outs
    res = []
    for p, o in zip(problems, outs):
        t = p._total()
        res.append([p._split(o[g * t:(g + 1) * t]) for g in range(nout)])
    return res


def save_plans(path: str) -> None:
    """Write the tuned plans to a text file (ssa_plans_export)."""
    with open(path, "w") as f:
        f.write(L.plans_export())


def load_plans(path: str) -> None:
    """Read tuned plans from a text file (ssa_plans_import)."""
    with open(path) as f:
        L.plans_import(f.read())
