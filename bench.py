"""Benchmark: batched MSSA decompositions on one GB300 (or N replicas).

Workload: the MSSA configuration -- 16 float32 series of lengths U{2000..8000}
(shared periods 12 and 50, random amplitudes and phases, exp(0.0002 t) trend,
N(0, 0.2^2) noise), window L = 1000, rank r = 20.  One step is the whole hot
path over a batch of B such problems (distinct seeds): shapes and weights,
data spectra, Lanczos decomposition, reconstruction of the groups {1}, {2,3},
{4,5} plus the residual.

  value  decompositions/s with the series already resident in HBM (device
         pointers through the C ABI; reconstructions written to HBM);
  e2e    the same through the C ABI from pinned host buffers, the host->device
         copies of the series and the device->host copy of the results inside
         the timed region.
Between timed steps L2 is flushed by writing a 512 MiB buffer.

--impl reference times the CPU FP64 oracle (explicit trajectory matrix,
S = X X^T eigendecomposition, direct diagonal averaging) on the same problems.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

WORKLOAD = "mssa_16x2000-8000_L1000"
CFG = W.CONFIGS[WORKLOAD]
GROUPS = [[0], [1, 2], [3, 4]]
METRIC = "ssa_decomps_per_s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def problem_series(seed):
    return W.mssa_series(CFG["s"], seed=seed)


def problem_seed(rank, i):
    """Seed of problem i on a rank: every replica draws its own problems."""
    return 2 + rank * 100003 + i


def max_over_ranks(ms, dist, device):
    """The slowest rank's time -- the job ends with it; unchanged on one process."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ oracle arm
def run_oracle(n_problems, base_seed):
    from oracle import ssa_oracle as O
    t0 = time.perf_counter()
    for i in range(n_problems):
        xs = problem_series(base_seed + i)
        P = O.Problem.multi([np.asarray(x, np.float64) for x in xs], CFG["L"])
        s, U, V = O.decompose(P, CFG["rank"])
        O.reconstruct(P, s, U, V, GROUPS, residual=True)
    return time.perf_counter() - t0


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(budget_s=12.0):
    """Time the oracle on as many problems as fit in about budget_s."""
    n, total = 0, 0.0
    while total < budget_s and n < 8:
        total += run_oracle(1, 1000 + n)
        n += 1
    return {"value": n / total, "unit": "decomps/s", "cores": cpu_cores(), "kind": "oracle",
            "sample": f"{n} MSSA problems (16 series, L=1000, r=20) through the FP64 oracle, "
                      f"{total:.1f} s"}


# ------------------------------------------------------------------ clocks
class Clocks:
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        rows = []
        for line in (getattr(self, "out", "") or "").splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 6:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[2 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ GPU arm
# ------------------------------------------------------------------ serving
SERVE_N_MAX = 200000  # longest series of the serving mix


def serve_submit(srv, q, seed):
    g = [[0], [1, 2]]
    if q.kind == "1d":
        return srv.submit_series(q.data, q.L, q.rank, groups=g, residual=True, seed=seed)
    if q.kind == "mssa":
        return srv.submit_multi(q.data, q.L, q.rank, groups=g, residual=True, seed=seed)
    return srv.submit_image(q.data, q.window[0], q.window[1], q.rank, mask=q.mask, groups=g, residual=True,
                            seed=seed)


def serve_at_spec(pkg, n_sat, n_open, prec, budget, seed, load=0.8):
    """Config 5 as specified: first the saturating throughput C, closed loop
    (n_sat requests all queued at once, completions per second of wall time),
    then an open-loop Poisson stream of n_open further requests at
    load * C (arrival times of the generator's stream rescaled to that rate),
    whose p50 / p99 are service latencies (arrival to result in host memory)."""
    import dataclasses
    reqs = W.serving_requests(n=n_sat + n_open, rate_hz=1000.0, seed=seed, n_max=SERVE_N_MAX)
    sat = run_serving(pkg, reqs[:n_sat], prec, budget, None)
    lam = load * sat["throughput_rps"]
    rest = reqs[n_sat:]
    t0 = rest[0].arrival_s
    scaled = [dataclasses.replace(q, arrival_s=(q.arrival_s - t0) * 1000.0 / lam) for q in rest]
    opn = run_serving(pkg, scaled, prec, budget, lam)
    return {"saturation": sat, "poisson": opn, "load": load,
            "what": "closed-loop capacity, then Poisson arrivals at load x capacity; latencies of the Poisson part"}


def run_serving(pkg, reqs, prec, budget, rate_hz):
    """Open-loop serving: each request is submitted when its Poisson arrival
    time comes up on the server's clock; latency runs from that arrival time
    to the request's completion (results in host memory).  rate_hz None:
    closed loop, every request queued at the start (arrival = start)."""
    if rate_hz is None:
        import dataclasses
        reqs = [dataclasses.replace(q, arrival_s=0.0) for q in reqs]
    from paper_1309_5050_gb300 import _lib
    srv = pkg.Server(memory_budget=budget, prec=prec)
    for q in reqs[:8]:                      # warm-up requests (not counted)
        serve_submit(srv, q, 1)
    srv.drain()
    for t in srv.finished():
        srv.take(t)
    _lib.profile_reset()
    _lib.profile_enable(True)
    l0 = _lib.kernel_launches()
    n = len(reqs)
    arrival = {}
    lat, status, restarts = [], {}, []
    max_live = max_q = 0
    i = 0
    t0 = srv.clock()
    t_last = t0
    steps = 0
    step_s = []
    while len(lat) < n:
        now = srv.clock() - t0
        while i < n and reqs[i].arrival_s <= now:
            arrival[serve_submit(srv, reqs[i], 1000 + i)] = reqs[i].arrival_s
            i += 1
        st = srv.stats()
        max_live = max(max_live, st["live"])
        max_q = max(max_q, st["queued"])
        if st["queued"] == 0 and st["live"] == 0:
            if i < n:
                dt = reqs[i].arrival_s - (srv.clock() - t0)
                if dt > 0:
                    time.sleep(dt)
            continue
        ts0 = time.perf_counter()
        srv.step()
        step_s.append(time.perf_counter() - ts0)
        steps += 1
        for t in srv.finished():
            r = srv.take(t)
            lat.append(r["t_done"] - t0 - arrival.pop(t))
            status[r["status"]] = status.get(r["status"], 0) + 1
            restarts.append(r["restarts"])
            t_last = max(t_last, r["t_done"])
    srv.close()
    launches = _lib.kernel_launches() - l0
    prof = _lib.profile_read()
    _lib.profile_enable(False)
    wall = t_last - t0
    kinds = {}
    for q in reqs:
        kinds[q.kind] = kinds.get(q.kind, 0) + 1
    return {"requests": n, "rate_hz": rate_hz if rate_hz is not None else "closed loop", "kinds": kinds,
            "throughput_rps": n / wall, "wall_s": wall,
            "p50_ms": 1000 * float(np.percentile(lat, 50)), "p99_ms": 1000 * float(np.percentile(lat, 99)),
            "mean_ms": 1000 * float(np.mean(lat)), "max_live": max_live, "max_queued": max_q,
            "server_steps": steps, "step_ms_mean": 1000 * float(np.mean(step_s)),
            "step_ms_max": 1000 * float(np.max(step_s)), "mean_restarts": float(np.mean(restarts)),
            "statuses": {str(k): v for k, v in status.items()}, "budget_bytes": budget,
            "series_n_max": SERVE_N_MAX, "prec": prec, "gpu_launches": int(launches),
            "phases_ms": {k: v[0] for k, v in prof.items()}}


def mv1d_algorithmic(probs):
    """Algorithmic bytes of one k_mv1d launch over the batch, per direction,
    and its FFT flops (average of the two).  Per problem and channel q with
    grid M_q = next power of two >= N_q (>= 16), H_q = M_q / 2:
      X v   : v slice (K_q fp32) + spectrum ((H_q+1) complex fp32) + partial u (L fp32)
      X^T u : u (L fp64) + spectrum + v_j slice (K_q fp32) + q slice (K_q fp32)
    (the X^T u launch carries the fused long-side step).  Flops: two packed
    real FFTs of M_q points, 5 H log2 H each, per channel."""
    L = CFG["L"]
    ba = bt = fl = 0.0
    for lens, _ in probs:
        for n in lens:
            M = 16
            while M < n:
                M *= 2
            H = M // 2
            K = int(n) - L + 1
            spec = (H + 1) * 8
            ba += K * 4 + spec + L * 4
            bt += L * 8 + spec + 2 * K * 4
            fl += 2 * 5 * H * np.log2(H)
    return {"bytes_A": ba, "bytes_AT": bt, "flops": fl}


def mv1d_traffic(batch):
    """DRAM bytes per k_mv1d launch (average of the two directions) from the
    committed ncu summary, when it was taken on this batch size and the
    kernel's sources are unchanged since; else None."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "k_mv1d_mssa_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None, "no committed capture"
    if d.get("sources") != MV1D_SOURCES:
        return None, "capture keyed to other sources"
    h = hashlib.sha256()
    for rel in MV1D_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    if h.hexdigest() != d.get("sources_sha256"):
        return None, "kernel sources changed since the capture"
    if int(d.get("batch", -1)) != int(batch):
        return None, f"capture taken at batch {d.get('batch')}"
    return float(d["dram_bytes_per_launch"]), "profiles/k_mv1d_mssa_traffic.json"


MV1D_SOURCES = ["paper_1309_5050_gb300/csrc/k_matvec.cu", "paper_1309_5050_gb300/csrc/fft_block.cuh",
                "paper_1309_5050_gb300/csrc/tma.cuh", "paper_1309_5050_gb300/csrc/common.cuh"]
DECOMP_SPLIT_MIN = 64   # mirrors the library's split of large batches into two streams


def write_traffic(csv_path, batch, command):
    """Summarise an ncu launch capture of k_mv1d (metrics dram__bytes_read.sum,
    dram__bytes_write.sum) into profiles/k_mv1d_mssa_traffic.json, keyed by
    the kernel's source hash so a later change voids it."""
    import csv
    import hashlib
    rows = list(csv.reader(open(csv_path)))
    hdr = [r for r in rows if r and r[0] == "ID"][0]
    per = {}
    for r in rows:
        if not r or r[0] == "ID" or len(r) != len(hdr):
            continue
        d = dict(zip(hdr, r))
        if "k_mv1d" not in d["Kernel Name"]:
            continue
        v = float(d["Metric Value"].replace(",", ""))
        scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "ns": 1, "nsecond": 1,
                 "usecond": 1e3, "us": 1e3, "msecond": 1e6, "ms": 1e6}.get(d["Metric Unit"], 1)
        e = per.setdefault(d["ID"], {"kernel": d["Kernel Name"].split("(")[0]})
        e[d["Metric Name"]] = v * scale
    launches = [e for e in per.values() if "dram__bytes_read.sum" in e]
    tot = [e["dram__bytes_read.sum"] + e.get("dram__bytes_write.sum", 0.0) for e in launches]
    h = hashlib.sha256()
    for rel in MV1D_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    out = {"kernel": "k_mv1d", "workload": WORKLOAD, "batch": batch, "command": command,
           "launches": [{"kernel": e["kernel"], "dram_bytes": t, "ns": e.get("gpu__time_duration.sum")}
                        for e, t in zip(launches, tot)],
           "dram_bytes_per_launch": sum(tot) / max(len(tot), 1),
           "sources": MV1D_SOURCES, "sources_sha256": h.hexdigest()}
    with open(os.path.join(ROOT, "profiles", "k_mv1d_mssa_traffic.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


# ------------------------------------------------------------------ configs 1, 3, 4
# The other workloads of the method, each timed as its own step (shapes and
# weights, spectra, decomposition, reconstruction of the signal groups plus
# the residual) in both precision forms.  The series workload is latency-bound
# alone, so B distinct series (seeds seed, seed + 1, ...) run per step, as the
# MSSA headline does; an image is one problem per step.
CONFIG_RUNS = {
    "series_1d_n1000": {"batch": 456, "groups": [[0, 1], [2, 3]]},
    "image_1024x1024_w64": {"batch": 1, "groups": [list(range(8)), list(range(8, 12)), list(range(12, 16))]},
    "shaped_2048x2048_disc40holes_w32": {"batch": 1,
                                         "groups": [[0], list(range(1, 9)), list(range(9, 13)), list(range(13, 17))]},
}


def config_input(name, i):
    """Host data of problem i of a workload (i = 0: the workload's own seed)."""
    cfg = W.CONFIGS[name]
    seed = cfg["seed"] + i
    if cfg["kind"] == "1d":
        return W.series_1d(cfg["n"], seed=seed)
    if cfg["kind"] == "2d":
        return W.harmonic_image(cfg["nx"], cfg["ny"], seed=seed)
    x, _, _ = W.shaped_image(cfg["nx"], cfg["ny"], seed=seed)
    return x


def pow2_at_least(n, lo=16):
    m = lo
    while m < n:
        m *= 2
    return m


def product_algorithmic_bytes(name, prec, K):
    """Floor bytes of one trajectory product (average of X v and X^T u) of one
    problem: the input vector, the data's half spectrum and the output vector,
    each read or written once.  X v reads v (K) and writes u (L); X^T u reads
    the FP64 window-side vector u (L) and writes v (K) -- for a series, whose
    long-side Lanczos step is fused into that store, also reading v_j (K)."""
    cfg = W.CONFIGS[name]
    t = 4 if prec == "fp32" else 8
    if cfg["kind"] == "1d":
        H = pow2_at_least(cfg["n"]) // 2
        spec, L = (H + 1) * 2 * t, cfg["L"]
        a = K * t + spec + L * t
        at = L * 8 + spec + 2 * K * t
    else:
        mx, my = pow2_at_least(cfg["nx"]), pow2_at_least(cfg["ny"], 1)
        spec, L = (mx // 2 + 1) * my * 2 * t, cfg["lx"] * cfg["ly"]
        a = K * t + spec + L * t
        at = L * 8 + spec + K * t
    return (a + at) / 2.0


def run_config(pkg, torch, name, prec, stream, flush, steps, warmup):
    """decompositions/s of one workload in one precision form, with the phase
    profile and the roofline of the trajectory product."""
    from paper_1309_5050_gb300 import _lib
    cfg = W.CONFIGS[name]
    run = CONFIG_RUNS[name]
    B, groups = run["batch"], run["groups"]
    hosts = [config_input(name, i) for i in range(B)]
    if cfg["kind"] == "1d":
        dev = [torch.from_numpy(np.ascontiguousarray(h, np.float64)).cuda() for h in hosts]
    else:
        # column-major bytes: a (ny, nx) row-major tensor viewed transposed
        dev = [torch.from_numpy(np.ascontiguousarray(h.T, np.float32)).cuda() for h in hosts]
    total = hosts[0].size
    nout = len(groups) + 1
    outs = [torch.empty(total * nout, dtype=torch.float64, device="cuda") for _ in range(B)]
    info = {}

    def step():
        if cfg["kind"] == "1d":
            ps = pkg.embed_series_batch(dev, cfg["L"], stream=stream)
        else:
            ps = [pkg.SSA.image(d.t(), cfg["lx"], cfg["ly"], stream=stream) for d in dev]
        pkg.decompose_batch(ps, cfg["rank"], prec)
        if not info:
            info.update(ps[0].info())
        pkg.reconstruct_batch(ps, groups, residual=True, outs=outs)
        for p in ps:
            p.close()

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    _lib.profile_reset()
    _lib.profile_enable(True)
    l0 = _lib.kernel_launches()
    ts = []
    for _ in range(steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    launches = _lib.kernel_launches() - l0
    prof = _lib.profile_read()
    _lib.profile_enable(False)
    ms = sum(ts) / len(ts)
    mv_ms, _, mv_calls = prof["matvec"]
    engines = 2 if B >= DECOMP_SPLIT_MIN else 1
    per_call = product_algorithmic_bytes(name, prec, int(info["K"])) * B / engines
    mv_avg = mv_ms / max(mv_calls, 1)
    hbm, src = peaks()
    achieved = per_call / (mv_avg / 1000.0) / 1e9
    kernel = "k_mv1d" if cfg["kind"] == "1d" else "k_mv_xfwd + k_ypass + k_mv_xinv"
    return {"decomps_per_s": B / (ms / 1000.0), "ms_per_step": ms, "batch": B, "steps": steps,
            "ms_p50": float(np.percentile(ts, 50)), "ms_max": float(np.max(ts)),
            "krylov_dim": info.get("krylov_dim"), "restarts": info.get("restarts"),
            "gpu_launches_per_step": launches / steps,
            "phases_ms_per_step": {k: v[0] / steps for k, v in prof.items()},
            "product": {"kernels": kernel, "bound": "hbm", "algorithmic_bytes_per_call": per_call,
                        "ms_per_call": mv_avg, "achieved": achieved, "unit": "GB/s", "peak": hbm,
                        "frac": achieved / hbm, "peak_source": f"{src} (MEASURED_PEAKS hbm_gbs)",
                        "calls_timed": mv_calls,
                        "what": "one call = every problem's product in one direction (one engine's launch set)"}}


def tuned_config(pkg, torch, name, prec, stream, flush, steps, warmup):
    """run_config with the fixed plan, then ssa_autotune on one problem of the
    workload (Krylov dimension; y-pass tile width for images), then
    run_config again when the chosen plan differs: the plan table is keyed by
    size class, so the batched decompositions of the second run use it."""
    cfg = W.CONFIGS[name]
    base = run_config(pkg, torch, name, prec, stream, flush, steps, warmup)
    h = config_input(name, 0)
    if cfg["kind"] == "1d":
        d = torch.from_numpy(np.ascontiguousarray(h, np.float64)).cuda()
        p = pkg.embed_series_batch([d], cfg["L"], stream=stream)[0]
    else:
        d = torch.from_numpy(np.ascontiguousarray(h.T, np.float32)).cuda()
        p = pkg.SSA.image(d.t(), cfg["lx"], cfg["ly"], stream=stream)
    t = p.autotune(cfg["rank"], prec)
    p.close()
    plan = {"krylov_dim": t["krylov_dim"], "ytk": t["ytk"] or None, "candidates_timed": t["n_tried"],
            "one_problem_ms_fixed_plan": t["ms_default"], "one_problem_ms_chosen": t["ms_best"],
            "fixed_krylov_dim": base["krylov_dim"]}
    if t["ms_best"] >= t["ms_default"]:
        base["plan"] = dict(plan, applied=False, gain=1.0)
        return base
    tuned = run_config(pkg, torch, name, prec, stream, flush, steps, warmup)
    tuned["plan"] = dict(plan, applied=True, decomps_per_s_fixed_plan=base["decomps_per_s"],
                         gain=tuned["decomps_per_s"] / base["decomps_per_s"])
    return tuned


def oracle_sample(name, budget_s):
    """The CPU oracle on a bounded sample of one workload, in this process
    (the caller sets the BLAS thread count through the environment)."""
    from oracle import ssa_oracle as O
    cfg = W.CONFIGS[name]
    if cfg["kind"] == "mssa":
        n, total = 0, 0.0
        while total < budget_s and n < 8:
            total += run_oracle(1, 1000 + n)
            n += 1
        return {"value": n / total, "sample": f"{n} full problems (decomposition + reconstruction), {total:.1f} s"}
    if cfg["kind"] == "1d":
        groups = CONFIG_RUNS[name]["groups"]
        n, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < budget_s and n < 200:
            x = config_input(name, n)
            P = O.Problem.series(x, cfg["L"])
            sg, U, V = O.decompose(P, cfg["rank"])
            O.reconstruct(P, sg, U, V, groups, residual=True)
            n += 1
        total = time.perf_counter() - t0
        return {"value": n / total, "sample": f"{n} full problems (decomposition + reconstruction), {total:.1f} s"}
    # images: Step 2 as the oracle runs it (S = X X^T over column blocks, eigh,
    # V = X^T U / sigma) on the first column blocks, scaled to all of them;
    # the explicit reconstruction (an L x K matrix per group, 15-16 GB) is left out
    x = config_input(name, 0)
    P = O.Problem.image(x, cfg["lx"], cfg["ly"])
    nblk = sum(1 for _ in range(0, P.K, 4096))
    S = np.zeros((P.L, P.L))
    t0 = time.perf_counter()
    done = 0
    blocks = []
    for _, Xb in P.column_blocks():
        S += Xb @ Xb.T
        blocks.append(Xb)
        done += 1
        if time.perf_counter() - t0 > budget_s / 2:
            break
    t_s = time.perf_counter() - t0
    t1 = time.perf_counter()
    lam, U = np.linalg.eigh(S)
    U = U[:, ::-1][:, :cfg["rank"]]
    t_e = time.perf_counter() - t1
    t2 = time.perf_counter()
    for Xb in blocks:
        Xb.T @ U
    t_v = time.perf_counter() - t2
    est = (t_s + t_v) * nblk / done + t_e
    return {"value": 1.0 / est, "extrapolated_s": est,
            "sample": f"decomposition only: S = X X^T and V = X^T U on {done} of {nblk} column blocks "
                      f"({time.perf_counter() - t0:.1f} s), scaled to all blocks, plus eigh of S; the explicit "
                      f"reconstruction (L x K per group) does not fit the host and is left out"}


def oracle_baselines(names, budget_s):
    """Each workload's oracle sample on all host cores and on one thread, each
    in a fresh interpreter (the BLAS thread count is fixed at start-up)."""
    out = {}
    for name in names:
        out[name] = {}
        for label, threads in (("all_cores", None), ("one_thread", 1)):
            env = dict(os.environ)
            if threads:
                for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
                    env[v] = str(threads)
            r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", name,
                                "--oracle-budget", str(budget_s)], env=env, capture_output=True, text=True)
            try:
                d = json.loads(r.stdout.strip().splitlines()[-1])
            except Exception:
                d = {"error": (r.stderr or r.stdout)[-300:]}
            d.update({"unit": "decomps/s", "cores": threads or cpu_cores(), "kind": "oracle"})
            out[name][label] = d
    return out


def _probe_info(pkg, probs, cfg, stream, args):
    """Krylov dimension the library uses for one problem of the workload."""
    lens, flat = probs[0]
    p = pkg.SSA.multi_concat(flat, lens, cfg["L"], stream=stream)
    p.decompose(cfg["rank"], args.prec, krylov_dim=args.krylov_dim)
    info = p.info()
    # w-correlation matrix of the elementary components (Sec. 2.2): one call
    # reconstructs the r components and sums their weighted Gram matrix
    p.wcor()
    t0 = time.perf_counter()
    reps = 5
    for _ in range(reps):
        p.wcor()
    info["wcor_ms"] = (time.perf_counter() - t0) * 1000.0 / reps
    p.close()
    return info


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=456)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-fp64-form", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--krylov-dim", type=int, default=0, help="0: the library default min(2r+16, 112, min(L,K))")
    ap.add_argument("--serve-requests", type=int, default=2000, help="requests of the Poisson part")
    ap.add_argument("--serve-saturation", type=int, default=1000, help="requests of the closed-loop part")
    ap.add_argument("--serve-load", type=float, default=0.8, help="Poisson rate as a fraction of capacity")
    ap.add_argument("--serve-rate", type=float, default=1000.0, help="--serve-only: open-loop rate (0: closed)")
    ap.add_argument("--serve-budget-gb", type=float, default=40.0)
    ap.add_argument("--serve-only", action="store_true", help="run only the serving stream")
    ap.add_argument("--write-traffic", default=None,
                    help="ncu CSV of k_mv1d dram bytes -> profiles/k_mv1d_mssa_traffic.json (no GPU use)")
    ap.add_argument("--traffic-command", default="")
    ap.add_argument("--configs", default=",".join(CONFIG_RUNS),
                    help="other workloads timed after the headline (comma list; empty: none)")
    ap.add_argument("--config-steps", type=int, default=5)
    ap.add_argument("--oracle-budget", type=float, default=6.0, help="seconds of oracle work per sample")
    ap.add_argument("--oracle-sample", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--configs-only", action="store_true",
                    help="time only the --configs workloads (profiling runs); no headline line")
    ap.add_argument("--config-precs", default="fp32,fp64")
    args = ap.parse_args()
    if args.write_traffic:
        write_traffic(args.write_traffic, args.batch, args.traffic_command)
        return 0
    if args.oracle_sample:
        print(json.dumps(oracle_sample(args.oracle_sample, args.oracle_budget)), flush=True)
        return 0
    configs = [c for c in args.configs.split(",") if c]

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return 0
        for _ in range(args.warmup):
            run_oracle(1, 5000)
        times = [run_oracle(1, 6000 + i) for i in range(args.steps)]
        tot = sum(times)
        value = args.steps / tot
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "decomps/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1000 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "batch": 1, "series": 16, "L": 1000, "rank": 20,
                           "l2": "n/a (host)"},
                "cpu_baseline": {"value": value, "unit": "decomps/s", "cores": cpu_cores(), "kind": "oracle",
                                 "sample": f"{args.steps} MSSA problems, one per step"},
                "e2e": {"value": value, "unit": "decomps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0

    import torch
    import paper_1309_5050_gb300 as pkg
    from paper_1309_5050_gb300 import _lib

    # a process pool is never used; the oracle legs run before CUDA work (in
    # process, and in fresh interpreters for the per-workload samples)
    cpu = None
    oracles = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline()
        oracles = oracle_baselines(configs + [WORKLOAD], args.oracle_budget)

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    pkg.load()
    if args.configs_only:
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        out = {}
        for name in configs:
            out[name] = {pr: tuned_config(pkg, torch, name, pr, stream, flush, args.config_steps, args.warmup)
                         for pr in args.config_precs.split(",")}
        if rank == 0:
            print(json.dumps({"configs": out}), flush=True)
        return 0
    if args.serve_only:
        # only the serving stream (profiling and latency studies)
        with Clocks(local) as ck:
            if args.serve_rate > 0:
                reqs = W.serving_requests(n=args.serve_requests, rate_hz=args.serve_rate, seed=5 + rank,
                                          n_max=SERVE_N_MAX)
                serving = run_serving(pkg, reqs, args.prec, int(args.serve_budget_gb * (1 << 30)), args.serve_rate)
                value = serving["throughput_rps"]
            else:
                serving = serve_at_spec(pkg, args.serve_saturation, args.serve_requests, args.prec,
                                        int(args.serve_budget_gb * (1 << 30)), 5 + rank, args.serve_load)
                value = serving["saturation"]["throughput_rps"]
        if rank == 0:
            print(json.dumps({"metric": "serving_requests_per_s", "value": value, "unit": "req/s",
                              "higher_is_better": True, "serving": serving, "clocks": ck.summary(),
                              "data": "synthetic"}), flush=True)
        return 0
    B = args.batch

    # inputs: B problems per rank, distinct seeds per rank
    probs = []
    for i in range(B):
        xs = problem_series(problem_seed(rank, i))
        lens = np.array([len(x) for x in xs], dtype=np.int64)
        flat = np.concatenate(xs).astype(np.float32)
        probs.append((lens, flat))
    dev_inputs = [torch.from_numpy(f).to(dev) for _, f in probs]
    host_inputs = [torch.from_numpy(f).pin_memory() for _, f in probs]
    nout = len(GROUPS) + 1
    dev_outs = [torch.empty(int(l.sum()) * nout, dtype=torch.float64, device=dev) for l, _ in probs]
    host_outs = [torch.empty(int(l.sum()) * nout, dtype=torch.float64).pin_memory() for l, _ in probs]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    restarts = []

    def step(inputs, outs, prec):
        ps = pkg.embed_multi_batch(inputs, [l for l, _ in probs], CFG["L"], stream=stream)
        pkg.decompose_batch(ps, CFG["rank"], prec, krylov_dim=args.krylov_dim)
        inf0 = ps[0].info()
        restarts.append((inf0["restarts"], inf0["jacobi_sweeps"], inf0["jacobi_sweeps_fp32"]))
        if outs[0].is_cuda:
            pkg.reconstruct_batch(ps, GROUPS, residual=True, outs=outs)
        else:
            # results through device buffers, then one read back per problem
            pkg.reconstruct_batch(ps, GROUPS, residual=True, outs=dev_outs)
            for d, h in zip(dev_outs, outs):
                h.copy_(d, non_blocking=True)
        for p in ps:
            p.close()

    def timed(nsteps, inputs, outs, prec, profile=False):
        ts = []
        for _ in range(nsteps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(inputs, outs, prec)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return ts

    # warm-up
    for _ in range(args.warmup):
        step(dev_inputs, dev_outs, args.prec)
    torch.cuda.synchronize()

    # timed region (device-resident inputs), with phase profiling and clocks
    _lib.profile_reset()
    _lib.profile_enable(True)
    l0 = _lib.kernel_launches()
    with Clocks(local) as ck:
        ts = timed(args.steps, dev_inputs, dev_outs, args.prec)
    launches = _lib.kernel_launches() - l0
    prof = _lib.profile_read()
    _lib.profile_enable(False)
    clocks = ck.summary()

    ps_info = _probe_info(pkg, probs, CFG, stream, args)
    ms = max_over_ranks(sum(ts) / len(ts), dist, dev)
    value = world * B / (ms / 1000.0)

    # end to end from pinned host memory (one untimed step first, as for the device path)
    step(host_inputs, host_outs, args.prec)
    torch.cuda.synchronize()
    ts_e2e = timed(max(2, args.steps), host_inputs, host_outs, args.prec)
    ms_e2e = max_over_ranks(sum(ts_e2e) / len(ts_e2e), dist, dev)
    h2d = int(sum(f.nbytes for _, f in probs))
    d2h = int(sum(o.numel() * 8 for o in host_outs))

    # FP64 form on the same problems (fewer steps)
    fp64 = None
    if not args.no_fp64_form and args.prec == "fp32":
        step(dev_inputs, dev_outs, "fp64")
        t64 = timed(max(1, args.steps // 3), dev_inputs, dev_outs, "fp64")
        ms64 = max_over_ranks(sum(t64) / len(t64), dist, dev)
        fp64 = {"value": world * B / (ms64 / 1000.0), "unit": "decomps/s", "ms_per_step": ms64}

    # serving: a Poisson stream of mixed requests through ssa_server_*
    serving = None
    if args.serve_requests > 0:
        serving = serve_at_spec(pkg, args.serve_saturation, args.serve_requests, args.prec,
                                int(args.serve_budget_gb * (1 << 30)), 5 + rank, args.serve_load)

    # the other workloads, both forms
    per_config = {}
    for name in configs:
        per_config[name] = {}
        for pr in args.config_precs.split(","):
            per_config[name][pr] = tuned_config(pkg, torch, name, pr, stream, flush, args.config_steps, 3)
        if oracles:
            per_config[name]["oracle"] = oracles.get(name)
    if oracles:
        per_config.setdefault(WORKLOAD, {})["oracle"] = oracles.get(WORKLOAD)

    # roofline of the series product (k_mv1d), the dominant kernel
    hbm, src = peaks()
    total_ms = sum(v[0] for v in prof.values())
    dom = max(prof, key=lambda k: prof[k][0])
    mv_ms, mv_launch, mv_calls = prof["matvec"]
    alg = mv1d_algorithmic(probs)
    mv_avg_ms = mv_ms / max(mv_calls, 1)          # one phase instance = one k_mv1d launch
    # the library runs batches of DECOMP_SPLIT_MIN or more problems as two
    # interleaved halves on two streams: one launch covers half the batch
    groups = 2 if B >= DECOMP_SPLIT_MIN else 1
    per_call = (alg["bytes_A"] + alg["bytes_AT"]) / 2.0 / groups
    achieved = per_call / (mv_avg_ms / 1000.0) / 1e9
    flops = alg["flops"] / groups / (mv_avg_ms / 1000.0) / 1e12
    alu_peak = 152 * 128 * 2 * 2.07e9 / 1e12      # FP32 FMA lanes x 2 flops x max SM clock
    traffic, traffic_src = mv1d_traffic(B)
    roof = {"kernel": "k_mv1d (fused FFT trajectory product, both directions)", "bound": "hbm",
            "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": traffic, "traffic_source": traffic_src, "peak_source": f"{src} (MEASURED_PEAKS hbm_gbs)",
            "algorithmic_bytes_per_launch": per_call, "launches_timed": mv_calls,
            "streams": groups,
            "alu": {"achieved": flops, "peak": alu_peak, "unit": "TFLOP/s", "frac": flops / alu_peak,
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"},
            "phase_share": {k: (v[0] / total_ms if total_ms else 0.0) for k, v in prof.items()},
            "dominant_phase": dom}

    if rank == 0:
        ts_sorted = sorted(ts)
        line = {"metric": METRIC, "value": value, "unit": "decomps/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if args.prec == "fp32" else "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "batch_per_gpu": B, "series": 16, "series_len": [2000, 8000],
                           "L": CFG["L"], "rank": CFG["rank"], "groups": GROUPS, "residual": True,
                           "precision_form": "fp32 FFT + fp64 reorth" if args.prec == "fp32" else "fp64",
                           "l2": "flushed (512 MiB write) between timed steps", "parallelism": f"replicas x{world}"},
                "latency_ms": {"p50": float(np.percentile(ts_sorted, 50)), "p99": float(np.percentile(ts_sorted, 99)),
                               "what": "completion of one batch"},
                "fp64_form": fp64,
                "serving": serving,
                "roofline": roof,
                "cpu_baseline": cpu,
                "e2e": {"value": world * B / (ms_e2e / 1000.0), "unit": "decomps/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e},
                "gpu_launches": int(launches),
                "wcor": {"ms_per_call": ps_info["wcor_ms"], "components": CFG["rank"],
                         "what": "ssa_wcor, elementary w-correlations of one problem, host call"},
                "lanczos": {"krylov_dim": ps_info["krylov_dim"], "restarts_first_problem": restarts[-1][0],
                            "last_jacobi_sweeps_first_problem": {"fp64": restarts[-1][1], "fp32": restarts[-1][2]}},
                "phases_ms": {k: v[0] / args.steps for k, v in prof.items()},
                "configs": per_config,
                "clocks": clocks}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
