// Long-side Ritz vectors of the FP32 form on the 5th-generation tensor cores.
//
// After the small SVD B = P Sigma Q^T (Sec. 2.4: the role of PROPACK /
// nu-TRLan's Ritz extraction) the long basis is rotated in place:
//   V[:, 0:kk] <- V[:, 0:kc] C,   C = Q[0:kc, 0:kk] * colscale (kc = k + 1),
// a dense contraction of Kl x kc by kc x kk per problem -- the one place on the
// path where the work is a GEMM.  A tile is 128 rows of one problem's basis
// (M = 128, N = kk rounded up to 16, K = kc in chunks of 32); a CTA works
// through a few consecutive tiles:
//   1. a chunk of the rows of the basis columns and of the coefficients
//      is loaded (lane = row, coalesced along the rows) and stored into the
//      K-major core-matrix layout the MMA reads (8 rows x 16 bytes per core
//      matrix, no swizzle), one 16-byte store per core-matrix row;
//   2. each FP32 value x is split into hi = x rounded to TF32 and
//      lo = x - hi (exact); the tensor core reads lo's leading 11 bits, so
//      hi + lo carries x to about 2^-22 |x|;
//   3. one thread issues tcgen05.mma kind::tf32 for hi*hi + hi*lo + lo*hi
//      (the lo*lo term is below FP32 rounding) per K step of 8, accumulating
//      in FP32 in tensor memory (TMEM), and commits to an mbarrier;
//   4. the warps read their 32 TMEM lanes (one row each) with tcgen05.ld and
//      write the kk new columns, coalesced along the rows.
// The in-place update is safe: a tile's rows are all read before any is
// written, and only by the CTA that writes them (the loads that run ahead
// read the CTA's next tile, never rows already written).  On a restart column k (the
// residual direction) moves to column kk.
#include "lanczos.h"
#include "launch.h"
#include "tma.cuh"

#include <algorithm>
#include <atomic>

namespace ssa {

namespace {

constexpr int RTC_M = 128;          // rows per CTA = TMEM lanes
constexpr int RTC_NT = 256;         // eight warps: two per quarter of the 128 TMEM lanes
constexpr int RTC_POLL = 1 << 22;   // bounded wait on the MMA barrier

__device__ int g_ritz_tc_timeouts;
std::atomic<int> g_rtc_plan_fail{0};   // launches skipped: no scratch for the tile plan

// Operand layout: element (r, c) of an operand with kp K-columns, K-major
// core matrices, sits at byte ((r / 8) (kp / 4) + c / 4) * 128 + 16 (r % 8)
// + 4 (c % 4): core (r / 8, c / 4), row r % 8, element c % 4.

// shared-memory matrix descriptor (no swizzle): start address, leading byte
// offset (next core matrix along K), stride byte offset (next 8-row group),
// fixed 0b001 at bits 46-48
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// x rounded to the 10 explicit mantissa bits of TF32, to nearest with ties
// away from zero, by integer arithmetic on the bit pattern (adding half a TF32
// unit to the magnitude bits carries into the exponent where it should; finite
// inputs only)
__device__ __forceinline__ float tf32_hi(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// x = hi + lo with hi the TF32 rounding of x; lo = x - hi is exact in FP32,
// |lo| <= 2^-11 |x|, and the tensor core reads only its leading 11 bits,
// which leaves an error below 2^-22 |x|
__device__ __forceinline__ void tf32_split(float4 x, float4& h, float4& l) {
  h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
  l = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtm, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(dtm),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

}  // namespace

// The launch's tiles, compacted to the problems that take part (their small
// SVD is done, or the final pass), by k_ritz_tc_plan: a tile prefix over the
// taking-part problems and one record per problem.
struct RtcRec {
  float* V; const float* Cs; int64_t ldv; int64_t Kl;
  int32_t ldcs, k, kk, pad_;
};
struct RtcPlan {
  int32_t nact, total;  // taking-part problems, their tiles
  int32_t* pre;         // nact + 1 tile offsets
  RtcRec* rec;
};

// plan layout in its scratch block: the header, n + 1 tile offsets from byte
// RTC_OFF_PRE, n records from rtc_off_rec(n)
constexpr size_t RTC_OFF_PRE = 64;
__host__ __device__ inline size_t rtc_off_rec(int n) {
  return (RTC_OFF_PRE + sizeof(int32_t) * (size_t)(n + 1) + 63) & ~(size_t)63;
}

__global__ void __launch_bounds__(1024) k_ritz_tc_plan(const RitzItem<float>* __restrict__ items, int n,
                                                       int final_pass, unsigned char* scratch) {
  __shared__ int32_t wt[32], wf[32];    // per-warp tile and problem counts
  __shared__ int32_t carry[2];          // tiles, problems of the earlier 1024-item slices
  RtcPlan* pl = reinterpret_cast<RtcPlan*>(scratch);
  int32_t* const pre = reinterpret_cast<int32_t*>(scratch + RTC_OFF_PRE);
  RtcRec* const rec = reinterpret_cast<RtcRec*>(scratch + rtc_off_rec(n));
  if (threadIdx.x == 0) carry[0] = carry[1] = 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int base = 0; base < n; base += blockDim.x) {
    const int i = base + threadIdx.x;
    int cnt = 0, k = 0, kk = 0;
    if (i < n) {
      const RitzItem<float>& it = items[i];
      const LzState* st = it.st;
      if (final_pass || (st->active && st->svd_done)) {
        k = st->k;
        kk = final_pass ? min(st->r, k) : st->kk;
        if (kk > 0) cnt = (int)((it.Kl + RTC_M - 1) / RTC_M);
      }
    }
    // block exclusive scans of the tile counts and of the taking-part flags
    const int flag = cnt > 0 ? 1 : 0;
    int tinc = cnt, finc = flag;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int a = __shfl_up_sync(0xffffffffu, tinc, o), b = __shfl_up_sync(0xffffffffu, finc, o);
      if (lane >= o) { tinc += a; finc += b; }
    }
    __syncthreads();                    // carry of the earlier slices read by all
    const int c0 = carry[0], c1 = carry[1];
    if (lane == 31) { wt[warp] = tinc; wf[warp] = finc; }
    __syncthreads();
    int toff = 0, foff = 0;
    for (int w = 0; w < warp; ++w) { toff += wt[w]; foff += wf[w]; }
    const int texc = c0 + toff + tinc - cnt, fexc = c1 + foff + finc - flag;
    if (flag) {
      const RitzItem<float>& it = items[i];
      RtcRec r;
      r.V = it.V; r.Cs = it.Cs; r.ldv = it.ldv; r.Kl = it.Kl; r.ldcs = it.ldcs; r.k = k; r.kk = kk; r.pad_ = 0;
      rec[fexc] = r;
      pre[fexc] = texc;
    }
    __syncthreads();                    // everyone has its offsets before the carry moves
    if (threadIdx.x == 0) {
      int tt = 0, ff = 0;
      for (int w = 0; w < nw; ++w) { tt += wt[w]; ff += wf[w]; }
      carry[0] = c0 + tt; carry[1] = c1 + ff;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    pl->nact = carry[1];
    pl->total = carry[0];
    pl->pre = pre;
    pl->rec = rec;
    pre[carry[1]] = carry[0];
  }
}

// Each CTA takes RTC_TPC consecutive tiles of the compacted list (the
// hardware scheduler still balances CTAs between the SMs, and between this
// launch and the other engine's stream).  A tile's K = k + 1 basis columns
// come in chunks of KC = 32 (four MMA K steps); the CTA's chunks, tile after
// tile, form one sequence of units, held alternately in two register buffers.
// A unit's values go to shared memory (split into TF32 hi / lo in the
// core-matrix layout the MMA reads), and right after the MMAs are issued the
// buffer is refilled with the unit two places ahead -- so the basis loads stay
// in flight through the MMA wait and the tile's write-back, and no register
// copy waits on them.  About 40 KB of shared memory and three CTAs per SM
// (the two buffers take 32 registers a thread; at four CTAs the 64-register
// cap spilled); the contraction is memory-bound (kk of 20-60 columns per row
// read).
constexpr int RTC_KC = 32;
// (row group of 32, column group of 4) tasks of one chunk per thread
constexpr int RTC_TASKS = (RTC_M / 32) * (RTC_KC / 4) / (RTC_NT / 32);
static_assert((RTC_M / 32) * (RTC_KC / 4) % (RTC_NT / 32) == 0, "whole tasks per warp");
constexpr int RTC_CTAS_PER_SM = 3;
constexpr int RTC_TPC = 8;          // tiles per CTA

__global__ void __launch_bounds__(RTC_NT, RTC_CTAS_PER_SM) k_ritz_tc(const RtcPlan* __restrict__ plan,
                                                                    int final_pass, int np_max) {
  const int nact = plan->nact, total = plan->total;
  const int32_t* __restrict__ pre = plan->pre;
  const RtcRec* __restrict__ rec = plan->rec;
  const int t0 = (int)blockIdx.x * RTC_TPC;
  if (t0 >= total) return;
  const int t1 = min(t0 + RTC_TPC, total);
  const int ncol = np_max <= 32 ? 32 : (np_max <= 64 ? 64 : 128);   // TMEM columns (power of two >= 32)
  extern __shared__ __align__(128) unsigned char smraw[];
  float* ahi = reinterpret_cast<float*>(smraw);            // RTC_M x RTC_KC, core-matrix layout
  float* alo = ahi + RTC_M * RTC_KC;
  float* bhi = alo + RTC_M * RTC_KC;                        // np_max x RTC_KC
  float* blo = bhi + np_max * RTC_KC;
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t taddr_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&taddr_s)),
                 "r"(ncol)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) mbar_init(&bar);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = taddr_s;

  int rb0;
  const int j0 = tile_item(pre, nact, t0, rb0);
  // load cursor: the next unit to bring into registers
  int lt = t0, lch = 0, lj = j0;
  // the thread's RTC_TASKS (row, four-column group) values of the load
  // cursor's unit; the cursor moves on by one unit
  auto load_next = [&](float4 (&x)[RTC_TASKS]) {
    if (lt >= t1) return;
    const RtcRec& b = rec[lj];
    const int64_t r0 = (int64_t)(lt - pre[lj]) * RTC_M;
    const int nr = (int)imin64(RTC_M, b.Kl - r0), kc = b.k + 1;
#pragma unroll
    for (int t = 0; t < RTC_TASKS; ++t) {
      const int q = warp + t * (RTC_NT / 32);
      const int c = lch * RTC_KC + 4 * (q / (RTC_M / 32));
      const int r = (q % (RTC_M / 32)) * 32 + lane;
      x[t] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (r < nr) {
        const float* src = b.V + r0 + r + b.ldv * c;
        if (c < kc) x[t].x = src[0];
        if (c + 1 < kc) x[t].y = src[b.ldv];
        if (c + 2 < kc) x[t].z = src[2 * b.ldv];
        if (c + 3 < kc) x[t].w = src[3 * b.ldv];
      }
    }
    if (++lch * RTC_KC >= kc) {
      lch = 0;
      ++lt;
      while (lj + 1 < nact && pre[lj + 1] <= lt) ++lj;
    }
  };

  // process cursor: the unit whose values the buffer now holds
  int pt = t0, pch = 0, pj = j0;
  uint32_t commits = 0;
  auto process = [&](float4 (&x)[RTC_TASKS]) -> bool {
    const RtcRec& a = rec[pj];
    const int64_t r0 = (int64_t)(pt - pre[pj]) * RTC_M;
    const int nr = (int)imin64(RTC_M, a.Kl - r0);
    const int k = a.k, kc = k + 1, kk = a.kk;
    const int np = (kk + 15) & ~15;
    const int c0 = pch * RTC_KC;
    // 1. the unit's basis rows and coefficients, split into TF32 hi / lo,
    //    into the K-major core-matrix layout.  Lane = row: each thread holds
    //    the 16 bytes of one core-matrix row (four columns of one row; a
    //    warp's loads of a column are 128 contiguous bytes), stored with one
    //    16-byte store per part, so each group of eight lanes fills one
    //    contiguous 128-byte core matrix (no bank conflicts).
#pragma unroll
    for (int t = 0; t < RTC_TASKS; ++t) {
      const int q = warp + t * (RTC_NT / 32);
      const int g = q / (RTC_M / 32);
      const int r = (q % (RTC_M / 32)) * 32 + lane;
      float4 h, l;
      tf32_split(x[t], h, l);
      const uint32_t off = (uint32_t)((((r >> 3) * (RTC_KC / 4) + g) << 7) + ((r & 7) << 4));
      *reinterpret_cast<float4*>(smraw + off) = h;
      *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(alo) + off) = l;
    }
    for (int q = warp; q < ((np + 31) / 32) * (RTC_KC / 4); q += RTC_NT / 32) {
      const int ngs = (np + 31) / 32, g = q / ngs;
      const int nn = (q % ngs) * 32 + lane, c = c0 + 4 * g;
      if (nn < np) {
        float4 y = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        const float* src = a.Cs + (int64_t)c * a.ldcs + nn;   // zero past kk
        if (c < kc) y.x = src[0];
        if (c + 1 < kc) y.y = src[a.ldcs];
        if (c + 2 < kc) y.z = src[2 * a.ldcs];
        if (c + 3 < kc) y.w = src[3 * a.ldcs];
        float4 h, l;
        tf32_split(y, h, l);
        const uint32_t off = (uint32_t)((((nn >> 3) * (RTC_KC / 4) + g) << 7) + ((nn & 7) << 4));
        *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(bhi) + off) = h;
        *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(blo) + off) = l;
      }
    }
    // generic-proxy stores become visible to the tensor core (async proxy);
    // the previous tile's TMEM reads are ordered before these MMAs
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // 2. one thread: D (128 x np, FP32 in TMEM) += Ahi Bhi + Ahi Blo + Alo Bhi
    if (tid == 0) {
      // kind::tf32: D F32 (bits 4-5 = 1), A and B TF32 (bits 7-9, 10-12 = 2),
      // both K-major, N / 8 at bits 17-22, M / 16 at bits 24-28
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(np >> 3) << 17) |
                             ((uint32_t)(RTC_M >> 4) << 24);
      const uint32_t kstep = 2 * 128;                   // 8 K-elements = two core matrices
      const uint32_t lbo = 128, sbo = (uint32_t)(RTC_KC / 4) * 128;
      const uint32_t sa = smem_u32(ahi), sl = smem_u32(alo), sb = smem_u32(bhi), sm = smem_u32(blo);
      for (int ks = 0; ks < RTC_KC / 8; ++ks) {
        const uint32_t o = ks * kstep;
        mma_tf32(tmem, smem_desc(sa + o, lbo, sbo), smem_desc(sb + o, lbo, sbo), idesc, (pch | ks) ? 1u : 0u);
        mma_tf32(tmem, smem_desc(sa + o, lbo, sbo), smem_desc(sm + o, lbo, sbo), idesc, 1u);
        mma_tf32(tmem, smem_desc(sl + o, lbo, sbo), smem_desc(sb + o, lbo, sbo), idesc, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&bar))
                   : "memory");
    }
    // 3. the buffer is free: the unit two places ahead goes into it
    load_next(x);
    // 4. the next unit overwrites the operands: wait for these MMAs
    bool ok = mbar_wait_bounded(&bar, commits & 1u, RTC_POLL);
    ++commits;
    if (!ok && tid == 0) atomicAdd(&g_ritz_tc_timeouts, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!__syncthreads_and(ok)) return false;
    if (c0 + RTC_KC < kc) { ++pch; return true; }
    // 5. the tile is complete.  TMEM -> rows: warp w reads lanes 32 (w % 4)..
    //    (its rows), warps 0-3 the even groups of eight columns, warps 4-7
    //    the odd ones
    const int quarter = warp & 3, half = warp >> 2;
    const int row = quarter * 32 + lane;
    const int64_t ldb = a.ldv;
    float* out = a.V + r0 + row;
    for (int cb = half * 8; cb < np; cb += 16) {
      uint32_t v[8];
      const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)cb;
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                   : "r"(ta));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < nr) {
#pragma unroll
        for (int c = 0; c < 8; ++c)
          if (cb + c < kk) out[ldb * (cb + c)] = __uint_as_float(v[c]);
      }
    }
    // restart: the residual direction (column k, not written above) moves to kk
    if (!final_pass)
      for (int e = tid; e < nr; e += RTC_NT) a.V[r0 + e + ldb * kk] = a.V[r0 + e + ldb * k];
    // the next tile's first MMA overwrites the accumulator after its barrier
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    pch = 0;
    ++pt;
    while (pj + 1 < nact && pre[pj + 1] <= pt) ++pj;
    return true;
  };

  float4 xa[RTC_TASKS], xb[RTC_TASKS];
  load_next(xa);
  load_next(xb);
  while (pt < t1) {
    if (!process(xa) || pt >= t1) break;
    if (!process(xb)) break;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncol) : "memory");
}

size_t ritz_tc_smem(int kkmax) {
  const int np = (kkmax + 15) & ~15;
  return sizeof(float) * (size_t)(2 * RTC_M * RTC_KC + 2 * np * RTC_KC);
}

void launch_ritz_tc(const RitzItem<float>* items, int n, int kmax, int kkmax, const int32_t* pre, int tiles,
                    int final_pass, cudaStream_t st) {
  (void)kmax; (void)pre;
  if (n <= 0 || tiles <= 0) return;
  set_max_smem((const void*)k_ritz_tc);
  const int np = (kkmax + 15) & ~15;
  // the plan (stream-ordered scratch, written by k_ritz_tc_plan)
  unsigned char* d = nullptr;
  if (cudaMallocAsync((void**)&d, rtc_off_rec(n) + sizeof(RtcRec) * (size_t)n, st) != cudaSuccess) {
    g_rtc_plan_fail.fetch_add(1);       // reported with the timeouts
    return;
  }
  k_ritz_tc_plan<<<1, 1024, 0, st>>>(items, n, final_pass, d); count_launch();
  const int grid = (tiles + RTC_TPC - 1) / RTC_TPC;
  k_ritz_tc<<<grid, RTC_NT, ritz_tc_smem(kkmax), st>>>(reinterpret_cast<const RtcPlan*>(d), final_pass, np);
  count_launch();
  cudaFreeAsync(d, st);
}


// device address of a counter on the current device (looked up once per device)
static int* counter_word(const void* sym, int* (&cache)[64]) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  if (!cache[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, sym) != cudaSuccess) return nullptr;
    cache[dev] = static_cast<int*>(p);
  }
  return cache[dev];
}

int* ritz_tc_timeout_word() {
  static int* cache[64] = {};
  return counter_word((const void*)&g_ritz_tc_timeouts, cache);
}
int ritz_tc_plan_failures() { return g_rtc_plan_fail.exchange(0); }

int ritz_tc_timeouts(cudaStream_t st) {
  if (g_rtc_plan_fail.exchange(0) != 0) return 1;
  int h = 0, z = 0;
  if (cudaMemcpyFromSymbolAsync(&h, g_ritz_tc_timeouts, sizeof(int), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return -1;
  if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
  if (h) cudaMemcpyToSymbolAsync(g_ritz_tc_timeouts, &z, sizeof(int), 0, cudaMemcpyHostToDevice, st);
  return h;
}

}  // namespace ssa
