// Long-side Ritz vectors of the FP32 form on the 5th-generation tensor cores.
//
// After the small SVD B = P Sigma Q^T (Sec. 2.4: the role of PROPACK /
// nu-TRLan's Ritz extraction) the long basis is rotated in place:
//   V[:, 0:kk] <- V[:, 0:kc] C,   C = Q[0:kc, 0:kk] * colscale (kc = k + 1),
// a dense contraction of Kl x kc by kc x kk per problem -- the one place on the
// path where the work is a GEMM.  Each CTA owns 128 rows of one problem's
// basis (M = 128, N = kk rounded up to 16, K = kc in chunks of 32):
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
// written, and only by the CTA that writes them.  On a restart column k (the
// residual direction) moves to column kk.
#include "lanczos.h"
#include "launch.h"
#include "tma.cuh"

namespace ssa {

namespace {

constexpr int RTC_M = 128;          // rows per CTA = TMEM lanes
constexpr int RTC_NT = 256;         // eight warps: two per quarter of the 128 TMEM lanes
constexpr int RTC_POLL = 1 << 22;   // bounded wait on the MMA barrier

__device__ int g_ritz_tc_timeouts;

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

// One CTA per 128-row tile.  K is taken in chunks of KC = 32 (four MMA K
// steps), so a CTA holds one chunk of the rows (hi in place of the raw
// values, lo beside it) and of the coefficients: about 40 KB of shared
// memory, and several CTAs per SM keep enough rows in flight -- the
// contraction is memory-bound (kk of 20-60 columns per row read).
constexpr int RTC_KC = 32;
// (row group of 32, column group of 4) tasks of one chunk per thread
constexpr int RTC_TASKS = (RTC_M / 32) * (RTC_KC / 4) / (RTC_NT / 32);
static_assert((RTC_M / 32) * (RTC_KC / 4) % (RTC_NT / 32) == 0, "whole tasks per warp");

__global__ void __launch_bounds__(RTC_NT, 4) k_ritz_tc(const RitzItem<float>* __restrict__ items,
                                                  const int32_t* __restrict__ tpre, int n, int final_pass, int np_max) {
  int rblk;
  const RitzItem<float> it = items[tile_item(tpre, n, blockIdx.x, rblk)];
  const LzState* st = it.st;
  if (!final_pass && (!st->active || !st->svd_done)) return;
  const int k = st->k;
  const int kk = final_pass ? min(st->r, k) : st->kk;
  const int64_t r0 = (int64_t)rblk * RTC_M;
  if (r0 >= it.Kl || kk <= 0) return;
  const int nr = (int)imin64(RTC_M, it.Kl - r0);
  const int kc = k + 1;
  const int nchunk = (kc + RTC_KC - 1) / RTC_KC;
  const int np = (kk + 15) & ~15;
  const int ncol = np_max <= 32 ? 32 : (np_max <= 64 ? 64 : 128);   // TMEM columns (power of two >= 32)
  extern __shared__ __align__(128) unsigned char smraw[];
  float* ahi = reinterpret_cast<float*>(smraw);            // RTC_M x RTC_KC, core-matrix layout
  float* alo = ahi + RTC_M * RTC_KC;
  float* bhi = alo + RTC_M * RTC_KC;                        // np_max x RTC_KC
  float* blo = bhi + np_max * RTC_KC;
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t taddr_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float* basis = it.V;
  const int64_t ldb = it.ldv;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&taddr_s)),
                 "r"(ncol)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) mbar_init(&bar);
  // kind::tf32: D F32 (bits 4-5 = 1), A and B TF32 (bits 7-9, 10-12 = 2),
  // both K-major, N / 8 at bits 17-22, M / 16 at bits 24-28
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(np >> 3) << 17) |
                         ((uint32_t)(RTC_M >> 4) << 24);
  bool ok = true;
  // the thread's RTC_TASKS (row, four-column group) values of chunk ch
  auto load_chunk = [&](int ch, float4 (&x)[RTC_TASKS]) {
#pragma unroll
    for (int t = 0; t < RTC_TASKS; ++t) {
      const int q = warp + t * (RTC_NT / 32);
      const int c = ch * RTC_KC + 4 * (q / (RTC_M / 32));
      const int r = (q % (RTC_M / 32)) * 32 + lane;
      x[t] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (r < nr) {
        const float* src = basis + r0 + r + ldb * c;
        if (c < kc) x[t].x = src[0];
        if (c + 1 < kc) x[t].y = src[ldb];
        if (c + 2 < kc) x[t].z = src[2 * ldb];
        if (c + 3 < kc) x[t].w = src[3 * ldb];
      }
    }
  };
  float4 xa[RTC_TASKS];
  load_chunk(0, xa);
  for (int ch = 0; ch < nchunk; ++ch) {
    const int c0 = ch * RTC_KC;
    // 1. this chunk's basis rows and coefficients, split into TF32 hi / lo,
    //    into the K-major core-matrix layout the MMA reads.  Lane = row:
    //    four 4-byte loads (one per column of a group of four; 32 consecutive
    //    rows of a column are 128 contiguous bytes) give each thread the 16
    //    bytes of one core-matrix row, stored with one 16-byte store per
    //    part, so each group of eight lanes fills one contiguous 128-byte
    //    core matrix (no bank conflicts, no separate split pass).  The next
    //    chunk's loads are issued first, so they are in flight during this
    //    chunk's stores and MMAs.
    float4 xn[RTC_TASKS];
    if (ch + 1 < nchunk) load_chunk(ch + 1, xn);
#pragma unroll
    for (int t = 0; t < RTC_TASKS; ++t) {
      const int q = warp + t * (RTC_NT / 32);
      const int g = q / (RTC_M / 32);
      const int r = (q % (RTC_M / 32)) * 32 + lane;
      float4 h, l;
      tf32_split(xa[t], h, l);
      const uint32_t off = (uint32_t)((((r >> 3) * (RTC_KC / 4) + g) << 7) + ((r & 7) << 4));
      *reinterpret_cast<float4*>(smraw + off) = h;
      *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(alo) + off) = l;
    }
#pragma unroll
    for (int t = 0; t < RTC_TASKS; ++t) xa[t] = xn[t];
    for (int q = warp; q < ((np + 31) / 32) * (RTC_KC / 4); q += RTC_NT / 32) {
      const int ngs = (np + 31) / 32, g = q / ngs;
      const int nn = (q % ngs) * 32 + lane, c = c0 + 4 * g;
      if (nn < np) {
        float4 x = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        const float* src = it.Cs + (int64_t)c * it.ldcs + nn;   // zero past kk
        if (c < kc) x.x = src[0];
        if (c + 1 < kc) x.y = src[it.ldcs];
        if (c + 2 < kc) x.z = src[2 * it.ldcs];
        if (c + 3 < kc) x.w = src[3 * it.ldcs];
        float4 h, l;
        tf32_split(x, h, l);
        const uint32_t off = (uint32_t)((((nn >> 3) * (RTC_KC / 4) + g) << 7) + ((nn & 7) << 4));
        *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(bhi) + off) = h;
        *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(blo) + off) = l;
      }
    }
    // generic-proxy stores become visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // 3. one thread: D (128 x np, FP32 in TMEM) += Ahi Bhi + Ahi Blo + Alo Bhi
    if (tid == 0) {
      const uint32_t tmem = taddr_s;
      const uint32_t kstep = 2 * 128;                   // 8 K-elements = two core matrices
      const uint32_t lbo = 128, sbo = (uint32_t)(RTC_KC / 4) * 128;
      const uint32_t sa = smem_u32(ahi), sl = smem_u32(alo), sb = smem_u32(bhi), sm = smem_u32(blo);
      for (int ks = 0; ks < RTC_KC / 8; ++ks) {
        const uint32_t o = ks * kstep;
        mma_tf32(tmem, smem_desc(sa + o, lbo, sbo), smem_desc(sb + o, lbo, sbo), idesc, (ch | ks) ? 1u : 0u);
        mma_tf32(tmem, smem_desc(sa + o, lbo, sbo), smem_desc(sm + o, lbo, sbo), idesc, 1u);
        mma_tf32(tmem, smem_desc(sl + o, lbo, sbo), smem_desc(sb + o, lbo, sbo), idesc, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&bar))
                   : "memory");
    }
    // the next chunk overwrites the operands: wait for these MMAs
    ok = mbar_wait_bounded(&bar, (uint32_t)(ch & 1), RTC_POLL);
    if (!ok && tid == 0) atomicAdd(&g_ritz_tc_timeouts, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!__syncthreads_and(ok)) { ok = false; break; }
  }
  const uint32_t tmem = taddr_s;
  // 4. TMEM -> rows: warp w reads lanes 32 (w % 4).. (its rows), warps 0-3
  //    the even groups of eight columns, warps 4-7 the odd ones
  if (ok) {
    const int quarter = warp & 3, half = warp >> 2;
    const int row = quarter * 32 + lane;
    float* out = basis + r0 + row;
    for (int cb = half * 8; cb < np; cb += 16) {
      uint32_t v[8];
      const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)cb;
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                   : "r"(ta));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < nr) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (cb + j < kk) out[ldb * (cb + j)] = __uint_as_float(v[j]);
      }
    }
    // restart: the residual direction (column k, not written above) moves to kk
    if (!final_pass)
      for (int t = tid; t < nr; t += RTC_NT) basis[r0 + t + ldb * kk] = basis[r0 + t + ldb * k];
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
  (void)kmax;
  if (n <= 0 || tiles <= 0) return;
  set_max_smem((const void*)k_ritz_tc);
  const int np = (kkmax + 15) & ~15;
  k_ritz_tc<<<tiles, RTC_NT, ritz_tc_smem(kkmax), st>>>(items, pre, n, final_pass, np); count_launch();
}

int ritz_tc_timeouts(cudaStream_t st) {
  int h = 0, z = 0;
  if (cudaMemcpyFromSymbolAsync(&h, g_ritz_tc_timeouts, sizeof(int), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return -1;
  if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
  if (h) cudaMemcpyToSymbolAsync(g_ritz_tc_timeouts, &z, sizeof(int), 0, cudaMemcpyHostToDevice, st);
  return h;
}

}  // namespace ssa
