// Golub-Kahan-Lanczos bidiagonalisation with one-sided full
// re-orthogonalisation and thick restart; Ritz extraction by a one-sided
// Jacobi SVD of the small B in FP64.  See lanczos.h for the recurrences.
//
// The paper delegates this step to PROPACK / nu-TRLan (Sec. 2.4, 4.2); the
// method computes the same r leading eigentriples (Sec. 2.1, Step 2).
#include <algorithm>
#include <type_traits>
#include "lanczos.h"
#include "launch.h"
#include "tma.cuh"
#include "ff.cuh"

namespace ssa {


__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; result valid in every thread (uses red[32]).
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; ++i) t += red[i];   // fixed order: deterministic
  return t;
}

__device__ __forceinline__ double hash_uniform(uint64_t seed, uint64_t i) {
  // SplitMix64 output function (Steele, Lea, Flood 2014) -> [-1, 1)
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

// Seed of the replacement vector after a breakdown at step j on one side
// (0 short, 1 long): distinct from the start vector's stream and per step.
__device__ __forceinline__ uint64_t breakdown_seed(uint64_t seed, int side, int j) {
  uint64_t z = seed ^ 0xD1B54A32D192ED03ull;
  z += 0x632BE59BD9B4E019ull * (uint64_t)(2 * (j + 1) + side);
  z = (z ^ (z >> 29)) * 0xBF58476D1CE4E5B9ull;
  return z ^ (z >> 32);
}

__device__ __forceinline__ bool lz_skip(const LzState* st, int j) {
  return !st->active || j >= st->k || j < -1;
}

// partial dots out[i] = sum over this block's rows of U[row, i] * pv[row - r0]
__device__ void block_dots(const double* __restrict__ U, int64_t ldu, int64_t r0, int nrows,
                           const double* pv, int j, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i < j; i += nw) {
    const double* col = U + ldu * i + r0;
    double acc = 0.0;
    for (int t = lane; t < nrows; t += 32) acc += col[t] * pv[t];
    acc = warp_sum(acc);
    if (lane == 0) out[i] = acc;
  }
}

// ------------------------------------------------------------ short side
// step 1: p = sum of the channel partial products A v_j; partial dots U^T p.
// The coupling terms beta_{j-1} u_{j-1} (or rho_i u_i after a restart) are
// not subtracted explicitly: they are exactly the components along U that the
// first Gram-Schmidt pass removes.
__global__ void __launch_bounds__(SHORT_RB) k_short1(const ShortItem* __restrict__ items, const int32_t* __restrict__ tpre,
                                                     int n, int s) {
  int blk;
  const ShortItem it = items[tile_item(tpre, n, blockIdx.x, blk)];
  const int j = it.st->jc + s;
  if (j < 0 || lz_skip(it.st, j)) return;
  __shared__ double pv[SHORT_RB];
  const int64_t r0 = (int64_t)blk * SHORT_RB;
  const int nrows = (int)imin64(SHORT_RB, it.Ls - r0);
  const int64_t row = r0 + threadIdx.x;
  double val = 0.0;
  if ((int)threadIdx.x < nrows) {
    // sum of the channel partial products, loads issued four at a time
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    int q = 0;
    if (it.parts_double) {
      const double* pp = (const double*)it.parts + row;
      for (; q + 3 < it.n_part; q += 4) {
        const double x0 = pp[(q + 0) * it.part_ld], x1 = pp[(q + 1) * it.part_ld];
        const double x2 = pp[(q + 2) * it.part_ld], x3 = pp[(q + 3) * it.part_ld];
        acc[0] += x0; acc[1] += x1; acc[2] += x2; acc[3] += x3;
      }
      for (; q < it.n_part; ++q) acc[0] += pp[q * it.part_ld];
    } else {
      const float* pp = (const float*)it.parts + row;
      for (; q + 3 < it.n_part; q += 4) {
        const float x0 = pp[(q + 0) * it.part_ld], x1 = pp[(q + 1) * it.part_ld];
        const float x2 = pp[(q + 2) * it.part_ld], x3 = pp[(q + 3) * it.part_ld];
        acc[0] += (double)x0; acc[1] += (double)x1; acc[2] += (double)x2; acc[3] += (double)x3;
      }
      for (; q < it.n_part; ++q) acc[0] += (double)pp[q * it.part_ld];
    }
    val = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    it.p[row] = val;
  }
  pv[threadIdx.x] = val;
  __syncthreads();
  block_dots(it.U, it.ldu, r0, nrows, pv, j, it.cpa + (int64_t)blk * (KMAX + 1));
}

// steps 2 and 3: p -= U c (c summed from the partials in fixed order); step 2
// also forms the partial dots of the second Gram-Schmidt pass, step 3 the
// partial squared norm.
template <int PASS>
__global__ void __launch_bounds__(SHORT_RB) k_short23(const ShortItem* __restrict__ items, const int32_t* __restrict__ tpre,
                                                      int n, int s) {
  int blk;
  const ShortItem it = items[tile_item(tpre, n, blockIdx.x, blk)];
  const int j = it.st->jc + s;
  if (j < 0 || lz_skip(it.st, j)) return;
  __shared__ double c[KMAX + 1];
  __shared__ double pv[SHORT_RB];
  __shared__ double red[32];
  const double* src = (PASS == 2) ? it.cpa : it.cpb;
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    double a = 0.0;
    for (int b = 0; b < it.nblk; ++b) a += src[(int64_t)b * (KMAX + 1) + i];
    c[i] = a;
  }
  __syncthreads();
  const int64_t r0 = (int64_t)blk * SHORT_RB;
  const int nrows = (int)imin64(SHORT_RB, it.Ls - r0);
  const int64_t row = r0 + threadIdx.x;
  double val = 0.0;
  if ((int)threadIdx.x < nrows) {
    val = it.p[row];
    for (int i = 0; i < j; ++i) val -= it.U[row + it.ldu * i] * c[i];
    it.p[row] = val;
  }
  if (PASS == 2) {
    pv[threadIdx.x] = val;
    __syncthreads();
    block_dots(it.U, it.ldu, r0, nrows, pv, j, it.cpb + (int64_t)blk * (KMAX + 1));
  } else {
    const double tot = block_sum(val * val, red);
    if (threadIdx.x == 0) it.npart[blk] = tot;
  }
}

// Whole short-side step of one problem in one block (Ls <= SHORT_FUSED_MAX):
// p = sum of the channel partial products; classical Gram-Schmidt against
// U[:, 0:j]; a second pass only when the first left a component above a
// rounding-level fraction of the remaining norm (the criterion of Daniel,
// Gragg, Kaufman and Stewart); alpha_j = ||p||, u_j = p / alpha_j,
// B[j, j] = alpha_j.  One launch per step instead of four, and each warp's
// dot products run over all rows, so the FP64 reductions stay a small part of
// the FP64 work.  The long side is not re-orthogonalised, so U must stay
// orthogonal to FP64 rounding (the loss in V grows with U's times the
// condition of B): the component left along U is measured, not bounded from
// the norms -- a norm-ratio test let ghost singular values through on long
// noisy series.
template <int NT>
__device__ __forceinline__ void short_dots(const double* __restrict__ U, int64_t ldu, const double* p, int64_t Ls,
                                           int j, double* c) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = warp; i < j; i += NT / 32) {
    const double* col = U + ldu * i;
    // two accumulators: every extra one costs an FP64 add per lane
    double a0 = 0.0, a1 = 0.0;
    int64_t t = lane;
    for (; t + 32 < Ls; t += 64) { a0 = fma(col[t], p[t], a0); a1 = fma(col[t + 32], p[t + 32], a1); }
    if (t < Ls) a0 = fma(col[t], p[t], a0);
    const double tot = warp_sum(a0 + a1);
    if (lane == 0) c[i] = tot;
  }
}

// p -= U c over the block's rows; returns this thread's share of ||p||^2
__device__ __forceinline__ double short_update(const double* __restrict__ U, int64_t ldu, double* p, int64_t Ls, int j,
                                               const double* c) {
  double nn = 0.0;
  for (int64_t row = threadIdx.x; row < Ls; row += blockDim.x) {
    double s0 = 0.0, s1 = 0.0;
    int i = 0;
    for (; i + 1 < j; i += 2) { s0 = fma(U[row + ldu * i], c[i], s0); s1 = fma(U[row + ldu * (i + 1)], c[i + 1], s1); }
    if (i < j) s0 = fma(U[row + ldu * i], c[i], s0);
    const double v = p[row] - (s0 + s1);
    p[row] = v;
    nn = fma(v, v, nn);
  }
  return nn;
}

// Breakdown level of the short side (lanczos.h): the products' rounding level
// or BD_REL_* times the largest coefficient, whichever is larger.
__device__ __forceinline__ double short_bd_level(const ShortItem& it, const LzState* st) {
  return fmax(st->bd_floor, (it.parts_double ? BD_REL_FP64 : BD_REL_FP32) * st->anorm);
}

// After a breakdown at step j: p (Ls values, shared or global memory of this
// block) <- a seeded random vector, orthogonalised twice against U[:, 0:j].
// NT = blockDim.x.  Returns ||p||^2; every thread gets it.
template <int NT>
__device__ double short_random(const ShortItem& it, double* p, int64_t Ls, int j, double* c, double* red) {
  const uint64_t sd = breakdown_seed(it.seed, 0, j);
  for (int64_t row = threadIdx.x; row < Ls; row += blockDim.x) p[row] = hash_uniform(sd, (uint64_t)row);
  __syncthreads();
  double nn = 0.0;
  for (int pass = 0; pass < 2; ++pass) {
    short_dots<NT>(it.U, it.ldu, p, Ls, j, c);
    __syncthreads();
    nn = block_sum(short_update(it.U, it.ldu, p, Ls, j, c), red);
  }
  return nn;
}

// B[j, j] = alpha_j (0 after a breakdown, which is counted); one thread.
__device__ __forceinline__ void short_coef(const ShortItem& it, LzState* st, int j, bool ok, double alpha) {
  it.B[j + (int64_t)it.ldb * j] = ok ? alpha : 0.0;
  if (ok) { if (alpha > st->anorm) st->anorm = alpha; }
  else st->breakdown += 1;
}

// step 4: alpha_j = ||p||, u_j = p / alpha_j, B[j,j] = alpha_j
__global__ void __launch_bounds__(SHORT_RB) k_short4(const ShortItem* __restrict__ items, const int32_t* __restrict__ tpre,
                                                     int n, int s) {
  int blk;
  const ShortItem it = items[tile_item(tpre, n, blockIdx.x, blk)];
  LzState* st = it.st;
  const int j = st->jc + s;
  if (j < 0 || lz_skip(st, j)) return;
  __shared__ double alpha_s;
  __shared__ int ok_s;
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int b = 0; b < it.nblk; ++b) a += it.npart[b];
    alpha_s = sqrt(a);
    // every block of the problem takes this decision: anorm only grows, to
    // alpha_j, when alpha_j passes, so a block reading it late agrees
    ok_s = alpha_s > short_bd_level(it, st);
  }
  __syncthreads();
  const double alpha = alpha_s;
  const bool ok = ok_s != 0;
  if (ok) {
    const int64_t row = (int64_t)blk * SHORT_RB + threadIdx.x;
    if (row < it.Ls) it.U[row + it.ldu * j] = it.p[row] / alpha;
    if (blk == 0 && threadIdx.x == 0) short_coef(it, st, j, true, alpha);
    return;
  }
  // breakdown (rare): block 0 alone builds the whole replacement vector; the
  // other blocks of the problem write nothing (they took the same decision)
  if (blk != 0) return;
  __shared__ double c[KMAX + 1];
  __shared__ double red[32];
  const double nn = short_random<SHORT_RB>(it, it.p, it.Ls, j, c, red);
  const double inv = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
  for (int64_t row = threadIdx.x; row < it.Ls; row += blockDim.x) it.U[row + it.ldu * j] = it.p[row] * inv;
  if (threadIdx.x == 0) short_coef(it, st, j, false, 0.0);
}

constexpr int SHORT_FUSED_NT = 512;
__global__ void __launch_bounds__(SHORT_FUSED_NT) k_short_fused(const ShortItem* __restrict__ items, int s) {
  const ShortItem it = items[blockIdx.x];
  LzState* st = it.st;
  const int j = st->jc + s;
  if (j < 0 || lz_skip(st, j)) return;
  extern __shared__ __align__(16) double sp[];      // p, Ls values
  __shared__ double c[KMAX + 1];
  __shared__ double red[32];
  __shared__ int second;
  const int Ls = (int)it.Ls;
  const double level = short_bd_level(it, st);   // read before thread 0 may raise anorm
  double* p = sp;
  for (int row = threadIdx.x; row < Ls; row += blockDim.x) {
    int q = 0;
    if (it.parts_double) {
      double a0 = 0.0, a1 = 0.0;
      const double* pp = (const double*)it.parts + row;
      for (; q + 1 < it.n_part; q += 2) { a0 += pp[q * it.part_ld]; a1 += pp[(q + 1) * it.part_ld]; }
      if (q < it.n_part) a0 += pp[q * it.part_ld];
      p[row] = a0 + a1;
    } else {
      // FP32 products: their channel sum in FP32 (the products carry FP32
      // error already), one conversion; GB300's FP64 pipe is the bound here
      float a0 = 0.0f, a1 = 0.0f;
      const float* pp = (const float*)it.parts + row;
      for (; q + 1 < it.n_part; q += 2) { a0 += pp[q * it.part_ld]; a1 += pp[(q + 1) * it.part_ld]; }
      if (q < it.n_part) a0 += pp[q * it.part_ld];
      p[row] = (double)(a0 + a1);
    }
  }
  __syncthreads();
  short_dots<SHORT_FUSED_NT>(it.U, it.ldu, p, Ls, j, c);
  __syncthreads();
  double nn = block_sum(short_update(it.U, it.ldu, p, Ls, j, c), red);
  __syncthreads();
  short_dots<SHORT_FUSED_NT>(it.U, it.ldu, p, Ls, j, c);
  __syncthreads();
  if (threadIdx.x == 0) {
    // second pass unless the first left less than thr ||p|| along U: 1e-12
    // when the products are FP32 (far below their own error), 1e-14 in the
    // FP64 form
    const double thr = it.parts_double ? 1e-14 : 1e-12;
    double cc = 0.0;
    for (int i = 0; i < j; ++i) cc = fma(c[i], c[i], cc);
    second = cc > thr * thr * nn;
  }
  __syncthreads();
  if (second) nn = block_sum(short_update(it.U, it.ldu, p, Ls, j, c), red);
  double alpha = sqrt(nn);
  const bool ok = alpha > level;
  if (!ok) {
    __syncthreads();
    nn = short_random<SHORT_FUSED_NT>(it, p, Ls, j, c, red);
    alpha = sqrt(nn);
  }
  const double inv = alpha > 0.0 ? 1.0 / alpha : 0.0;
  for (int row = threadIdx.x; row < Ls; row += blockDim.x) it.U[row + it.ldu * j] = p[row] * inv;
  if (threadIdx.x == 0) short_coef(it, st, j, ok, alpha);
}

void launch_short_fused(const ShortItem* items, int n, int64_t max_ls, int s, cudaStream_t st) {
  if (n <= 0) return;
  set_max_smem((const void*)k_short_fused);
  k_short_fused<<<n, SHORT_FUSED_NT, sizeof(double) * (size_t)max_ls, st>>>(items, s); count_launch();
}

// ------------------------------------------------------------ short side, float-float
// The FP32 form's short side: the steps above in float-float arithmetic
// (ff.cuh) on U's (hi, lo) copy, held as two FP32 arrays Uh and Ul (leading
// dimension ldf = Ls rounded up to a multiple of four, zero pad rows).
// GB300's FP64 pipe issues about 1.7 FMAs per clock per SM against about
// 118 FP32 FMAs, and the FP64 short side ran its FP64 pipe at 77% of peak; a
// float-float product-sum is about a dozen FP32 instructions.  The
// coefficients of the Gram-Schmidt passes carry about 48 bits, so U stays
// orthogonal to about n 2^-48 (n = Ls) -- far below the FP32 products' own
// error, which bounds what the FP32 form resolves.

template <int NT>
__device__ __forceinline__ ff block_sum_ffv(ffacc v, float2* red) {
  v = warp_sum_ff(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = make_float2(v.s, v.c);
  __syncthreads();
  ffacc t;
  for (int i = 0; i < NT / 32; ++i) { ffacc o; o.s = red[i].x; o.c = red[i].y; t.add(o); }   // fixed order
  return t.value();
}

// c[i] = U[:, i]^T p over rows [0, nrows) of U (from row r0) and p, i < j; a warp per column
template <int NT>
__device__ __forceinline__ void dots_ff(const float* __restrict__ Uh, const float* __restrict__ Ul, int64_t ldf,
                                        int64_t r0, const float2* p, int nrows, int j, float2* c) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = warp; i < j; i += NT / 32) {
    const float* __restrict__ ch = Uh + ldf * i + r0;
    const float* __restrict__ cl = Ul + ldf * i + r0;
    ffacc a0, a1;                   // two chains: the TwoSum of one is a dependent sequence
    int t = lane;
    // eight loads of each part issued before their arithmetic: U streams
    // from L2 / HBM, and one block per problem has few warps to hide that
    // latency with
    for (; t + 7 * 32 < nrows; t += 8 * 32) {
      float uh[8], ul[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) { uh[m] = ch[t + 32 * m]; ul[m] = cl[t + 32 * m]; }
#pragma unroll
      for (int m = 0; m < 8; m += 2) {
        const float2 p0 = p[t + 32 * m], p1 = p[t + 32 * (m + 1)];
        a0.fma(uh[m], ul[m], p0.x, p0.y);
        a1.fma(uh[m + 1], ul[m + 1], p1.x, p1.y);
      }
    }
    for (; t < nrows; t += 32) { const float2 pv = p[t]; a0.fma(ch[t], cl[t], pv.x, pv.y); }
    a0.add(a1);
    const ff v = warp_sum_ff(a0).value();
    if (lane == 0) c[i] = make_float2(v.hi, v.lo);
  }
}

// (U c)[row] for one row (Uh, Ul point at the row in column 0)
__device__ __forceinline__ ff update_row_ff(const float* __restrict__ Uh, const float* __restrict__ Ul, int64_t ldf,
                                           int j, const float2* c) {
  ffacc s0, s1;
  int i = 0;
  for (; i + 7 < j; i += 8) {         // eight loads of each part in flight (see dots_ff)
    float uh[8], ul[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) { uh[m] = Uh[ldf * (i + m)]; ul[m] = Ul[ldf * (i + m)]; }
#pragma unroll
    for (int m = 0; m < 8; m += 2) {
      s0.fma(uh[m], ul[m], c[i + m].x, c[i + m].y);
      s1.fma(uh[m + 1], ul[m + 1], c[i + m + 1].x, c[i + m + 1].y);
    }
  }
  for (; i < j; ++i) s0.fma(Uh[ldf * i], Ul[ldf * i], c[i].x, c[i].y);
  s0.add(s1);
  return s0.value();
}

// p[row] -= (U c)[row] for this thread's rows of [0, Ls); returns the
// thread's share of ||p||^2
__device__ __forceinline__ ffacc update_ff(const float* __restrict__ Uh, const float* __restrict__ Ul, int64_t ldf,
                                           float2* p, int Ls, int j, const float2* c) {
  ffacc nn;
  for (int row = threadIdx.x; row < Ls; row += blockDim.x) {
    const ff sv = update_row_ff(Uh + row, Ul + row, ldf, j, c);
    const float2 pr = p[row];
    const ff v = ff_add(ff{pr.x, pr.y}, ff_neg(sv));
    p[row] = make_float2(v.hi, v.lo);
    nn.fma(v.hi, v.lo, v.hi, v.lo);
  }
  return nn;
}

// After a breakdown at step j: p <- a seeded random vector (FP32 values of the
// FP64 form's sequence), orthogonalised twice against U[:, 0:j]; returns ||p||^2.
template <int NT>
__device__ ff short_random_ff(const ShortItem& it, float2* p, int Ls, int j, float2* c, float2* red) {
  const uint64_t sd = breakdown_seed(it.seed, 0, j);
  for (int row = threadIdx.x; row < Ls; row += blockDim.x)
    p[row] = make_float2((float)hash_uniform(sd, (uint64_t)row), 0.0f);
  __syncthreads();
  ff nn{0.0f, 0.0f};
  for (int pass = 0; pass < 2; ++pass) {
    dots_ff<NT>(it.Uh, it.Ul, it.ldf, 0, p, Ls, j, c);
    __syncthreads();
    nn = block_sum_ffv<NT>(update_ff(it.Uh, it.Ul, it.ldf, p, Ls, j, c), red);
  }
  return nn;
}

// u_j = p / alpha into Uh, Ul and U (thread's rows of [r0, r0 + nrows)), and
// the zero pad rows past Ls from the block that owns row Ls - 1
__device__ __forceinline__ void write_u_ff(const ShortItem& it, const float2* p, int64_t r0, int nrows, int j,
                                           float2 inv) {
  for (int t = threadIdx.x; t < nrows; t += blockDim.x) {
    const float2 pr = p[t];
    const ff u = ff_mul(ff{pr.x, pr.y}, ff{inv.x, inv.y});
    it.Uh[r0 + t + it.ldf * j] = u.hi;
    it.Ul[r0 + t + it.ldf * j] = u.lo;
    it.U[r0 + t + it.ldu * j] = ff_to_double(make_float2(u.hi, u.lo));
  }
  if (r0 + nrows == it.Ls)
    for (int64_t t = it.Ls + threadIdx.x; t < it.ldf; t += blockDim.x) {
      it.Uh[t + it.ldf * j] = 0.0f;
      it.Ul[t + it.ldf * j] = 0.0f;
    }
}

// sum of the FP32 channel partial products at one row (FP32 form: they carry
// FP32 error already)
__device__ __forceinline__ float parts_row(const ShortItem& it, int64_t row) {
  const float* pp = (const float*)it.parts + row;
  float a0 = 0.0f, a1 = 0.0f;
  int q = 0;
  for (; q + 1 < it.n_part; q += 2) { a0 += pp[q * it.part_ld]; a1 += pp[(q + 1) * it.part_ld]; }
  if (q < it.n_part) a0 += pp[q * it.part_ld];
  return a0 + a1;
}

// alpha = sqrt(nn), the breakdown decision and 1 / alpha as float-float;
// one thread
__device__ __forceinline__ void alpha_ff(ff nn, double level, double& alpha, int& ok, float2& inv) {
  alpha = sqrt(fmax(ff_to_double(make_float2(nn.hi, nn.lo)), 0.0));
  ok = alpha > level;
  inv = ff_from_double(alpha > 0.0 ? 1.0 / alpha : 0.0);
}

// Whole step of one problem in one block, U streamed through shared memory:
// each Gram-Schmidt pass (U^T p, or p -= U c) reads the columns in chunks
// that bulk copies (cp.async.bulk, the TMA engine) bring into SHORT_TMA_S
// rotating stage buffers, completing on one mbarrier per stage, while the
// warps work on the previous chunk.  A float-float pass brings cw columns of
// both parts per chunk, an FP32 pass 2 cw columns of the hi part (the same
// bytes: half the chunks).  A dot product pass gives each column 16 /
// (columns per chunk) warps (partial sums, reduced in fixed order at the end
// of the pass); an update pass keeps each thread's rows' running sums in
// registers across the chunks.
constexpr int SHORT_TMA_NT = 512;
constexpr int MBAR_POLL_LIMIT_SHORT = 1 << 22;
constexpr int SHORT_TMA_S = 3;
constexpr int SHORT_TMA_RPP = SHORT_FUSED_MAX / (2 * SHORT_TMA_NT);   // row pairs per thread, at most
__device__ int g_short_tma_timeouts;

struct ShortStream {
  float* stage;       // stage s: 2 cw columns of sld floats at stage + s * 2 cw sld
  int64_t sld;        // column stride of the stage buffers (the launch's largest ldf)
  uint64_t* bar;      // one mbarrier per stage
  int cw;             // float-float columns per chunk
  uint32_t g;         // chunks consumed so far, over all passes: chunk g used stage
                      // g % S in its (g / S)-th phase
};

// chunk q of a pass (columns [q w, min(j, q w + w)) of the pass's chunk
// width w) into stage (g0 + q) % S; FF: the hi parts, then the lo parts.
// One thread.
template <bool FF>
__device__ __forceinline__ void short_issue(const ShortItem& it, const ShortStream& ss, uint32_t g0, int q, int j,
                                            int w) {
  const int s = (int)((g0 + q) % SHORT_TMA_S);
  const int c0 = q * w, cn = min(w, j - c0);
  const uint32_t bytes = (uint32_t)(sizeof(float) * it.ldf);
  float* dst = ss.stage + (int64_t)s * 2 * ss.cw * ss.sld;
  // the stage was last read by generic loads: order them before the async writes
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_arrive_expect(&ss.bar[s], bytes * (uint32_t)cn * (FF ? 2u : 1u));
  for (int ci = 0; ci < cn; ++ci) {
    bulk_copy(dst + (int64_t)ci * ss.sld, it.Uh + it.ldf * (c0 + ci), bytes, &ss.bar[s]);
    if (FF) bulk_copy(dst + (int64_t)(w + ci) * ss.sld, it.Ul + it.ldf * (c0 + ci), bytes, &ss.bar[s]);
  }
}

// One pass over columns [0, j) in one of four forms:
//   SP_DOT_FF / SP_DOT_32: part[i * wpc + slot] = partial sums of U[:, i]^T p
//     (float-float, or FP32 from the hi parts of U and p);
//   SP_UPD_FF / SP_UPD_32 / SP_UPD_FC: acc += (U c) for the thread's row
//     pairs (2 (threadIdx.x + m NT), + 1), m < RPP: float-float, or FP32
//     from the hi parts (SP_UPD_FC subtracts that FP32 sum from the
//     float-float p exactly, see k_short_fused_ff).
// The FP32 dot pass takes rows in fours (16-byte loads of the hi part), the
// others in pairs; p and every column of U have zero pad rows up to ldf.
// Ends with the block synchronised.
enum ShortPass { SP_DOT_FF, SP_DOT_32, SP_UPD_FF, SP_UPD_32, SP_UPD_FC };

// columns per chunk of a pass: cw float-float, else 2 cw hi parts (at most 16:
// a dot pass gives each column at least one warp)
template <int MODE>
__device__ __forceinline__ int pass_width(const ShortStream& ss) {
  return (MODE == SP_DOT_FF || MODE == SP_UPD_FF) ? ss.cw : min(2 * ss.cw, SHORT_TMA_NT / 32);
}

template <int MODE, int RPP>
__device__ __forceinline__ void short_pass(const ShortItem& it, ShortStream& ss, int j, int Ls, const float2* p,
                                           const float2* c, float2* part, ffacc (&acc)[2 * RPP],
                                           float (&acc32)[2 * RPP]) {
  constexpr bool DOTS = MODE == SP_DOT_FF || MODE == SP_DOT_32;
  constexpr bool FF = MODE == SP_DOT_FF || MODE == SP_UPD_FF;
  const int w = pass_width<MODE>(ss);
  const int nch = (j + w - 1) / w;
  if (nch == 0) return;
  const uint32_t g0 = ss.g;
  if (threadIdx.x == 0)
    for (int q = 0; q < min(SHORT_TMA_S, nch); ++q) short_issue<FF>(it, ss, g0, q, j, w);
  const int wpc = (SHORT_TMA_NT / 32) / w;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int np2 = (Ls + 1) >> 1, np4 = (Ls + 3) >> 2;
  const float4* p4 = reinterpret_cast<const float4*>(p);
  for (int q = 0; q < nch; ++q) {
    const uint32_t gq = g0 + q;
    const int s = (int)(gq % SHORT_TMA_S);
    if (!mbar_wait_bounded(&ss.bar[s], (gq / SHORT_TMA_S) & 1u, MBAR_POLL_LIMIT_SHORT) && threadIdx.x == 0)
      atomicAdd(&g_short_tma_timeouts, 1);
    const float* buf = ss.stage + (int64_t)s * 2 * ss.cw * ss.sld;
    const int c0 = q * w, cn = min(w, j - c0);
    if (DOTS) {
      const int ci = warp / wpc, slot = warp - ci * wpc;
      if (ci < cn) {
        float2 v;
        if (MODE == SP_DOT_FF) {
          const float2* ch = reinterpret_cast<const float2*>(buf + (int64_t)ci * ss.sld);
          const float2* cl = reinterpret_cast<const float2*>(buf + (int64_t)(w + ci) * ss.sld);
          ffacc a0, a1;
          for (int t = slot * 32 + lane; t < np2; t += 32 * wpc) {
            const float2 uh = ch[t], ul = cl[t];
            const float4 pv = p4[t];
            a0.fma(uh.x, ul.x, pv.x, pv.y);
            a1.fma(uh.y, ul.y, pv.z, pv.w);
          }
          a0.add(a1);
          a0 = warp_sum_ff(a0);
          v = make_float2(a0.s, a0.c);
        } else {
          const float4* ch = reinterpret_cast<const float4*>(buf + (int64_t)ci * ss.sld);
          float a0 = 0.0f, a1 = 0.0f;
          for (int t = slot * 32 + lane; t < np4; t += 32 * wpc) {
            const float4 uh = ch[t], p0 = p4[2 * t], p1 = p4[2 * t + 1];
            a0 = fmaf(uh.x, p0.x, a0);
            a1 = fmaf(uh.y, p0.z, a1);
            a0 = fmaf(uh.z, p1.x, a0);
            a1 = fmaf(uh.w, p1.z, a1);
          }
          a0 += a1;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) a0 += __shfl_xor_sync(0xffffffffu, a0, o);
          v = make_float2(a0, 0.0f);
        }
        if (lane == 0) part[(c0 + ci) * wpc + slot] = v;
      }
    } else {
      for (int ci = 0; ci < cn; ++ci) {
        const float2 cc = c[c0 + ci];
        const float2* ch = reinterpret_cast<const float2*>(buf + (int64_t)ci * ss.sld);
        const float2* cl = reinterpret_cast<const float2*>(buf + (int64_t)(w + ci) * ss.sld);
#pragma unroll
        for (int m = 0; m < RPP; ++m) {
          const int t = threadIdx.x + m * SHORT_TMA_NT;
          if (t < np2) {
            const float2 uh = ch[t];
            if (MODE == SP_UPD_FF) {
              const float2 ul = cl[t];
              acc[2 * m].fma(uh.x, ul.x, cc.x, cc.y);
              acc[2 * m + 1].fma(uh.y, ul.y, cc.x, cc.y);
            } else {                      // SP_UPD_32, SP_UPD_FC
              acc32[2 * m] = fmaf(uh.x, cc.x, acc32[2 * m]);
              acc32[2 * m + 1] = fmaf(uh.y, cc.x, acc32[2 * m + 1]);
            }
          }
        }
      }
    }
    __syncthreads();                      // every warp is done with stage s
    if (threadIdx.x == 0 && q + SHORT_TMA_S < nch) short_issue<FF>(it, ss, g0, q + SHORT_TMA_S, j, w);
  }
  ss.g = g0 + (uint32_t)nch;
}

// c[i] = U[:, i]^T p, i < j (FP32: from the hi parts of U and p, as float-float with lo = 0)
template <int MODE>
__device__ __forceinline__ void short_dots_tma(const ShortItem& it, ShortStream& ss, int j, int Ls, const float2* p,
                                               float2* c, float2* part) {
  ffacc none[2];
  float none32[2];
  short_pass<MODE, 1>(it, ss, j, Ls, p, c, part, none, none32);
  const int wpc = (SHORT_TMA_NT / 32) / pass_width<MODE>(ss);
  for (int i = threadIdx.x; i < j; i += SHORT_TMA_NT) {
    ffacc a;
    for (int sl = 0; sl < wpc; ++sl) {    // fixed order
      const float2 v = part[i * wpc + sl];
      ffacc o; o.s = v.x; o.c = v.y; a.add(o);
    }
    const ff v = a.value();
    c[i] = MODE == SP_DOT_FF ? make_float2(v.hi, v.lo) : make_float2(v.hi, 0.0f);
  }
  __syncthreads();
}

// p -= U c (float-float, or FP32 from the hi parts: then p stays FP32, lo = 0);
// returns ||p||^2 (every thread)
template <int MODE, int RPP>
__device__ __forceinline__ ff short_update_tma(const ShortItem& it, ShortStream& ss, int j, int Ls, float2* p,
                                               const float2* c, float2* part, float2* red) {
  ffacc acc[2 * RPP];
  float acc32[2 * RPP];
#pragma unroll
  for (int m = 0; m < 2 * RPP; ++m) acc32[m] = 0.0f;
  short_pass<MODE, RPP>(it, ss, j, Ls, p, c, part, acc, acc32);
  const int np2 = (Ls + 1) >> 1;
  float4* p4 = reinterpret_cast<float4*>(p);
  ffacc nn;
#pragma unroll
  for (int m = 0; m < RPP; ++m) {
    const int t = threadIdx.x + m * SHORT_TMA_NT;
    if (t < np2) {
      float4 w = p4[t];
      if (MODE == SP_UPD_FF) {
        const ff v0 = ff_add(ff{w.x, w.y}, ff_neg(acc[2 * m].value()));
        const ff v1 = ff_add(ff{w.z, w.w}, ff_neg(acc[2 * m + 1].value()));
        w = make_float4(v0.hi, v0.lo, v1.hi, v1.lo);
      } else if (MODE == SP_UPD_FC) {
        const ff v0 = ff_add(ff{w.x, w.y}, ff{-acc32[2 * m], 0.0f});
        const ff v1 = ff_add(ff{w.z, w.w}, ff{-acc32[2 * m + 1], 0.0f});
        w = make_float4(v0.hi, v0.lo, v1.hi, v1.lo);
      } else {
        w = make_float4(w.x - acc32[2 * m], 0.0f, w.z - acc32[2 * m + 1], 0.0f);
      }
      p4[t] = w;
      nn.fma(w.x, w.y, w.x, w.y);
      nn.fma(w.z, w.w, w.z, w.w);
    }
  }
  return block_sum_ffv<SHORT_TMA_NT>(nn, red);   // synchronises the block
}

// Gram-Schmidt of the step: a first pass in FP32 (U's hi parts; the FP32
// products carry FP32 error already, so its rounding costs nothing the data
// resolves), then a float-float pass, whose dot products measure what the
// first left along U; its update runs unless that is below 1e-12 ||p|| (the
// criterion of Daniel, Gragg, Kaufman and Stewart), and in FP32 products of
// the hi parts subtracted exactly from the float-float p when the remainder
// is at most 1e-6 ||p|| (the usual case: the first pass leaves about 6e-8).
// RPP: row pairs per thread, 2 RPP NT >= every item's Ls.
template <int RPP>
__global__ void __launch_bounds__(SHORT_TMA_NT) k_short_fused_ff(const ShortItem* __restrict__ items, int s,
                                                                 int64_t sld, int cw) {
  const ShortItem it = items[blockIdx.x];
  LzState* st = it.st;
  const int j = st->jc + s;
  if (j < 0 || lz_skip(st, j)) return;
  extern __shared__ __align__(16) float2 smf[];
  __shared__ float2 c[KMAX + 1];
  __shared__ float2 red[32];
  __shared__ __align__(8) uint64_t bar[SHORT_TMA_S];
  __shared__ int second, ok_s;
  __shared__ double alpha_s;
  __shared__ float2 inv_s;
  const int Ls = (int)it.Ls;
  float2* p = smf;                                            // sld values (zero pad rows up to ldf)
  ShortStream ss;
  ss.stage = reinterpret_cast<float*>(smf + sld);            // S 2 cw sld floats
  ss.sld = sld;
  ss.bar = bar;
  ss.cw = cw;
  ss.g = 0;
  float2* part = smf + sld * (1 + (int64_t)SHORT_TMA_S * cw); // (KMAX + 1) 16 / cw values
  const double level = short_bd_level(it, st);   // read before thread 0 may raise anorm
  if (threadIdx.x == 0)
    for (int q = 0; q < SHORT_TMA_S; ++q) mbar_init(&bar[q]);
  for (int row = threadIdx.x; row < it.ldf; row += SHORT_TMA_NT)
    p[row] = make_float2(row < Ls ? parts_row(it, row) : 0.0f, 0.0f);
  __syncthreads();
  short_dots_tma<SP_DOT_32>(it, ss, j, Ls, p, c, part);
  ff nn = short_update_tma<SP_UPD_32, RPP>(it, ss, j, Ls, p, c, part, red);
  short_dots_tma<SP_DOT_FF>(it, ss, j, Ls, p, c, part);
  if (threadIdx.x == 0) {
    float cc = 0.0f;
    for (int i = 0; i < j; ++i) cc = fmaf(c[i].x, c[i].x, cc);
    // 0: nothing left along U; 1: ||c|| <= 1e-6 ||p||, so FP32 products of
    // the hi parts carry U c to within sqrt(j) eps32 ||c||: below 1e-12 ||p||
    // at worst, about 3e-14 ||p|| in the usual case (||c|| near 6e-8 ||p||);
    // U's lo parts and c's low bits contribute less; 2: float-float
    second = cc > 1e-24f * nn.hi ? (cc > 1e-12f * nn.hi ? 2 : 1) : 0;
  }
  __syncthreads();
  if (second == 1) nn = short_update_tma<SP_UPD_FC, RPP>(it, ss, j, Ls, p, c, part, red);
  else if (second == 2) nn = short_update_tma<SP_UPD_FF, RPP>(it, ss, j, Ls, p, c, part, red);
  if (threadIdx.x == 0) { double a; int o; float2 iv; alpha_ff(nn, level, a, o, iv); alpha_s = a; ok_s = o; inv_s = iv; }
  __syncthreads();
  if (!ok_s) {
    // breakdown: a seeded random vector, orthogonalised twice in float-float
    const uint64_t sd = breakdown_seed(it.seed, 0, j);
    for (int row = threadIdx.x; row < Ls; row += SHORT_TMA_NT)
      p[row] = make_float2((float)hash_uniform(sd, (uint64_t)row), 0.0f);
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
      short_dots_tma<SP_DOT_FF>(it, ss, j, Ls, p, c, part);
      nn = short_update_tma<SP_UPD_FF, RPP>(it, ss, j, Ls, p, c, part, red);
    }
    if (threadIdx.x == 0) { double a; int o; float2 iv; alpha_ff(nn, 0.0, a, o, iv); inv_s = iv; }
    __syncthreads();
  }
  write_u_ff(it, p, 0, Ls, j, inv_s);
  if (threadIdx.x == 0) short_coef(it, st, j, ok_s != 0, alpha_s);
}

// shared memory of k_short_fused_ff for stage column stride sld and cw
// float-float columns per chunk: p (sld float-float values), the stages
// (S x 2 cw x sld floats) and the dot partials
static size_t short_tma_smem(int64_t sld, int cw) {
  return sizeof(float2) * ((size_t)sld * (1 + SHORT_TMA_S * (size_t)cw) + (size_t)(KMAX + 1) * (16 / cw));
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

int* short_tma_timeout_word() {
  static int* cache[64] = {};
  return counter_word((const void*)&g_short_tma_timeouts, cache);
}

int short_tma_timeouts(cudaStream_t st) {
  int h = 0, z = 0;
  if (cudaMemcpyFromSymbolAsync(&h, g_short_tma_timeouts, sizeof(int), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return -1;
  if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
  if (h) cudaMemcpyToSymbolAsync(g_short_tma_timeouts, &z, sizeof(int), 0, cudaMemcpyHostToDevice, st);
  return h;
}

// Row-block form (problems with more rows than one block should carry, or
// too few problems to fill the SMs).  p: the item's work vector as Ls
// float-float values; cpa / cpb: nblk x (KMAX+1) float-float partial dots;
// npart: nblk float-float partial squared norms.
__global__ void __launch_bounds__(SHORT_RB) k_short1_ff(const ShortItem* __restrict__ items,
                                                        const int32_t* __restrict__ tpre, int n, int s) {
  int blk;
  const ShortItem it = items[tile_item(tpre, n, blockIdx.x, blk)];
  const int j = it.st->jc + s;
  if (j < 0 || lz_skip(it.st, j)) return;
  __shared__ float2 pv[SHORT_RB];
  const int64_t r0 = (int64_t)blk * SHORT_RB;
  const int nrows = (int)imin64(SHORT_RB, it.Ls - r0);
  float2 v = make_float2(0.0f, 0.0f);
  if ((int)threadIdx.x < nrows) {
    v.x = parts_row(it, r0 + threadIdx.x);
    reinterpret_cast<float2*>(it.p)[r0 + threadIdx.x] = v;
  }
  pv[threadIdx.x] = v;
  __syncthreads();
  dots_ff<SHORT_RB>(it.Uh, it.Ul, it.ldf, r0, pv, nrows, j,
                    reinterpret_cast<float2*>(it.cpa) + (int64_t)blk * (KMAX + 1));
}

template <int PASS>
__global__ void __launch_bounds__(SHORT_RB) k_short23_ff(const ShortItem* __restrict__ items,
                                                         const int32_t* __restrict__ tpre, int n, int s) {
  int blk;
  const ShortItem it = items[tile_item(tpre, n, blockIdx.x, blk)];
  const int j = it.st->jc + s;
  if (j < 0 || lz_skip(it.st, j)) return;
  __shared__ float2 c[KMAX + 1];
  __shared__ float2 pv[SHORT_RB];
  __shared__ float2 red[32];
  const float2* src = reinterpret_cast<const float2*>(PASS == 2 ? it.cpa : it.cpb);
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    ffacc a;
    for (int b = 0; b < it.nblk; ++b) {       // fixed order
      const float2 q = src[(int64_t)b * (KMAX + 1) + i];
      ffacc o; o.s = q.x; o.c = q.y; a.add(o);
    }
    const ff v = a.value();
    c[i] = make_float2(v.hi, v.lo);
  }
  __syncthreads();
  const int64_t r0 = (int64_t)blk * SHORT_RB;
  const int nrows = (int)imin64(SHORT_RB, it.Ls - r0);
  float2* p = reinterpret_cast<float2*>(it.p) + r0;
  ffacc nn;
  float2 val = make_float2(0.0f, 0.0f);
  if ((int)threadIdx.x < nrows) {
    const int row = threadIdx.x;
    const ff sv = update_row_ff(it.Uh + r0 + row, it.Ul + r0 + row, it.ldf, j, c);
    const ff v = ff_add(ff{p[row].x, p[row].y}, ff_neg(sv));
    val = make_float2(v.hi, v.lo);
    p[row] = val;
    nn.fma(v.hi, v.lo, v.hi, v.lo);
  }
  if (PASS == 2) {
    pv[threadIdx.x] = val;
    __syncthreads();
    dots_ff<SHORT_RB>(it.Uh, it.Ul, it.ldf, r0, pv, nrows, j,
                      reinterpret_cast<float2*>(it.cpb) + (int64_t)blk * (KMAX + 1));
  } else {
    const ff tot = block_sum_ffv<SHORT_RB>(nn, red);
    if (threadIdx.x == 0) reinterpret_cast<float2*>(it.npart)[blk] = make_float2(tot.hi, tot.lo);
  }
}

__global__ void __launch_bounds__(SHORT_RB) k_short4_ff(const ShortItem* __restrict__ items,
                                                        const int32_t* __restrict__ tpre, int n, int s) {
  int blk;
  const ShortItem it = items[tile_item(tpre, n, blockIdx.x, blk)];
  LzState* st = it.st;
  const int j = st->jc + s;
  if (j < 0 || lz_skip(st, j)) return;
  __shared__ double alpha_s;
  __shared__ int ok_s;
  __shared__ float2 inv_s;
  if (threadIdx.x == 0) {
    ffacc a;
    for (int b = 0; b < it.nblk; ++b) {
      const float2 q = reinterpret_cast<const float2*>(it.npart)[b];
      ffacc o; o.s = q.x; o.c = q.y; a.add(o);
    }
    // every block of the problem takes this decision: anorm only grows, to
    // alpha_j, when alpha_j passes, so a block reading it late agrees
    double al; int ok; float2 iv;
    alpha_ff(a.value(), short_bd_level(it, st), al, ok, iv);
    alpha_s = al; ok_s = ok; inv_s = iv;
  }
  __syncthreads();
  float2* p = reinterpret_cast<float2*>(it.p);
  if (ok_s) {
    const int64_t r0 = (int64_t)blk * SHORT_RB;
    const int nrows = (int)imin64(SHORT_RB, it.Ls - r0);
    write_u_ff(it, p + r0, r0, nrows, j, inv_s);
    if (blk == 0 && threadIdx.x == 0) short_coef(it, st, j, true, alpha_s);
    return;
  }
  // breakdown (rare): block 0 alone builds the whole replacement vector
  if (blk != 0) return;
  __shared__ float2 c[KMAX + 1];
  __shared__ float2 red[32];
  const ff nn = short_random_ff<SHORT_RB>(it, p, (int)it.Ls, j, c, red);
  __syncthreads();
  if (threadIdx.x == 0) { double a; int o; float2 iv; alpha_ff(nn, 0.0, a, o, iv); inv_s = iv; }
  __syncthreads();
  write_u_ff(it, p, 0, (int)it.Ls, j, inv_s);
  if (threadIdx.x == 0) short_coef(it, st, j, false, 0.0);
}

__global__ void __launch_bounds__(256) k_uf_sync(const ShortItem* __restrict__ items, const int32_t* __restrict__ ncols) {
  const ShortItem it = items[blockIdx.y];
  const int64_t n = it.ldf * (int64_t)ncols[blockIdx.y];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / it.ldf, row = e - c * it.ldf;
    const float2 v = row < it.Ls ? ff_from_double(it.U[row + it.ldu * c]) : make_float2(0.0f, 0.0f);
    it.Uh[row + it.ldf * c] = v.x;
    it.Ul[row + it.ldf * c] = v.y;
  }
}

void launch_short_fused_ff(const ShortItem* items, int n, int64_t max_ls, int s, cudaStream_t st) {
  if (n <= 0) return;
  const int64_t sld = (max_ls + 3) & ~int64_t(3);
  // chunks of about 32 KB: cw = the largest power of two <= 32 KB / (8 bytes x column), in [1, 16]
  int cw = 1;
  while (cw < 16 && (int64_t)sizeof(float2) * sld * (2 * cw) <= 32768) cw *= 2;
  const size_t sm = short_tma_smem(sld, cw);
  auto go = [&](auto kern) {
    set_max_smem((const void*)kern);
    kern<<<n, SHORT_TMA_NT, sm, st>>>(items, s, sld, cw);
    count_launch();
  };
  if (max_ls <= 2 * SHORT_TMA_NT) go(k_short_fused_ff<1>);
  else if (max_ls <= 4 * SHORT_TMA_NT) go(k_short_fused_ff<2>);
  else go(k_short_fused_ff<SHORT_TMA_RPP>);
}

void launch_short_steps_ff(const ShortItem* items, const int32_t* tpre, int n, int tiles, int s, cudaStream_t st) {
  if (n <= 0 || tiles <= 0) return;
  k_short1_ff<<<tiles, SHORT_RB, 0, st>>>(items, tpre, n, s); count_launch();
  k_short23_ff<2><<<tiles, SHORT_RB, 0, st>>>(items, tpre, n, s); count_launch();
  k_short23_ff<3><<<tiles, SHORT_RB, 0, st>>>(items, tpre, n, s); count_launch();
  k_short4_ff<<<tiles, SHORT_RB, 0, st>>>(items, tpre, n, s); count_launch();
}

void launch_uf_sync(const ShortItem* items, const int32_t* ncols, int n, cudaStream_t st) {
  if (n <= 0) return;
  k_uf_sync<<<dim3(16, n), 256, 0, st>>>(items, ncols); count_launch();
}

// ------------------------------------------------------------ long side

// q = sum(partials) - alpha_j v_j ; partial squared norms
template <typename T>
__global__ void __launch_bounds__(256) k_long1(const LongItem<T>* __restrict__ items, const int32_t* __restrict__ tpre,
                                               int n, int s) {
  int blk;
  const LongItem<T> it = items[tile_item(tpre, n, blockIdx.x, blk)];
  const int j = it.st->jc + s;
  if (j < 0 || lz_skip(it.st, j)) return;
  __shared__ double red[32];
  // alpha_j v_j with v_j = colscale[j] * V[:, j] (stored unnormalised)
  const T coef = (T)(it.B[j + (int64_t)it.ldb * j] * it.colscale[j]);
  const T* vj = it.V + it.ldv * j;
  T* qn = it.V + it.ldv * (j + 1);
  const int64_t r0 = (int64_t)blk * LONG_RB;
  double acc = 0.0;
  for (int t = threadIdx.x; t < LONG_RB; t += blockDim.x) {
    const int64_t row = r0 + t;
    if (row >= it.Kl) break;
    T v = T(0);
    for (int q = 0; q < it.n_part; ++q) v += it.parts[q * it.part_ld + row];
    v = v - coef * vj[row];
    qn[row] = v;
    acc += (double)v * (double)v;
  }
  const double tot = block_sum(acc, red);
  if (threadIdx.x == 0) it.npart[blk] = tot;
}

template <typename T>
__global__ void __launch_bounds__(256) k_long_init(const LongItem<T>* __restrict__ items, const int32_t* __restrict__ tpre,
                                                   int n) {
  int blk;
  const LongItem<T> it = items[tile_item(tpre, n, blockIdx.x, blk)];
  if (!it.st->active) return;
  __shared__ double red[32];
  const int64_t r0 = (int64_t)blk * LONG_RB;
  double acc = 0.0;
  for (int t = threadIdx.x; t < LONG_RB; t += blockDim.x) {
    const int64_t row = r0 + t;
    if (row >= it.Kl) break;
    const T v = (T)hash_uniform(it.seed, (uint64_t)row);
    it.V[row] = v;
    acc += (double)v * (double)v;
  }
  const double tot = block_sum(acc, red);
  if (threadIdx.x == 0) it.npart[blk] = tot;
}

// beta_j = ||q|| from the partial norms (fixed order); column j+1 of V keeps q
// and its scale 1/beta_j is recorded; B[j, j+1] = beta_j (beta_k at the end).
// A beta_j at the breakdown level (lanczos.h) is set to 0 and v_{j+1} is the
// zero vector (scale 0).  The next short step then sees A v_{j+1} = 0, a
// breakdown there, and continues from a random u_{j+1} orthogonal to U; the
// long step after it forms X^T u_{j+1}, which is orthogonal to v_0..v_j in
// exact arithmetic (A v_i lies in span U_{j+1} for i <= j) -- so the long
// side never needs its own re-orthogonalisation.  When the data's column
// space is already inside span U, X^T u_{j+1} is rounding again and the step
// repeats: the remaining singular values are zero and B holds zero blocks.
template <typename T>
__global__ void __launch_bounds__(32) k_long_norm(const LongItem<T>* __restrict__ items, int s) {
  // one warp per problem: the partials (one per channel, or per block for
  // the start vector) summed in a fixed order; FP64 work on GB300's FP64
  // pipe is charged per warp instruction, so more warps would only cost
  const LongItem<T> it = items[blockIdx.x];
  LzState* st = it.st;
  const int j = st->jc + s;
  if (lz_skip(st, j)) return;
  double a = 0.0;
  const int nb = (s < 0) ? it.nblk : it.nsum;    // start vector: its blocks; a step: nsum partials
  for (int b = threadIdx.x; b < nb; b += 32) a += it.npart[b];
  a = warp_sum(a);
  if (threadIdx.x != 0) return;
  const double level = fmax(st->bd_floor, (sizeof(T) == 8 ? BD_REL_FP64 : BD_REL_FP32) * st->anorm);
  const double beta = sqrt(a);
  const bool ok = j < 0 || beta > level;         // (the start vector is random: never replaced)
  it.colscale[j + 1] = (ok && beta > 0.0) ? 1.0 / beta : 0.0;
  if (j < 0) return;
  const double coupling = ok ? beta : 0.0;
  if (j + 1 < st->k) it.B[j + (int64_t)it.ldb * (j + 1)] = coupling;
  else st->beta_k = coupling;
  if (ok) { if (beta > st->anorm) st->anorm = beta; }
  else st->breakdown += 1;
  st->jc = j + 1;   // last kernel of the step: the next step of this problem
}

// ------------------------------------------------------------ small SVD
// One-sided (Hestenes) Jacobi on the columns of W = B (k x k): rotate column
// pairs until all are orthogonal; sigma_i are the final column norms and
// P_i = W_i / sigma_i the left singular vectors.  The right vectors follow as
// Q = W0^T P diag(1/sigma) from the original matrix W0.
// When k equals the short dimension the short basis is complete and
// A = U_k [B | beta_k e_k] V_{k+1}^T holds exactly, so W gets that extra
// column and the singular values are exact (no restart needed).
//
// GB300 runs FP64 at two lanes per clock per SM and FP32 at 128, so the
// rotations are found in FP32 and FP64 only polishes them:
//  1. FP32 Jacobi on a copy of W0 scaled by a power of two, accumulating the
//     rotations in V (nc x nc), until every pair's cosine is at the rounding
//     level of an FP32 dot product;
//  2. one Newton-Schulz step makes V orthogonal in FP64: V' = V - V E / 2
//     with E = V^T V - I summed in FP64 (products of FP32 entries are exact
//     in FP64); V E is of the size of E and needs only FP32.  This leaves
//     |V'^T V' - I| ~ 3|E|^2 / 4;
//  3. W = W0 V' in FP64 (W0 is upper triangular with a few nonzeros per
//     row: bidiagonal plus the restart column), and the FP64 Jacobi below
//     runs on W.  Its columns start orthogonal to FP32 level, so it needs
//     about two sweeps and a check sweep where it needs nine from W0.
// W0 V' J = P Sigma with V' J orthogonal to FP64 rounding is an SVD of W0,
// so sigma, P and Q are FP64-accurate whatever the FP32 steps did (they only
// decide how many FP64 sweeps remain).  The FP32 form runs step 3's sweeps
// and what follows in float-float instead (bsvd_tail_ff), to its tolerance.
//
// In the FP64 sweeps one thread owns one column pair of a round-robin round
// (dot product, rotation parameters, column update), the squared column norms
// are carried by the exact Jacobi update (a' = a - t g, b' = b + t g) and
// refreshed once per sweep, and no rotation is accumulated (Q is formed once
// at the end).
// Outputs: sig (k), P (k x k, ld ldb), Q ((k+1) x k, ld ldb+1; row k is zero
// unless the extra column was used).
constexpr int BSVD_NT = 512;
constexpr int BSVD_T32 = 16;   // lanes per column pair in the FP32 sweeps (latency-bound: many lanes)
constexpr int BSVD_T64 = 4;    // lanes per column pair in the FP64 sweeps (FP64 issue-bound: few lanes,
                               // so the per-pair scalar work is repeated by few warps)

// sqrt of a non-negative FP32 value from the hardware reciprocal square root
__device__ __forceinline__ float sqrt_approx(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }

__device__ __forceinline__ double block_max(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; ++i) t = fmax(t, red[i]);
  return t;
}

// column pair of team t in round rd of the round-robin order over n2 slots
// (n2 even; slots >= nc are empty): -1 when the team has no pair
// (rd < n2 - 1 and slot <= n2 - 1, so slot - 1 + rd < 2 (n2 - 1): the
// remainder is one conditional subtraction, not an integer division)
__device__ __forceinline__ void jacobi_pair(int t, int rd, int n2, int nc, int& a, int& b) {
  a = b = -1;
  if (t >= n2 / 2) return;
  const int m = n2 - 1, sa = t, sb = n2 - 1 - t;
  int xa = sa - 1 + rd, xb = sb - 1 + rd;
  xa -= xa >= m ? m : 0;
  xb -= xb >= m ? m : 0;
  a = (sa == 0) ? 0 : 1 + xa;
  b = (sb == 0) ? 0 : 1 + xb;
  if (a >= nc || b >= nc) a = b = -1;
}

// FP32 form: the polish of k_bsvd (from W = W0 V' on) in float-float
// arithmetic on the FP32 pipes instead of FP64 -- the one-sided Jacobi
// sweeps, the column norms, the Newton-Schulz step on the left vectors and
// the products for Q.  A phase-stamped build of k_bsvd put the FP64 sweeps
// at half its time (1.5 M of 3.1 M cycles at batch 456), paced by GB300's
// FP64 pipe whether a round rotated or only tested.  Float-float carries
// about 48 bits, far inside the sweeps' stopping cosine (jtol = 1e-10 in
// this form) and the left vectors' orthogonality after the Newton-Schulz
// step.  W is scaled by a power of two (largest entry in [1, 2)) before the
// split, so that FP32 exponents hold it, and the norms are scaled back.
// Rotations: the tangent t in FP32 from the float-float norms and dot
// product (as in the FP64 form, the next sweep removes what an FP32 angle
// leaves), the cosine and sine in float-float from t -- 1 - t^2 / 2 below
// |t| = 1e-4 (the next term is below 4e-17), else 1 / sqrt(1 + t^2) by one
// Newton step on rsqrtf -- so each rotation is orthogonal to float-float
// rounding.  Teams of 16 lanes per column pair, as in the FP32 sweeps.
__device__ void bsvd_tail_ff(const SvdItem& it, LzState* st, int k, int nc, bool aug, int cs, int lv, double* W,
                             const double* bp, int bld, float jtol, int nkeep_fast, int sweeps32, double* sm,
                             double* nrm2d, double* nrm, int* order, unsigned char* keep, int* rotated) {
  float2* W2 = reinterpret_cast<float2*>(W);   // column c at W2 + c * cs (the FP64 layout)
  float2* nrm2 = reinterpret_cast<float2*>(nrm2d);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int team = lane / BSVD_T32, q = lane % BSVD_T32;
  const int nteams = nw * (32 / BSVD_T32);
  const int n2 = nc + (nc & 1);
  __shared__ int ex_s;

  // 1. scale: the largest |W| as a bit pattern (non-negative doubles order like
  //    their patterns), its binary exponent, then W 2^-ex split in place
  {
    long long mb = 0;
    for (int e = threadIdx.x; e < k * nc; e += blockDim.x) {
      const int c = e / k, i = e - c * k;
      const long long b = __double_as_longlong(W[c * cs + i]) & 0x7FFFFFFFFFFFFFFFll;
      mb = b > mb ? b : mb;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long v = __shfl_xor_sync(0xffffffffu, mb, o);
      mb = v > mb ? v : mb;
    }
    if (threadIdx.x == 0) ex_s = 0;
    __syncthreads();
    if (lane == 0) atomicMax(&ex_s, (int)((mb >> 52) & 0x7FF));   // exponent field of the largest entry
    __syncthreads();
  }
  const int ex = ex_s > 0 ? ex_s - 1023 : 0;   // W 2^-ex has its largest entry in [1, 2)
  for (int e = threadIdx.x; e < k * nc; e += blockDim.x) {
    const int c = e / k, i = e - c * k;
    W2[c * cs + i] = ff_from_double_scaled(W[c * cs + i], ex);
  }
  __syncthreads();

  // 2. sweeps
  int sweeps = 0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    sweeps = sweep + 1;
    const int nkeep = sweep < 6 ? nkeep_fast : nc;
    for (int c = warp; c < nc; c += nw) {
      const float2* w = W2 + c * cs;
      ffacc a;
      for (int i = lane; i < k; i += 32) a.fma(w[i], w[i]);
      const ff v = warp_sum_ff(a).value();
      if (lane == 0) nrm2[c] = make_float2(v.hi, v.lo);
    }
    __syncthreads();
    // ranks by the hi parts (non-negative floats order like their patterns)
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      const int v = __float_as_int(nrm2[c].x);
      int rk = 0;
      for (int b = 0; b < nc; ++b) {
        const int u = __float_as_int(nrm2[b].x);
        rk += (u > v) || (u == v && b < c);
      }
      keep[c] = rk < nkeep;
    }
    if (threadIdx.x == 0) *rotated = 0;
    __syncthreads();
    for (int rd = 0; rd < n2 - 1; ++rd) {
      for (int t0 = warp * (32 / BSVD_T32); t0 < n2 / 2; t0 += nteams) {
        int a, b;
        jacobi_pair(t0 + team, rd, n2, nc, a, b);
        if (a >= 0 && !keep[a] && !keep[b]) a = b = -1;
        float2* __restrict__ wa = W2 + (a < 0 ? 0 : a) * cs;
        float2* __restrict__ wb = W2 + (b < 0 ? 0 : b) * cs;
        ffacc g;
        if (a >= 0)
          for (int i = q; i < k; i += BSVD_T32) g.fma(wa[i], wb[i]);
        const ff ga = team_sum_ff<BSVD_T32>(g).value();
        bool rot = false;
        float tt = 0.0f;
        ff al{0.0f, 0.0f}, be{0.0f, 0.0f};
        if (a >= 0) {
          al = ff{nrm2[a].x, nrm2[a].y};
          be = ff{nrm2[b].x, nrm2[b].y};
          rot = ga.hi != 0.0f && al.hi > 0.0f && be.hi > 0.0f && fabsf(ga.hi) > jtol * sqrtf(al.hi) * sqrtf(be.hi);
        }
        if (rot) {
          const float dz = ff_add(be, ff_neg(al)).hi, g2 = 2.0f * ga.hi;
          const float zeta = dz / g2, az = fabsf(zeta);
          tt = az > 1e18f ? 0.5f / zeta : copysignf(1.0f, zeta) / (az + sqrtf(fmaf(zeta, zeta, 1.0f)));
          if (!(fabsf(tt) > 0.0f && fabsf(tt) <= 2.0f)) rot = false;
        }
        if (rot) {
          ff cn;
          float p2, e2;                   // t^2 = p2 + e2 exactly
          p2 = tt * tt;
          e2 = __fmaf_rn(tt, tt, -p2);
          if (fabsf(tt) < 1e-4f) {
            cn = ff_add(ff{1.0f, 0.0f}, ff{-0.5f * p2, -0.5f * e2});
          } else {
            const ff x = ff_add(ff{1.0f, 0.0f}, ff{p2, e2});      // 1 + t^2
            const float y0 = rsqrtf(x.hi);
            const ff r = ff_mul(x, ff_mul(ff{y0, 0.0f}, ff{y0, 0.0f}));
            const float er = ff_add(ff{1.0f, 0.0f}, ff_neg(r)).hi;   // 1 - x y0^2, near FP32 rounding
            cn = ff_add(ff{y0, 0.0f}, ff{0.5f * y0 * er, 0.0f});
          }
          const ff sn = ff_mul(cn, ff{tt, 0.0f});
          for (int m = q; m < k; m += BSVD_T32) {
            const ff x{wa[m].x, wa[m].y}, y{wb[m].x, wb[m].y};
            const ff xa = ff_add(ff_mul(cn, x), ff_neg(ff_mul(sn, y)));
            const ff yb = ff_add(ff_mul(sn, x), ff_mul(cn, y));
            wa[m] = make_float2(xa.hi, xa.lo);
            wb[m] = make_float2(yb.hi, yb.lo);
          }
        }
        __syncwarp();   // every lane of the team has read the old norms
        if (rot && q == 0) {
          const ff tg = ff_mul(ff{tt, 0.0f}, ga);
          const ff na = ff_add(al, ff_neg(tg)), nb = ff_add(be, tg);
          nrm2[a] = make_float2(na.hi, na.lo);
          nrm2[b] = make_float2(nb.hi, nb.lo);
          *rotated = 1;
        }
      }
      __syncthreads();
    }
    const int any = *rotated;
    __syncthreads();
    if (!any) break;
  }

  // 3. norms (scaled back), order, 1 / sigma; columns normalised in place
  double* inv = nrm2d;                 // reused: the squared norms are dead
  __shared__ float2 invs[KMAX + 2];    // 1 / (scaled norm) as float-float
  for (int c = warp; c < nc; c += nw) {
    const float2* w = W2 + c * cs;
    ffacc a;
    for (int i = lane; i < k; i += 32) a.fma(w[i], w[i]);
    const ff v = warp_sum_ff(a).value();
    if (lane == 0) {
      const double ns = sqrt(fmax(ff_to_double(make_float2(v.hi, v.lo)), 0.0));   // scaled norm
      nrm[c] = ldexp(ns, ex);
      invs[c] = ns > 0.0 ? ff_from_double(1.0 / ns) : make_float2(0.0f, 0.0f);
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    const long long v = __double_as_longlong(nrm[c]);
    int rk = 0;
    for (int b = 0; b < nc; ++b) {
      const long long u = __double_as_longlong(nrm[b]);
      rk += (u > v) || (u == v && b < c);
    }
    order[rk] = c;
    inv[c] = nrm[c] > 0.0 ? 1.0 : 0.0;      // a nonzero flag (Q uses invs)
  }
  for (int e = threadIdx.x; e < nc * k; e += blockDim.x) {
    const int c = e / k, i = e - c * k;
    const ff p = ff_mul(ff{W2[c * cs + i].x, W2[c * cs + i].y}, ff{invs[c].x, invs[c].y});
    W2[c * cs + i] = make_float2(p.hi, p.lo);
  }
  __syncthreads();

  // 4. one Newton-Schulz step on the left vectors P: P - P F / 2 with
  //    F = P^T P - I summed in float-float (F is of the size of jtol, so P F in FP32)
  {
    float* F32 = reinterpret_cast<float*>(sm);                   // nc x lv
    float* P32 = F32 + (size_t)nc * lv;                           // nc x cs
    for (int e = threadIdx.x; e < nc * k; e += blockDim.x) {
      const int c = e / k, i = e - c * k;
      P32[c * cs + i] = W2[c * cs + i].x;
    }
    // upper triangle a <= b, one pair per thread (a whole float-float dot
    // product each: no reductions across lanes)
    {
      const int npair = nc * (nc + 1) / 2;
      int a = 0, rem = threadIdx.x, len = nc;
      while (a < nc && rem >= len) { rem -= len; ++a; --len; }
      for (int e = threadIdx.x; e < npair; e += blockDim.x) {
        const int b = a + rem;
        const float2* pa = W2 + a * cs;
        const float2* pb = W2 + b * cs;
        ffacc f0, f1;
        int i = 0;
        for (; i + 1 < k; i += 2) { f0.fma(pa[i], pb[i]); f1.fma(pa[i + 1], pb[i + 1]); }
        if (i < k) f0.fma(pa[i], pb[i]);
        f0.add(f1);
        const float fv = ff_add(f0.value(), ff{a == b ? -1.0f : 0.0f, 0.0f}).hi;
        F32[b * lv + a] = fv;
        F32[a * lv + b] = fv;
        rem += blockDim.x;
        while (a < nc && rem >= len) { rem -= len; ++a; --len; }
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nc * k; e += blockDim.x) {
      const int c = e / k, i = e - c * k;
      float acc = 0.0f;
      for (int jj = 0; jj < nc; ++jj) acc = fmaf(P32[jj * cs + i], F32[c * lv + jj], acc);
      const ff p = ff_add(ff{W2[c * cs + i].x, W2[c * cs + i].y}, ff{-0.5f * acc, 0.0f});
      W2[c * cs + i] = make_float2(p.hi, p.lo);
    }
    __syncthreads();
  }

  // 5. outputs: P_i = W_{o(i)}, sigma, Q_i = W0^T P_i / sigma_i
  const int kd = it.ldb, kq = it.ldb + 1;
  for (int e = threadIdx.x; e < kd * kd; e += blockDim.x) {
    const int c = e / kd, i = e - c * kd;
    double pv = 0.0;
    if (c < k && i < k) pv = ff_to_double(W2[order[c] * cs + i]);
    it.P[i + (int64_t)kd * c] = pv;
  }
  for (int c = threadIdx.x; c < kd; c += blockDim.x) it.sig[c] = (c < k) ? nrm[order[c]] : 0.0;
  // first nonzero row of each column of B (upper triangular, a few nonzeros
  // per column; the restart's arrow column reaches row 0)
  __shared__ int bfirst[KMAX + 1];
  for (int jj = threadIdx.x; jj < k; jj += blockDim.x) {
    const double* bc = bp + (int64_t)bld * jj;
    int m = 0;
    while (m < jj && (__double_as_longlong(bc[m]) << 1) == 0) ++m;
    bfirst[jj] = m;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kq * kd; e += blockDim.x) {
    const int c = e / kq, j = e - c * kq;
    double qv = 0.0;
    if (c < k && j < nc) {
      const int o = order[c];
      if (inv[o] > 0.0) {
        const float2* pc = W2 + o * cs;        // P column
        ffacc acc;
        if (j < k) {
          const double* bc = bp + (int64_t)bld * j;
          for (int m = bfirst[j]; m <= j && m < k; ++m) {
            const double bv = bc[m];
            if ((__double_as_longlong(bv) << 1) != 0) acc.fma(ff_from_double_scaled(bv, ex), pc[m]);
          }
        } else {
          acc.fma(ff_from_double_scaled(st->beta_k, ex), pc[k - 1]);
        }
        // (B 2^-ex) P_i / (sigma_i 2^-ex): the scaled norm's inverse invs
        const ff av = ff_mul(acc.value(), ff{invs[o].x, invs[o].y});
        qv = ff_to_double(make_float2(av.hi, av.lo));
      }
    }
    it.Q[j + (int64_t)kq * c] = qv;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int r = min(st->r, k);
    const double s1 = nrm[order[0]], is1 = s1 > 0.0 ? 1.0 / s1 : 0.0;
    double mres = 0.0;
    int nconv = 0;
    bool conv = true;
    for (int i = 0; i < r; ++i) {
      const int o = order[i];
      const double pk = ff_to_double(W2[o * cs + (k - 1)]);
      const double res = aug ? 0.0 : fabs(st->beta_k * pk);
      const double rel = res * is1;
      if (rel > mres) mres = rel;
      if (rel <= st->tol) { if (nconv == i) ++nconv; }
      else conv = false;
    }
    if (st->full) { conv = true; nconv = r; }
    st->sigma1 = s1;
    st->maxres = mres;
    st->sweeps = sweeps;
    st->sweeps32 = sweeps32;
    st->nconv = nconv;
    st->converged = conv ? 1 : 0;
    st->restarts += 1;
    st->svd_done = 1;
    if (conv || st->restarts > st->max_restarts) st->active = 0;
  }
}

__global__ void __launch_bounds__(BSVD_NT, 2) k_bsvd(const SvdItem* __restrict__ items, int b_in_smem) {
  const SvdItem it = items[blockIdx.x];
  LzState* st = it.st;
  if (!st->active || st->jc < st->k || st->svd_done) return;   // only at the end of a cycle, once
  const int k = st->k, ld = it.ldb;
  const bool aug = st->full != 0;
  const int nc = aug ? k + 1 : k;       // columns of W
  const BsvdLayout lay = bsvd_layout(k, nc);
  const int cs = lay.cs, lv = lay.lv, s0 = lay.s0;
  extern __shared__ __align__(16) double sm[];
  float* W32 = reinterpret_cast<float*>(sm);                    // step 1, column c at W32 + c*cs
  double* V64 = sm;                                             // step 2, column c at V64 + c*s0
  float* V32 = reinterpret_cast<float*>(sm + (size_t)nc * s0);  // column c at V32 + c*lv
  float* E32 = V32 + (size_t)nc * lv;
  double* W = sm + (size_t)nc * s0;                              // step 3 on, over V32 and E32; column c at W + c*cs
  // B for the products with W0: a shared copy (region 2) or global memory
  double* Bs = b_in_smem ? W + (size_t)nc * lv : nullptr;       // region 2, column m at Bs + m*cs
  const double* bp = b_in_smem ? Bs : it.B;
  const int bld = b_in_smem ? cs : ld;
  __shared__ int rotated;
  __shared__ int ns_bad;
  __shared__ double nrm2[KMAX + 2];
  __shared__ double nrm[KMAX + 2];
  __shared__ float nrm2f[KMAX + 2];
  __shared__ int order[KMAX + 2];
  __shared__ unsigned char keep[KMAX + 2];
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int team = lane / BSVD_T64, q = lane % BSVD_T64;        // FP64 sweeps
  const int nteams = (blockDim.x >> 5) * (32 / BSVD_T64);
  const int team16 = lane / BSVD_T32, q16 = lane % BSVD_T32;    // FP32 sweeps
  const int nteams16 = (blockDim.x >> 5) * (32 / BSVD_T32);
  const int n2 = nc + (nc & 1);

  if (b_in_smem) {
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
      const int m = e / k, i = e - m * k;
      Bs[m * cs + i] = (i <= m) ? it.B[i + (int64_t)ld * m] : 0.0;
    }
  }
  // ---- step 1: FP32 Jacobi with accumulated rotations
  double mx = 0.0;
  for (int e = threadIdx.x; e < nc * k; e += blockDim.x) {
    const int c = e / k, i = e - c * k;
    const double v = (c < k) ? it.B[i + (int64_t)ld * c] : ((i == k - 1) ? st->beta_k : 0.0);
    mx = fmax(mx, fabs(v));
  }
  mx = block_max(mx, red);
  double scale = 1.0;
  if (mx > 0.0) {
    int ex = ((__double2hiint(mx) >> 20) & 0x7ff) - 1023;
    ex = ex > 1022 ? 1022 : ex;
    scale = __hiloint2double((1023 - ex) << 20, 0);          // 2^-ex: entries below 2 in magnitude
  }
  for (int e = threadIdx.x; e < nc * k; e += blockDim.x) {
    const int c = e / k, i = e - c * k;
    const double v = (c < k) ? it.B[i + (int64_t)ld * c] : ((i == k - 1) ? st->beta_k : 0.0);
    W32[c * cs + i] = (float)(v * scale);
  }
  for (int e = threadIdx.x; e < nc * nc; e += blockDim.x) {
    const int c = e / nc, m = e - c * nc;
    V32[c * lv + m] = (m == c) ? 1.0f : 0.0f;
  }
  if (threadIdx.x == 0) ns_bad = 0;
  __syncthreads();
  const float tol32 = 1.1920929e-7f * (float)(k > 8 ? k : 8);
  int sweeps32 = 0;
  for (int sweep = 0; sweep < 30; ++sweep) {
    sweeps32 = sweep + 1;
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      const float* w = W32 + c * cs;
      float a0 = 0.0f, a1 = 0.0f;
      int i = 0;
      for (; i + 1 < k; i += 2) { a0 = fmaf(w[i], w[i], a0); a1 = fmaf(w[i + 1], w[i + 1], a1); }
      if (i < k) a0 = fmaf(w[i], w[i], a0);
      nrm2f[c] = a0 + a1;
    }
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    // FP32 arithmetic is cheap and its rounds are latency-bound: a team of
    // BSVD_T32 lanes owns a pair, so each lane carries a few rows
    for (int rd = 0; rd < n2 - 1; ++rd) {
      for (int t0 = warp * (32 / BSVD_T32); t0 < n2 / 2; t0 += nteams16) {
        int a, b;
        jacobi_pair(t0 + team16, rd, n2, nc, a, b);
        float* __restrict__ wa = W32 + (a < 0 ? 0 : a) * cs;
        float* __restrict__ wb = W32 + (b < 0 ? 0 : b) * cs;
        float g0 = 0.0f, g1 = 0.0f;
        if (a >= 0) {
          int i = q16;
          for (; i + BSVD_T32 < k; i += 2 * BSVD_T32) {
            g0 = fmaf(wa[i], wb[i], g0);
            g1 = fmaf(wa[i + BSVD_T32], wb[i + BSVD_T32], g1);
          }
          if (i < k) g0 = fmaf(wa[i], wb[i], g0);
        }
        float ga = g0 + g1;
#pragma unroll
        for (int o = 1; o < BSVD_T32; o <<= 1) ga += __shfl_xor_sync(0xffffffffu, ga, o);
        bool rot = false;
        float tt = 0.0f, al = 0.0f, be = 0.0f;
        if (a >= 0) {
          al = nrm2f[a];
          be = nrm2f[b];
          // columns that vanished (or whose squared norms underflowed) are
          // left alone: their dot products are below FP32 resolution
          rot = ga != 0.0f && al > 0.0f && be > 0.0f && fabsf(ga) > tol32 * sqrt_approx(al) * sqrt_approx(be);
        }
        if (rot) {
          // approximate division and square roots: the FP64 steps make the
          // result exact whatever these rotations are
          const float zeta = __fdividef(be - al, 2.0f * ga), az = fabsf(zeta);
          tt = az > 1e18f ? __fdividef(0.5f, zeta)
                          : __fdividef(copysignf(1.0f, zeta), az + sqrt_approx(fmaf(zeta, zeta, 1.0f)));
          // |t| <= 1 for the inner rotation; a denormal divisor in the
          // approximate division can give 0, inf or NaN instead: no rotation
          if (!(fabsf(tt) > 0.0f && fabsf(tt) <= 2.0f)) rot = false;
        }
        if (rot) {
          const float cn = rsqrtf(fmaf(tt, tt, 1.0f)), sn = cn * tt;
          for (int m = q16; m < k; m += BSVD_T32) {
            const float x = wa[m], y = wb[m];
            wa[m] = cn * x - sn * y;
            wb[m] = sn * x + cn * y;
          }
          float* __restrict__ va = V32 + a * lv;
          float* __restrict__ vb = V32 + b * lv;
          for (int m = q16; m < nc; m += BSVD_T32) {
            const float x = va[m], y = vb[m];
            va[m] = cn * x - sn * y;
            vb[m] = sn * x + cn * y;
          }
        }
        __syncwarp();   // every lane of the team has read the old norms
        if (rot && q16 == 0) {
          nrm2f[a] = al - tt * ga;
          nrm2f[b] = be + tt * ga;
          rotated = 1;
        }
      }
      __syncthreads();
    }
    const int any = rotated;
    __syncthreads();
    if (!any) break;
  }

  // ---- step 2: V' = V - V E / 2, E = V^T V - I (W32 is dead: V64 takes its place)
  for (int e = threadIdx.x; e < nc * nc; e += blockDim.x) {
    const int c = e / nc, m = e - c * nc;
    V64[c * s0 + m] = (double)V32[c * lv + m];
  }
  __syncthreads();
  {
    // upper triangle a <= b, row by row; each thread walks its share in steps of blockDim.x
    const int npair = nc * (nc + 1) / 2;
    int a = 0, rem = threadIdx.x, len = nc;
    while (a < nc && rem >= len) { rem -= len; ++a; --len; }
    for (int e = threadIdx.x; e < npair; e += blockDim.x) {
      const int b = a + rem;
      const double* va = V64 + a * s0;
      const double* vb = V64 + b * s0;
      double e0 = 0.0, e1 = 0.0;
      int m = 0;
      for (; m + 1 < nc; m += 2) { e0 = fma(va[m], vb[m], e0); e1 = fma(va[m + 1], vb[m + 1], e1); }
      if (m < nc) e0 = fma(va[m], vb[m], e0);
      const double ed = (e0 + e1) - (a == b ? 1.0 : 0.0);
      // one step leaves |V'^T V' - I| ~ 3|E|^2/4: with |E| <= 3e-5 the
      // singular values of W0 V' are those of W0 to 4e-10 (also catches NaN)
      if (!(fabs(ed) <= 3e-5)) ns_bad = 1;
      const float ev = (float)ed;
      E32[b * lv + a] = ev;
      E32[a * lv + b] = ev;
      rem += blockDim.x;
      while (a < nc && rem >= len) { rem -= len; ++a; --len; }
    }
  }
  __syncthreads();
  if (ns_bad) {
    // V too far from orthogonal for one step (the FP32 sweeps went wrong or
    // did not settle): V' = I, and the FP64 sweeps orthogonalise W0 itself
    for (int e = threadIdx.x; e < nc * nc; e += blockDim.x) {
      const int c = e / nc, m = e - c * nc;
      V64[c * s0 + m] = (m == c) ? 1.0 : 0.0;
    }
  } else {
    for (int e = threadIdx.x; e < nc * nc; e += blockDim.x) {
      const int c = e / nc, m = e - c * nc;
      float acc = 0.0f;
      for (int j = 0; j < nc; ++j) acc = fmaf(V32[j * lv + m], E32[c * lv + j], acc);
      V64[c * s0 + m] -= 0.5 * (double)acc;
    }
  }
  __syncthreads();

  // ---- step 3: W = W0 V' (V32 and E32 are dead: W takes their place)
  for (int e = threadIdx.x; e < k * nc; e += blockDim.x) {
    const int i = e / nc, c = e - i * nc;
    const double* vc = V64 + c * s0;
    double acc = 0.0;
    for (int m = i; m < k; ++m) {         // B is upper triangular; zeros skipped by their bits
      const double b = bp[i + (int64_t)bld * m];
      if ((__double_as_longlong(b) << 1) != 0) acc = fma(b, vc[m], acc);
    }
    if (aug && i == k - 1) acc = fma(st->beta_k, vc[k], acc);   // the extra column of W0
    W[c * cs + i] = acc;
  }
  __syncthreads();
  // a pair is done once its cosine is at the rounding level of a k-term FP64
  // dot product (k eps; tighter never settles) or at 1e-3 of the residual
  // tolerance, whichever is larger: with cosines below c the singular values
  // are within a relative k c and the vectors orthogonal to c, far inside
  // what the residual test and the FP32 products resolve (FP32 form: tol
  // 1e-7, so 1e-10, and the sweeps after the first one only test)
  const double keps = 2.220446049250313e-16 * (double)(k > 8 ? k : 8);
  const bool relaxed = 1e-3 * st->tol > keps;
  const double jtol = relaxed ? 1e-3 * st->tol : keps;
  // FP32 form: pairs of two trailing columns are not rotated (below) -- for
  // the first sweeps only: when the trailing columns are nearly dependent
  // (a long cycle leaves B with singular values far below eps ||B||) the
  // leading ones never settle against them that way, and the FP64 sweeps
  // started from B itself (after a failed Newton-Schulz step) ran to the
  // sweep limit at k = 112; all pairs then converge in about ten sweeps
  const int nkeep_fast = relaxed ? min(nc, max(st->kk, st->r) + 4) : nc;
  if (it.ffpolish && relaxed) {
    bsvd_tail_ff(it, st, k, nc, aug, cs, lv, W, bp, bld, (float)jtol, nkeep_fast, sweeps32, sm, nrm2, nrm, order, keep,
                 &rotated);
    return;
  }
  int sweeps = 0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    sweeps = sweep + 1;
    const int nkeep = sweep < 6 ? nkeep_fast : nc;
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      const double* w = W + c * cs;
      double a0 = 0.0, a1 = 0.0;
      int i = 0;
      for (; i + 1 < k; i += 2) { a0 = fma(w[i], w[i], a0); a1 = fma(w[i + 1], w[i + 1], a1); }
      if (i < k) a0 = fma(w[i], w[i], a0);
      nrm2[c] = a0 + a1;
    }
    __syncthreads();
    // Only the leading kk triples are used (restart, Ritz vectors, residual
    // test), so in the FP32 form a pair of two columns ranked below kk + 4 by
    // norm is left alone: those columns need not be orthogonal to each other,
    // only to the leading ones, and their own norms are off by no more than
    // the FP32 sweeps left (~1e-6 relative), far from the leading ranks.
    // This skips the slowly converging noise clusters.
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      const long long v = __double_as_longlong(nrm2[c]);
      int rk = 0;
      for (int b = 0; b < nc; ++b) {
        const long long u = __double_as_longlong(nrm2[b]);
        rk += (u > v) || (u == v && b < c);
      }
      keep[c] = rk < nkeep;
    }
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    // A team of BSVD_T64 lanes owns one column pair (rows interleaved over the
    // team); teams fill whole warps, so a round's FP64 instructions run with
    // full warps on every scheduler of the SM.
    for (int rd = 0; rd < n2 - 1; ++rd) {
      for (int t0 = warp * (32 / BSVD_T64); t0 < n2 / 2; t0 += nteams) {
        int a, b;
        jacobi_pair(t0 + team, rd, n2, nc, a, b);
        if (a >= 0 && !keep[a] && !keep[b]) a = b = -1;
        double* __restrict__ wa = W + (a < 0 ? 0 : a) * cs;
        double* __restrict__ wb = W + (b < 0 ? 0 : b) * cs;
        double g0 = 0.0, g1 = 0.0;
        if (a >= 0) {
          int i = q;
          for (; i + BSVD_T64 < k; i += 2 * BSVD_T64) {
            g0 = fma(wa[i], wb[i], g0);
            g1 = fma(wa[i + BSVD_T64], wb[i + BSVD_T64], g1);
          }
          if (i < k) g0 = fma(wa[i], wb[i], g0);
        }
        double ga = g0 + g1;
#pragma unroll
        for (int o = 1; o < BSVD_T64; o <<= 1) ga += __shfl_xor_sync(0xffffffffu, ga, o);
        bool rot = false, small = false;
        double tt = 0.0, al = 0.0, be = 0.0;
        if (a >= 0) {
          al = nrm2[a];
          be = nrm2[b];
          // a pair is done once its cosine is below jtol
          rot = ga != 0.0 && ga * ga > jtol * jtol * (al * be);
        }
        if (rot) {
          // Tangent of the angle from zeta = (be - al) / (2 ga), formed in FP32
          // after scaling both terms by one power of two: an FP32 angle leaves
          // a ~1e-7 relative residual in the pair, which the next sweep
          // removes, and saves most of the FP64 instructions of a round.
          // Angles below FP32 resolution take the FP64 formula.  Cosine and
          // sine follow in FP64 from that tangent, so the rotation is
          // orthogonal to FP64 rounding whatever its angle.
          const double dz = be - al, g2 = 2.0 * ga;
          const double mx = fmax(fabs(dz), fabs(g2));
          int ex = ((__double2hiint(mx) >> 20) & 0x7ff) - 1023;
          ex = ex > 1022 ? 1022 : ex;
          const double sc = __hiloint2double((1023 - ex) << 20, 0);     // 2^-ex
          const float zn = (float)(dz * sc), zd = (float)(g2 * sc);
          float tf = 0.0f;
          if (zd != 0.0f) {
            const float zf = zn / zd, az = fabsf(zf);
            if (az < 1e18f) tf = copysignf(1.0f, zf) / (az + sqrtf(fmaf(zf, zf, 1.0f)));
          }
          small = tf != 0.0f && fabsf(tf) < 1e-4f;
          if (tf != 0.0f) {
            tt = (double)tf;
          } else {
            const double zeta = dz / g2;
            const double az = fabs(zeta);
            tt = az > 1e150 ? 0.5 / zeta : copysign(1.0, zeta) / (az + sqrt(1.0 + zeta * zeta));
          }
          if (!(fabs(tt) > 0.0 && fabs(tt) <= 2.0)) rot = false;
        }
        if (rot) {
          // |t| < 1e-4 (the polish after the FP32 sweeps): 1 / sqrt(1 + t^2)
          // = 1 - t^2 / 2 to FP64 rounding (the next term, 3 t^4 / 8, is below
          // 4e-17), so the rotation stays orthogonal without the square root
          const double cn = small ? fma(-0.5 * tt, tt, 1.0) : rsqrt(1.0 + tt * tt), sn = cn * tt;
          int m = q;
          for (; m + BSVD_T64 < k; m += 2 * BSVD_T64) {
            const double x0 = wa[m], x1 = wa[m + BSVD_T64];
            const double y0 = wb[m], y1 = wb[m + BSVD_T64];
            wa[m] = cn * x0 - sn * y0; wa[m + BSVD_T64] = cn * x1 - sn * y1;
            wb[m] = sn * x0 + cn * y0; wb[m + BSVD_T64] = sn * x1 + cn * y1;
          }
          for (; m < k; m += BSVD_T64) {
            const double x = wa[m], y = wb[m];
            wa[m] = cn * x - sn * y;
            wb[m] = sn * x + cn * y;
          }
        }
        __syncwarp();   // every lane of the team has read the old norms
        if (rot && q == 0) {
          nrm2[a] = al - tt * ga;
          nrm2[b] = be + tt * ga;
          rotated = 1;
        }
      }
      __syncthreads();
    }
    const int any = rotated;
    __syncthreads();
    if (!any) break;
  }
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    const double* w = W + c * cs;
    double a0 = 0.0;
    for (int i = 0; i < k; ++i) a0 = fma(w[i], w[i], a0);
    nrm[c] = sqrt(a0);
  }
  __syncthreads();
  // descending order of the norms, ties by column: each column counts the
  // columns ahead of it (non-negative doubles order like their bit patterns,
  // so the comparisons stay off the FP64 pipe); 1 / sigma once per column
  double* inv = nrm2;
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    const long long v = __double_as_longlong(nrm[c]);
    int rk = 0;
    for (int b = 0; b < nc; ++b) {
      const long long u = __double_as_longlong(nrm[b]);
      rk += (u > v) || (u == v && b < c);
    }
    order[rk] = c;
    inv[c] = nrm[c] > 0.0 ? 1.0 / nrm[c] : 0.0;
  }
  __syncthreads();
  // W <- W diag(1 / sigma): the left vectors, unsorted
  for (int e = threadIdx.x; e < nc * k; e += blockDim.x) {
    const int c = e / k, i = e - c * k;
    W[c * cs + i] *= inv[c];
  }
  __syncthreads();
  if (relaxed) {
    // The sweeps stopped at cosines below jtol > k eps: one Newton-Schulz step
    // P <- P - P F / 2, F = P^T P - I (summed in FP64), brings the left vectors
    // to orthogonality at FP64 rounding, which the restarted short basis U P
    // needs (zero columns stay zero).  F is of the size of jtol, so P F needs
    // only FP32.  Region 0 (V') is free: F and an FP32 copy of P go there.
    float* F32 = reinterpret_cast<float*>(sm);                   // nc x lv
    float* P32 = F32 + (size_t)nc * lv;                           // nc x cs
    for (int e = threadIdx.x; e < nc * k; e += blockDim.x) {
      const int c = e / k, i = e - c * k;
      P32[c * cs + i] = (float)W[c * cs + i];
    }
    const int npair = nc * (nc + 1) / 2;
    int a = 0, rem = threadIdx.x, len = nc;
    while (a < nc && rem >= len) { rem -= len; ++a; --len; }
    for (int e = threadIdx.x; e < npair; e += blockDim.x) {
      const int b = a + rem;
      const double* pa = W + a * cs;
      const double* pb = W + b * cs;
      double f0 = 0.0, f1 = 0.0;
      int i = 0;
      for (; i + 1 < k; i += 2) { f0 = fma(pa[i], pb[i], f0); f1 = fma(pa[i + 1], pb[i + 1], f1); }
      if (i < k) f0 = fma(pa[i], pb[i], f0);
      const float fv = (float)((f0 + f1) - (a == b ? 1.0 : 0.0));
      F32[b * lv + a] = fv;
      F32[a * lv + b] = fv;
      rem += blockDim.x;
      while (a < nc && rem >= len) { rem -= len; ++a; --len; }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nc * k; e += blockDim.x) {
      const int c = e / k, i = e - c * k;
      float acc = 0.0f;
      for (int j = 0; j < nc; ++j) acc = fmaf(P32[j * cs + i], F32[c * lv + j], acc);
      W[c * cs + i] -= 0.5 * (double)acc;
    }
    __syncthreads();
  }
  const int kd = ld, kq = ld + 1;
  // P_i = W_{o(i)}
  for (int e = threadIdx.x; e < kd * kd; e += blockDim.x) {
    const int c = e / kd, i = e - c * kd;
    double pv = 0.0;
    if (c < k && i < k) pv = W[order[c] * cs + i];
    it.P[i + (int64_t)kd * c] = pv;
  }
  for (int c = threadIdx.x; c < kd; c += blockDim.x) it.sig[c] = (c < k) ? nrm[order[c]] : 0.0;
  // first nonzero row of each column of B (upper triangular, a few nonzeros
  // per column; the restart's arrow column reaches row 0)
  __shared__ int bfirst[KMAX + 1];
  for (int jj = threadIdx.x; jj < k; jj += blockDim.x) {
    const double* bc = bp + (int64_t)bld * jj;
    int m = 0;
    while (m < jj && (__double_as_longlong(bc[m]) << 1) == 0) ++m;
    bfirst[jj] = m;
  }
  __syncthreads();
  // Q_i = W0^T P_i / sigma_i with W0 = [B | beta_k e_k]
  for (int e = threadIdx.x; e < kq * kd; e += blockDim.x) {
    const int c = e / kq, j = e - c * kq;
    double qv = 0.0;
    if (c < k && j < nc) {
      const int o = order[c];
      const double is = inv[o];
      if (is > 0.0) {
        const double* pc = W + o * cs;         // P column
        double acc = 0.0;
        if (j < k) {
          // B is upper triangular with a few nonzeros per column; zeros are
          // skipped by their bit pattern (no FP64 compare)
          const double* bc = bp + (int64_t)bld * j;
          for (int m = bfirst[j]; m <= j && m < k; ++m) {
            const double bv = bc[m];
            if ((__double_as_longlong(bv) << 1) != 0) acc = fma(bv, pc[m], acc);
          }
        } else {
          acc = st->beta_k * pc[k - 1];
        }
        qv = acc * is;
      }
    }
    it.Q[j + (int64_t)kq * c] = qv;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int r = min(st->r, k);
    const double s1 = nrm[order[0]], is1 = inv[order[0]];
    double mres = 0.0;
    int nconv = 0;
    bool conv = true;
    for (int i = 0; i < r; ++i) {
      const int o = order[i];
      const double pk = W[o * cs + (k - 1)];
      const double res = aug ? 0.0 : fabs(st->beta_k * pk);
      const double rel = res * is1;
      if (rel > mres) mres = rel;
      if (rel <= st->tol) { if (nconv == i) ++nconv; }
      else conv = false;
    }
    if (st->full) { conv = true; nconv = r; }
    st->sigma1 = s1;
    st->maxres = mres;
    st->sweeps = sweeps;
    st->sweeps32 = sweeps32;
    st->nconv = nconv;
    st->converged = conv ? 1 : 0;
    st->restarts += 1;
    st->svd_done = 1;
    if (conv || st->restarts > st->max_restarts) st->active = 0;
  }
}

// B <- [diag(sigma_1..kk) | rho] with rho_i = beta_k P[k-1, i]; jc <- kk.
// Only problems whose cycle ended with a small SVD and go on.
__global__ void k_restart(const SvdItem* __restrict__ items) {
  const SvdItem it = items[blockIdx.x];
  LzState* st = it.st;
  if (!st->active || !st->svd_done) return;
  const int k = st->k, kk = st->kk, ld = it.ldb;
  for (int e = threadIdx.x; e < ld * ld; e += blockDim.x) {
    const int c = e / ld, i = e - c * ld;
    double v = 0.0;
    if (c == i && c < kk) v = it.sig[c];
    else if (c == kk && i < kk) v = st->beta_k * it.P[(k - 1) + (int64_t)ld * i];
    it.B[e] = v;
  }
  // Ritz columns 0..kk-1 are unit vectors; column kk holds the old column k
  for (int c = threadIdx.x; c <= ld; c += blockDim.x)
    if (c < kk) it.colscale[c] = 1.0;
  __syncthreads();
  if (threadIdx.x == 0) {
    it.colscale[kk] = it.colscale[k];
    st->jc = kk;
    st->svd_done = 0;
  }
}

// ------------------------------------------------------------ Ritz vectors
// Long-side coefficients for one restart (or the final pass): Cs[i, c] =
// Q[i, c] * colscale[i] in T (the long basis is stored unnormalised), zero
// for c >= kk; one block per problem.
template <typename T>
__global__ void __launch_bounds__(256) k_ritz_coef(const RitzItem<T>* __restrict__ items, int final_pass) {
  const RitzItem<T> it = items[blockIdx.x];
  const LzState* st = it.st;
  if (!final_pass && (!st->active || !st->svd_done)) return;
  const int k = st->k;
  const int kk = final_pass ? min(st->r, k) : st->kk;
  const int kc = k + 1, cld = it.ldc + 1, ld = it.ldcs;
  for (int e = threadIdx.x; e < kc * ld; e += blockDim.x) {
    const int i = e / ld, c = e - i * ld;
    it.Cs[e] = (c < kk) ? (T)(it.Q[i + (int64_t)cld * c] * it.colscale[i]) : T(0);
  }
}

template <typename E>
__device__ __forceinline__ void lds4(const E* p, E* v) {
  if (sizeof(E) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = (E)q.x; v[1] = (E)q.y; v[2] = (E)q.z; v[3] = (E)q.w;
  } else {
    const double2 q0 = *reinterpret_cast<const double2*>(p);
    const double2 q1 = *reinterpret_cast<const double2*>(p + 2);
    v[0] = (E)q0.x; v[1] = (E)q0.y; v[2] = (E)q1.x; v[3] = (E)q1.y;
  }
}

// In place, by row blocks: basis[:, 0:kk] <- basis[:, 0:kc] C[0:kc, 0:kk]
// (kc = k on the short side, k + 1 on the long side, whose coefficients carry
// the extra row of the complete-basis case); on a restart the long basis also
// moves column k to column kk.  A block stages its RB rows of every column and
// the coefficients in shared memory; thread (rg, cg) accumulates a 4 x CW tile
// (rows 4 rg.., columns CW cg..) from 16-byte shared loads (the basis rows
// differ across a warp, the coefficients are one broadcast), and a warp
// writes 128 consecutive rows of a column.  FP32 takes 4 x 8 tiles: two
// shared loads of the basis per 32 FMA would otherwise bound the kernel.
template <typename T, bool SHORT>
__global__ void __launch_bounds__(256) k_ritz(const RitzItem<T>* __restrict__ items, const int32_t* __restrict__ tpre,
                                              int n, int final_pass) {
  typedef typename std::conditional<SHORT, double, T>::type E;
  constexpr int RB = RITZ_RB<E>();
  constexpr int CW = RITZ_CW<E>();
  constexpr int RG = RB / 4;           // row groups
  constexpr int CP = (256 / RG) * CW;  // columns per pass
  int rblk;
  const RitzItem<T> it = items[tile_item(tpre, n, blockIdx.x, rblk)];
  const LzState* st = it.st;
  if (!final_pass && (!st->active || !st->svd_done)) return;
  const int k = st->k;
  const int kk = final_pass ? min(st->r, k) : st->kk;
  const bool move = !SHORT && !final_pass;
  E* basis = SHORT ? (E*)it.U : (E*)it.V;
  const int64_t ldb = SHORT ? it.ldu : it.ldv;
  const int64_t nrow = SHORT ? it.Ls : it.Kl;
  const int kc = SHORT ? k : k + 1;
  const int64_t r0 = (int64_t)rblk * RB;
  if (r0 >= nrow) return;
  const int nr = (int)imin64(RB, nrow - r0);
  extern __shared__ __align__(16) unsigned char smraw[];
  E* blk = reinterpret_cast<E*>(smraw);               // RB x (k+1), column-major
  const int kkp = ((kk + CP - 1) / CP) * CP;
  E* cf = blk + (int64_t)RB * (k + 1);                 // kc x kkp, row-major in i
  const int ncol = SHORT ? k : k + 1;
  // The block's rows of every basis column and the coefficients arrive by
  // element-wise asynchronous copies: a thread issues all of its copies before
  // waiting, so the whole tile is in flight at once (a load loop through
  // registers keeps one or two per thread).
  for (int e = threadIdx.x; e < ncol * RB; e += blockDim.x) {
    const int c = e / RB, t = e - c * RB;
    if (t < nr) cp_async_elem<sizeof(E)>(blk + e, basis + r0 + t + ldb * c);
    else blk[e] = E(0);
  }
  if (SHORT) {
    for (int e = threadIdx.x; e < kc * kkp; e += blockDim.x) {
      const int i = e / kkp, c = e - i * kkp;
      if (c < kk) cp_async_elem<sizeof(E)>(cf + e, it.P + i + (int64_t)it.ldc * c);
      else cf[e] = E(0);
    }
  } else {
    for (int e = threadIdx.x; e < kc * kkp; e += blockDim.x) {
      const int i = e / kkp, c = e - i * kkp;
      cp_async_elem<sizeof(E)>(cf + e, it.Cs + (int64_t)i * it.ldcs + c);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  const int rg = threadIdx.x % RG, cg = threadIdx.x / RG;
  for (int c0 = 0; c0 < kk; c0 += CP) {
    const int cb = c0 + CW * cg;
    if (cb >= kk) continue;
    E acc[4][CW];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < CW; ++b) acc[a][b] = E(0);
    for (int i = 0; i < kc; ++i) {
      E av[4], bv[CW];
      lds4(blk + i * RB + 4 * rg, av);
#pragma unroll
      for (int h = 0; h < CW; h += 4) lds4(cf + i * kkp + cb + h, bv + h);
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < CW; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
#pragma unroll
    for (int b = 0; b < CW; ++b) {
      const int c = cb + b;
      if (c >= kk) break;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int t = 4 * rg + a;
        if (t < nr) basis[r0 + t + ldb * c] = acc[a][b];
      }
    }
  }
  if (move)
    for (int t = threadIdx.x; t < nr; t += blockDim.x) basis[r0 + t + ldb * kk] = blk[t + (int64_t)RB * k];
}

// ------------------------------------------------------------ outputs
// Sign convention: each pair (U_i, V_i) is flipped so that the entry of U_i
// (the window-side vector) with the largest magnitude is positive (first such
// entry on ties).
template <typename T>
__global__ void __launch_bounds__(256) k_sign(const FinalItem<T>* __restrict__ items) {
  const FinalItem<T> it = items[blockIdx.y];
  const int i = blockIdx.x;
  const int r = it.r;
  if (i >= r) return;
  const int keff = min(it.st->k, r);
  __shared__ double bv[256];
  __shared__ int64_t bi[256];
  double best = -1.0;
  int64_t bidx = 0;
  double bval = 0.0;
  const int64_t n = it.swapped ? it.Kl : it.Ls;
  for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
    const double v = it.swapped ? (double)it.V[t + it.ldv * i] : it.U[t + it.ldu * i];
    if (fabs(v) > best) { best = fabs(v); bidx = t; bval = v; }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = bidx;
  __shared__ double sval[256];
  sval[threadIdx.x] = bval;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      const int u = threadIdx.x + o;
      if (bv[u] > bv[threadIdx.x] || (bv[u] == bv[threadIdx.x] && bi[u] < bi[threadIdx.x])) {
        bv[threadIdx.x] = bv[u]; bi[threadIdx.x] = bi[u]; sval[threadIdx.x] = sval[u];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    it.sgn[i] = (sval[0] < 0.0) ? -1.0 : 1.0;
    it.sigma_out[i] = (i < keff) ? it.sig[i] : 0.0;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_final_copy(const FinalItem<T>* __restrict__ items) {
  const FinalItem<T> it = items[blockIdx.z];
  const int i = blockIdx.y;
  if (i >= it.r) return;
  const bool zero = i >= it.st->k;
  // the sign is +-1: applied in T to the T-typed long basis (no FP64 per
  // element there), in FP64 to the FP64 short basis before its conversion
  const double sg = it.sgn[i];
  const T sgt = (T)sg;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // window side (L) and origin side (K)
  const int64_t L = it.swapped ? it.Kl : it.Ls;
  const int64_t K = it.swapped ? it.Ls : it.Kl;
  for (int64_t t = t0; t < L; t += stride)
    it.Uo[t + L * i] = zero ? T(0) : (it.swapped ? sgt * it.V[t + it.ldv * i] : (T)(sg * it.U[t + it.ldu * i]));
  if (!it.swapped) {
    // the long side: eight loads issued before their stores (one at a time
    // left the copy latency-bound at a third of the copy rate)
    const T* __restrict__ src = it.V + it.ldv * i;
    T* __restrict__ dst = it.Vo + K * i;
    for (int64_t t = t0; t < K; t += 8 * stride) {
      T v[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int64_t x = t + m * stride;
        v[m] = (x < K && !zero) ? src[x] : T(0);
      }
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int64_t x = t + m * stride;
        if (x < K) dst[x] = zero ? T(0) : sgt * v[m];
      }
    }
  } else {
    for (int64_t t = t0; t < K; t += stride)
      it.Vo[t + K * i] = zero ? T(0) : (T)(sg * it.U[t + it.ldu * i]);
  }
}

// ------------------------------------------------------------ launchers
void launch_short_steps(const ShortItem* items, const int32_t* tpre, int n, int tiles, int s, cudaStream_t st) {
  if (n <= 0 || tiles <= 0) return;
  k_short1<<<tiles, SHORT_RB, 0, st>>>(items, tpre, n, s); count_launch();
  k_short23<2><<<tiles, SHORT_RB, 0, st>>>(items, tpre, n, s); count_launch();
  k_short23<3><<<tiles, SHORT_RB, 0, st>>>(items, tpre, n, s); count_launch();
  k_short4<<<tiles, SHORT_RB, 0, st>>>(items, tpre, n, s); count_launch();
}

template <typename T>
void launch_long_step(const LongItem<T>* items, const int32_t* tpre, int n, int tiles, int s, cudaStream_t st) {
  if (n <= 0) return;
  // problems whose step ran inside their X^T u products own no blocks here
  if (tiles > 0) { k_long1<T><<<tiles, 256, 0, st>>>(items, tpre, n, s); count_launch(); }
  k_long_norm<T><<<n, 32, 0, st>>>(items, s); count_launch();
}

template <typename T>
void launch_long_init(const LongItem<T>* items, const int32_t* tpre, int n, int tiles, cudaStream_t st) {
  if (n <= 0 || tiles <= 0) return;
  k_long_init<T><<<tiles, 256, 0, st>>>(items, tpre, n); count_launch();
  k_long_norm<T><<<n, 32, 0, st>>>(items, -1); count_launch();
}

void launch_bsvd(const SvdItem* items, int n, int kmax, cudaStream_t st) {
  if (n <= 0) return;
  const BsvdLayout lay = bsvd_layout(kmax, kmax + 1);
  // B in shared memory when two blocks still fit on an SM
  const int b_in_smem = 2 * (lay.bytes_b + 8192) <= (size_t)device_max_smem() ? 1 : 0;   // (+ static shared memory)
  const size_t sm = b_in_smem ? lay.bytes_b : lay.bytes;
  set_max_smem((const void*)k_bsvd);
  k_bsvd<<<n, BSVD_NT, sm, st>>>(items, b_in_smem); count_launch();
}

void launch_restart(const SvdItem* items, int n, cudaStream_t st) {
  if (n <= 0) return;
  k_restart<<<n, 256, 0, st>>>(items); count_launch();
}

// Short-side Ritz vectors of the FP32 form: U[:, 0:kk] <- U[:, 0:k] P in
// float-float from the basis's (hi, lo) copy, written to the copy and to the
// FP64 basis.  The FP64 product (k_ritz<T, true>) ran on GB300's FP64 pipe;
// a float-float product-sum is about a dozen FP32 instructions.  Tiling as
// k_ritz: 64-row blocks, 4 x 4 register tiles of 16 row groups, 64 columns
// per pass; the block's rows of every column and the coefficients (split
// with integer instructions) are staged in shared memory first, so the
// in-place update is safe.
constexpr int RITZ_FF_RB = 64;
__global__ void __launch_bounds__(256) k_ritz_short_ff(const RitzItem<float>* __restrict__ items,
                                                       const int32_t* __restrict__ tpre, int n, int final_pass) {
  constexpr int RB = RITZ_FF_RB, RG = RB / 4, CP = (256 / RG) * 4;
  int rblk;
  const RitzItem<float> it = items[tile_item(tpre, n, blockIdx.x, rblk)];
  const LzState* st = it.st;
  if (!final_pass && (!st->active || !st->svd_done)) return;
  const int k = st->k;
  const int kk = final_pass ? min(st->r, k) : st->kk;
  const int64_t r0 = (int64_t)rblk * RB;
  if (r0 >= it.Ls) return;
  const int nr = (int)imin64(RB, it.Ls - r0);
  extern __shared__ __align__(16) float2 smr[];
  float2* blk = smr;                                   // RB x k, column-major
  const int kkp = ((kk + CP - 1) / CP) * CP;
  float2* cf = blk + (int64_t)RB * k;                  // k x kkp, row-major in i
  for (int e = threadIdx.x; e < k * RB; e += blockDim.x) {
    const int c = e / RB, t = e - c * RB;
    blk[e] = t < nr ? make_float2(it.Uh[r0 + t + it.ldf * c], it.Ul[r0 + t + it.ldf * c]) : make_float2(0.0f, 0.0f);
  }
  for (int e = threadIdx.x; e < k * kkp; e += blockDim.x) {
    const int i = e / kkp, c = e - i * kkp;
    cf[e] = c < kk ? ff_from_double(it.P[i + (int64_t)it.ldc * c]) : make_float2(0.0f, 0.0f);
  }
  __syncthreads();
  const int rg = threadIdx.x % RG, cg = threadIdx.x / RG;
  for (int c0 = 0; c0 < kk; c0 += CP) {
    const int cb = c0 + 4 * cg;
    if (cb >= kk) continue;
    ffacc acc[4][4];
    for (int i = 0; i < k; ++i) {
      float2 av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = blk[i * RB + 4 * rg + a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = cf[i * kkp + cb + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b].fma(av[a], bv[b]);
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c = cb + b;
      if (c >= kk) break;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int t = 4 * rg + a;
        if (t < nr) {
          const ff v = acc[a][b].value();
          it.Uh[r0 + t + it.ldf * c] = v.hi;
          it.Ul[r0 + t + it.ldf * c] = v.lo;
          it.U[r0 + t + it.ldu * c] = ff_to_double(make_float2(v.hi, v.lo));
        }
      }
    }
  }
}

template <typename T>
void launch_ritz(const RitzItem<T>* items, int n, int kmax, int kkmax, const int32_t* pre_s, int tiles_s,
                 const int32_t* pre_l, int tiles_l, int final_pass, cudaStream_t st) {
  if (n <= 0) return;
  const int rs = RITZ_RB<double>(), rl = RITZ_RB<T>();
  const int cps = (256 / (rs / 4)) * RITZ_CW<double>(), cpl = (256 / (rl / 4)) * RITZ_CW<T>();
  const int kps = ((kmax + cps - 1) / cps) * cps, kpl = ((kmax + cpl - 1) / cpl) * cpl;
  const size_t sms = (size_t)rs * (kmax + 1) * sizeof(double) + (size_t)(kmax + 1) * kps * sizeof(double);
  const size_t sml = (size_t)rl * (kmax + 2) * sizeof(T) + (size_t)(kmax + 1) * kpl * sizeof(T);
  set_max_smem((const void*)k_ritz<T, true>);
  set_max_smem((const void*)k_ritz<T, false>);
  if (tiles_s > 0) {
    if constexpr (std::is_same<T, float>::value) {
      // the FP32 form's workspaces always carry the float-float copy
      const int kkp = ((kkmax + 63) / 64) * 64;
      const size_t smf = sizeof(float2) * ((size_t)RITZ_FF_RB * kmax + (size_t)kmax * kkp);
      set_max_smem((const void*)k_ritz_short_ff);
      k_ritz_short_ff<<<tiles_s, 256, smf, st>>>(items, pre_s, n, final_pass); count_launch();
    } else {
      k_ritz<T, true><<<tiles_s, 256, sms, st>>>(items, pre_s, n, final_pass); count_launch();
    }
  }
  if (tiles_l > 0) {
    k_ritz_coef<T><<<n, 256, 0, st>>>(items, final_pass); count_launch();
    if constexpr (std::is_same<T, float>::value)
      launch_ritz_tc(items, n, kmax, kkmax, pre_l, tiles_l, final_pass, st);
    else {
      k_ritz<T, false><<<tiles_l, 256, sml, st>>>(items, pre_l, n, final_pass); count_launch();
    }
  }
}

template <typename T>
void launch_finalize(const FinalItem<T>* items, int n, int max_r, int64_t max_rows, cudaStream_t st) {
  if (n <= 0) return;
  k_sign<T><<<dim3(max_r, n), 256, 0, st>>>(items); count_launch();
  // eight elements per thread: a block per 256 rows spent most of its time
  // starting up (one element each)
  unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((max_rows + 2047) / 2048, 1024));
  // (the long side's loop takes its eight in one batch: gx blocks x 256
  //  threads x 8 cover 2048 gx rows per pass)
  k_final_copy<T><<<dim3(gx, max_r, n), 256, 0, st>>>(items); count_launch();
}

#define INST(T)                                                                                        \
  template void launch_long_step<T>(const LongItem<T>*, const int32_t*, int, int, int, cudaStream_t);  \
  template void launch_long_init<T>(const LongItem<T>*, const int32_t*, int, int, cudaStream_t);       \
  template void launch_ritz<T>(const RitzItem<T>*, int, int, int, const int32_t*, int, const int32_t*,  \
                               int, int, cudaStream_t);                                                 \
  template void launch_finalize<T>(const FinalItem<T>*, int, int, int64_t, cudaStream_t);
INST(float)
INST(double)

}  // namespace ssa
