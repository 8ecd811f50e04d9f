// Shapes and weights (Sec. 5.1 and 6.2.3-6.2.4), computed exactly in integers.
//
//  * N  -- observed samples: inside the user mask and not NaN (Sec. 5.2);
//  * K  -- window origins kappa with L (+) {kappa} inside N (eq. sh_Ks).  The
//          paper finds K from one FFT product (Alg. find_ks) and keeps the
//          entries equal to L; here each origin tests the window's bit rows
//          against the observed bit rows directly, so no rounding is involved;
//  * w  -- w_k = #{(i, j) : l_i (+) k_j = k}, the diagonal-averaging weights
//          (Alg. qhankelization step 1); N' = {w > 0}.
// All sets are stored as per-column bit masks (bit x of column y).
#include <algorithm>
#include "common.cuh"
#include "shape.h"
#include "launch.h"

namespace ssa {

// 32 bits of a column bit-row starting at (possibly negative) bit position p;
// bits outside [0, 32*nw) read as zero.
__device__ __forceinline__ uint32_t extract32(const uint32_t* col, int nw, int p) {
  int w = p >> 5;                       // floor division for negative p
  int b = p & 31;
  uint32_t lo = (w >= 0 && w < nw) ? col[w] : 0u;
  uint32_t hi = (w + 1 >= 0 && w + 1 < nw) ? col[w + 1] : 0u;
  return __funnelshift_r(lo, hi, b);
}

// Observed bits; flags +-Inf inside the mask as bad input.
__global__ void k_obs_bits(const void* data, int data_double, const uint8_t* mask, int nx, int ny,
                           int words, uint32_t* bits, int* err) {
  const int y = blockIdx.y;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  bool ok = false;
  if (x < nx) {
    const int64_t g = x + (int64_t)nx * y;
    double v = data_double ? ((const double*)data)[g] : (double)((const float*)data)[g];
    bool m = mask ? (mask[g] != 0) : true;
    ok = m && !isnan(v);
    if (ok && isinf(v)) { atomicExch(err, 1); ok = false; }
  }
  const unsigned bal = __ballot_sync(0xffffffffu, ok);
  const int w = x >> 5;
  if ((threadIdx.x & 31) == 0 && w < words) bits[(int64_t)y * words + w] = bal;
}

// Origins: thread per candidate (kx, ky); a warp covers 32 consecutive kx.
// wrows: window bit rows, ey columns x wwords words (bit lx of column ly).
__global__ void k_origins(const uint32_t* obs, int nwords_obs, const uint32_t* wrows, int wwords, int ey,
                          int cx, int cy, int kwords, uint32_t* kbits) {
  const int ky = blockIdx.y;
  const int kx = blockIdx.x * blockDim.x + threadIdx.x;
  bool in = kx < cx && ky < cy;
  if (in) {
    for (int ly = 0; ly < ey && in; ++ly) {
      const uint32_t* col = obs + (int64_t)(ky + ly) * nwords_obs;
      const uint32_t* wr = wrows + (int64_t)ly * wwords;
      for (int t = 0; t < wwords; ++t) {
        const uint32_t wb = wr[t];
        if (wb == 0u) continue;
        const uint32_t o = extract32(col, nwords_obs, kx + 32 * t);
        if (wb & ~o) { in = false; break; }
      }
    }
  }
  const unsigned bal = __ballot_sync(0xffffffffu, in);
  const int w = kx >> 5;
  if ((threadIdx.x & 31) == 0 && w < kwords) kbits[(int64_t)ky * kwords + w] = bal;
}

__device__ __forceinline__ int block_sum_int(int v, int* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  int t = 0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  return t;
}

__global__ void k_col_popc(const uint32_t* bits, int words, int ncols, int32_t* cnt) {
  const int y = blockIdx.x;
  __shared__ int red[32];
  int c = 0;
  for (int w = threadIdx.x; w < words; w += blockDim.x) c += __popc(bits[(int64_t)y * words + w]);
  int tot = block_sum_int(c, red);
  if (threadIdx.x == 0) cnt[y] = tot;
}

// Exclusive prefix sum of n counts into base[0..n] (base[n] = total), one CTA.
__global__ void k_scan_counts(const int32_t* cnt, int n, int32_t* base) {
  __shared__ int wt[32];
  __shared__ int carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < n; b0 += blockDim.x) {
    const int i = b0 + threadIdx.x;
    const int v = i < n ? cnt[i] : 0;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wt[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
      int c = carry;
      for (int w = 0; w < nw; ++w) { int t = wt[w]; wt[w] = c; c += t; }
      carry = c;
    }
    __syncthreads();
    if (i < n) base[i] = x - v + wt[warp];
    __syncthreads();
  }
  if (threadIdx.x == 0) base[n] = carry;
}

// Weights: w(x, y) = sum over window columns ly of the number of origins in
// column y-ly at x-lx for lx in the window column (reversed rows make it an
// aligned AND + popcount).  rrows: reversed window rows, bit (ex-1-lx).
__global__ void k_weights(const uint32_t* kbits, int kwords, int kcols, const uint32_t* rrows, int rwords,
                          int ex, int ey, int nx, int ny, int32_t* w, uint32_t* nbits, int nwords) {
  const int y = blockIdx.y;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  int cnt = 0;
  if (x < nx) {
    for (int ly = 0; ly < ey; ++ly) {
      const int ky = y - ly;
      if (ky < 0 || ky >= kcols) continue;
      const uint32_t* col = kbits + (int64_t)ky * kwords;
      const uint32_t* rr = rrows + (int64_t)ly * rwords;
      const int p0 = x - ex + 1;
      for (int t = 0; t < rwords; ++t) {
        const uint32_t rb = rr[t];
        if (rb == 0u) continue;
        cnt += __popc(rb & extract32(col, kwords, p0 + 32 * t));
      }
    }
    w[x + (int64_t)nx * y] = cnt;
  }
  const unsigned bal = __ballot_sync(0xffffffffu, cnt > 0);
  const int wd = x >> 5;
  if ((threadIdx.x & 31) == 0 && wd < nwords) nbits[(int64_t)y * nwords + wd] = bal;
}

// ---------------------------------------------------------------- batched forms
// Batched kernels: one block per 256 grid rows of one column of one item
// (tiles laid out by tile_item).
__global__ void k_obs_batch(const ObsItem* __restrict__ items, const int32_t* __restrict__ pre, int n) {
  int t;
  const ObsItem it = items[tile_item(pre, n, blockIdx.x, t)];
  const int tx = (it.nx + 255) >> 8;
  const int y = t / tx;
  const int x = (t - y * tx) * 256 + threadIdx.x;
  bool ok = false;
  double sq = 0.0;
  if (x < it.nx) {
    const int64_t g = x + (int64_t)it.nx * y;
    const double v = it.data_double ? ((const double*)it.data)[g] : (double)((const float*)it.data)[g];
    ok = !isnan(v);
    if (ok && isinf(v)) { atomicExch(it.err, 1); ok = false; }
    if (ok) sq = v * v;
  }
  const unsigned bal = __ballot_sync(0xffffffffu, ok);
  const int w = x >> 5;
  if ((threadIdx.x & 31) == 0 && w < it.words) it.bits[(int64_t)y * it.words + w] = bal;
  // the block's sum of squares (warp sums, then warps in order: repeatable)
  __shared__ double wsum[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += wsum[i];
    it.sq[t] = tot;
  }
}

// ||x||_2 of each problem: its observation blocks' sums of squares, added in
// a fixed order (one block per problem).
__global__ void k_norm_batch(const NormItem* __restrict__ items) {
  const NormItem it = items[blockIdx.x];
  __shared__ double part[256];
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < it.n; i += blockDim.x) a += it.sq[i];
  part[threadIdx.x] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) tot += part[i];
    *it.out = sqrt(tot);
  }
}

// Set bits of a column bit row at positions < x, from the word prefix counts
// (x clamped to [0, 32 nw]).
__device__ __forceinline__ int bits_below(const uint32_t* col, const int32_t* pre, int nw, int x) {
  if (x <= 0) return 0;
  const int w = x >> 5;
  if (w >= nw) return pre[nw];
  const int b = x & 31;
  return pre[w] + (b ? __popc(col[w] & ((1u << b) - 1u)) : 0);
}

__global__ void k_prefix_batch(const PrefixItem* __restrict__ items, const int32_t* __restrict__ tpre, int n) {
  int y;
  const PrefixItem it = items[tile_item(tpre, n, blockIdx.x, y)];
  __shared__ int wt[32];
  __shared__ int carry;
  const uint32_t* col = it.bits + (int64_t)y * it.words;
  int32_t* pre = it.pre + (int64_t)y * (it.words + 1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwp = blockDim.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < it.words; b0 += blockDim.x) {
    const int i = b0 + threadIdx.x;
    const int v = i < it.words ? __popc(col[i]) : 0;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += t;
    }
    if (lane == 31) wt[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
      int c = carry;
      for (int w = 0; w < nwp; ++w) { const int t = wt[w]; wt[w] = c; c += t; }
      carry = c;
    }
    __syncthreads();
    if (i < it.words) pre[i] = x - v + wt[warp];
    __syncthreads();
  }
  if (threadIdx.x == 0) pre[it.words] = carry;
}

void launch_prefix_batch(const PrefixItem* it, const int32_t* pre, int n, int tiles, cudaStream_t st) {
  if (n <= 0 || tiles <= 0) return;
  k_prefix_batch<<<tiles, 256, 0, st>>>(it, pre, n); count_launch();
}

__global__ void k_origins_batch(const OriginItem* __restrict__ items, const int32_t* __restrict__ pre, int n) {
  int t;
  const OriginItem it = items[tile_item(pre, n, blockIdx.x, t)];
  const int tx = (it.cx + 255) >> 8;
  const int ky = t / tx;
  const int kx = (t - ky * tx) * 256 + threadIdx.x;
  bool in = kx < it.cx;
  if (in && it.interval) {
    // window column ly occupies rows [a, b]: all of kx + a .. kx + b observed
    for (int ly = 0; ly < it.ey && in; ++ly) {
      const int a = it.wint[2 * ly], b = it.wint[2 * ly + 1];
      if (a < 0) continue;
      const int64_t c = (int64_t)(ky + ly);
      const uint32_t* col = it.obs + c * it.nwords_obs;
      const int32_t* pre = it.opre + c * (it.nwords_obs + 1);
      const int s = kx + a, e = kx + b + 1;
      in = bits_below(col, pre, it.nwords_obs, e) - bits_below(col, pre, it.nwords_obs, s) == e - s;
    }
  } else if (in) {
    for (int ly = 0; ly < it.ey && in; ++ly) {
      const uint32_t* col = it.obs + (int64_t)(ky + ly) * it.nwords_obs;
      const uint32_t* wr = it.wrows + (int64_t)ly * it.wwords;
      for (int t = 0; t < it.wwords; ++t) {
        const uint32_t wb = wr[t];
        if (wb == 0u) continue;
        if (wb & ~extract32(col, it.nwords_obs, kx + 32 * t)) { in = false; break; }
      }
    }
  }
  const unsigned bal = __ballot_sync(0xffffffffu, in);
  const int w = kx >> 5;
  if ((threadIdx.x & 31) == 0 && w < it.kwords) it.kbits[(int64_t)ky * it.kwords + w] = bal;
}

__global__ void k_popc_batch(const CountItem* __restrict__ items, const int32_t* __restrict__ pre, int n) {
  int y;
  const CountItem it = items[tile_item(pre, n, blockIdx.x, y)];
  __shared__ int red[32];
  int c = 0;
  for (int w = threadIdx.x; w < it.words; w += blockDim.x) c += __popc(it.bits[(int64_t)y * it.words + w]);
  const int tot = block_sum_int(c, red);
  if (threadIdx.x == 0) it.cnt[y] = tot;
}

__global__ void k_scan_batch(const CountItem* __restrict__ items) {
  const CountItem it = items[blockIdx.x];
  __shared__ int wt[32];
  __shared__ int carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < it.ncols; b0 += blockDim.x) {
    const int i = b0 + threadIdx.x;
    const int v = i < it.ncols ? it.cnt[i] : 0;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wt[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
      int c = carry;
      for (int w = 0; w < nw; ++w) { const int t = wt[w]; wt[w] = c; c += t; }
      carry = c;
    }
    __syncthreads();
    if (i < it.ncols) it.colbase[i] = x - v + wt[warp];
    __syncthreads();
  }
  if (threadIdx.x == 0) { it.colbase[it.ncols] = carry; *it.total = carry; }
}

__global__ void k_weights_batch(const WeightItem* __restrict__ items, const int32_t* __restrict__ pre, int n) {
  int t;
  const WeightItem it = items[tile_item(pre, n, blockIdx.x, t)];
  const int tx = (it.nx + 255) >> 8;
  const int y = t / tx;
  const int x = (t - y * tx) * 256 + threadIdx.x;
  int cnt = 0;
  if (x < it.nx && it.interval) {
    // origins kx with kx + l = x for l in [a, b]: kx in [x - b, x - a]
    for (int ly = 0; ly < it.ey; ++ly) {
      const int ky = y - ly;
      if (ky < 0 || ky >= it.kcols) continue;
      const int a = it.wint[2 * ly], b = it.wint[2 * ly + 1];
      if (a < 0) continue;
      const uint32_t* col = it.kbits + (int64_t)ky * it.kwords;
      const int32_t* pre = it.kpre + (int64_t)ky * (it.kwords + 1);
      const int s = x - b, e = x - a + 1;
      if (e > s) cnt += bits_below(col, pre, it.kwords, e) - bits_below(col, pre, it.kwords, s);
    }
    it.w[x + (int64_t)it.nx * y] = cnt;
  } else if (x < it.nx) {
    for (int ly = 0; ly < it.ey; ++ly) {
      const int ky = y - ly;
      if (ky < 0 || ky >= it.kcols) continue;
      const uint32_t* col = it.kbits + (int64_t)ky * it.kwords;
      const uint32_t* rr = it.rrows + (int64_t)ly * it.rwords;
      const int p0 = x - it.ex + 1;
      for (int t = 0; t < it.rwords; ++t) {
        const uint32_t rb = rr[t];
        if (rb == 0u) continue;
        cnt += __popc(rb & extract32(col, it.kwords, p0 + 32 * t));
      }
    }
    it.w[x + (int64_t)it.nx * y] = cnt;
  }
  const unsigned bal = __ballot_sync(0xffffffffu, cnt > 0);
  const int wd = x >> 5;
  if ((threadIdx.x & 31) == 0 && wd < it.nwords) it.nbits[(int64_t)y * it.nwords + wd] = bal;
}

void launch_obs_batch(const ObsItem* it, const int32_t* pre, int n, int tiles, cudaStream_t st) {
  if (n <= 0 || tiles <= 0) return;
  k_obs_batch<<<tiles, 256, 0, st>>>(it, pre, n); count_launch();
}
void launch_norm_batch(const NormItem* it, int n, cudaStream_t st) {
  if (n <= 0) return;
  k_norm_batch<<<n, 256, 0, st>>>(it); count_launch();
}
void launch_origins_batch(const OriginItem* it, const int32_t* pre, int n, int tiles, cudaStream_t st) {
  if (n <= 0 || tiles <= 0) return;
  k_origins_batch<<<tiles, 256, 0, st>>>(it, pre, n); count_launch();
}
void launch_counts_batch(const CountItem* it, const int32_t* pre, int n, int tiles, cudaStream_t st) {
  if (n <= 0) return;
  if (tiles > 0) { k_popc_batch<<<tiles, 256, 0, st>>>(it, pre, n); count_launch(); }
  k_scan_batch<<<n, 1024, 0, st>>>(it); count_launch();
}
void launch_weights_batch(const WeightItem* it, const int32_t* pre, int n, int tiles, cudaStream_t st) {
  if (n <= 0 || tiles <= 0) return;
  k_weights_batch<<<tiles, 256, 0, st>>>(it, pre, n); count_launch();
}

// ---------------------------------------------------------------- launchers
void launch_obs_bits(const void* data, int data_double, const uint8_t* mask, int nx, int ny, int words,
                     uint32_t* bits, int* err, cudaStream_t st) {
  dim3 g((nx + 255) / 256, ny);
  k_obs_bits<<<g, 256, 0, st>>>(data, data_double, mask, nx, ny, words, bits, err); count_launch();
}

void launch_origins(const uint32_t* obs, int nwords_obs, const uint32_t* wrows, int wwords, int ey, int cx,
                    int cy, int kwords, uint32_t* kbits, cudaStream_t st) {
  dim3 g((cx + 255) / 256, cy);
  k_origins<<<g, 256, 0, st>>>(obs, nwords_obs, wrows, wwords, ey, cx, cy, kwords, kbits); count_launch();
}

void launch_col_counts(const uint32_t* bits, int words, int ncols, int32_t* cnt, int32_t* colbase,
                       cudaStream_t st) {
  k_col_popc<<<ncols, 256, 0, st>>>(bits, words, ncols, cnt); count_launch();
  k_scan_counts<<<1, 1024, 0, st>>>(cnt, ncols, colbase); count_launch();
}

void launch_weights(const uint32_t* kbits, int kwords, int kcols, const uint32_t* rrows, int rwords, int ex,
                    int ey, int nx, int ny, int32_t* w, uint32_t* nbits, int nwords, cudaStream_t st) {
  dim3 g((nx + 255) / 256, ny);
  k_weights<<<g, 256, 0, st>>>(kbits, kwords, kcols, rrows, rwords, ex, ey, nx, ny, w, nbits, nwords); count_launch();
}

}  // namespace ssa
