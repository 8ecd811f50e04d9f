// Grouped reconstruction: rank-one (quasi-)hankelization by FFT (Sec. 6.1.3,
// Alg. hankelization; Sec. 6.2.3, Alg. qhankelization and Alg. diagsums).
//
// For a group I the reconstruction is  sum_{i in I} sigma_i diagsums(U_i, V_i)
// divided by the weights w.  diagsums(U, V) is the linear convolution of U
// scattered on the window set with V scattered on the origin set, i.e.
// F^-1(F(U') . F(V')) (Lemma hbh_tbt_elmat).  Linearity lets the group be
// summed in frequency space, so each (group, channel) needs one inverse
// transform; F(U'_i) is shared by all channels and groups.
#include "fft_block.cuh"
#include "kernels.cuh"
#include "launch.h"
#include <algorithm>
#include "recon.h"

namespace ssa {

// (same scatter as the matvec x-pass; duplicated here to keep the translation
// units independent)
template <typename T, typename TI>
__device__ void rec_load_col(T* rb, int Mx, const TI* __restrict__ in, const MapDev& m, int y,
                             int32_t* s_pre, int32_t* s_wt) {
  if (m.dense || y >= m.by) {
    const bool ok = (y < m.by);
    const int64_t base = (int64_t)y * m.bx;
    const int xe = ok ? (int)min((int64_t)m.bx, m.limit - base) : 0;
    const TI* src = in + base;
    for (int x = threadIdx.x; x < Mx; x += blockDim.x) rb[x] = (x < xe) ? (T)src[x] : T(0);
  } else {
    const uint32_t* wb = m.bits + (int64_t)y * m.words;
    block_popc_scan(wb, m.words, s_pre, s_wt);
    const TI* src = in + m.colbase[y];
    for (int x = threadIdx.x; x < Mx; x += blockDim.x) {
      T v = T(0);
      if (x < m.bx) {
        const uint32_t w = wb[x >> 5];
        const int b = x & 31;
        if ((w >> b) & 1u) v = (T)src[s_pre[x >> 5] + __popc(w & ((1u << b) - 1u))];
      }
      rb[x] = v;
    }
  }
}

template <typename T>
struct RSmem {
  Cx<T>* A; Cx<T>* B; Cx<T>* C; Cx<T>* tab; int32_t* pre; int32_t* wt;
  __device__ RSmem(unsigned char* p, int H) {
    A = reinterpret_cast<Cx<T>*>(p);
    B = A + padded_len(H);
    C = B + padded_len(H);
    tab = C + padded_len(H);
    pre = reinterpret_cast<int32_t*>(tab + (H >> 2) + 1);   // octant table of W_{2H}
    wt = pre + ((2 * H) / 32 + 1);
  }
};

template <typename T>
__device__ Cx<T>* rec_forward(Cx<T>* A, Cx<T>* B, int log2H, const Cx<T>* tab, const Cx<T>* tw) {
  const int H = 1 << log2H;
  __syncthreads();
  Cx<T>* Z = block_fft_s<T, false>(A, B, log2H, 1, tab, log2H + 1);
  Cx<T>* G = (Z == A) ? B : A;
  for (int k = threadIdx.x; k <= H; k += blockDim.x) G[k] = untwist_fwd_s(Z, k, log2H, tab);
  __syncthreads();
  return G;
}

// Half spectrum of one column of a compact vector (U_i or V_i): x-pass.
template <typename T, typename TV>
__global__ void __launch_bounds__(512) k_rec_col_fft(const RecColItem<T, TV>* __restrict__ items,
                                                     const Cx<T>* __restrict__ tw) {
  const RecColItem<T, TV> it = items[blockIdx.y];
  const int y = blockIdx.x;
  if (y >= it.ncols) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int log2H = it.log2Mx - 1, H = 1 << log2H;
  RSmem<T> sm(smem, H);
  load_octant(sm.tab, it.log2Mx, tw);
  rec_load_col<T, TV>(reinterpret_cast<T*>(sm.A), 2 * H, it.vec, it.map, y, sm.pre, sm.wt);
  Cx<T>* G = rec_forward(sm.A, sm.B, log2H, sm.tab, tw);
  Cx<T>* dst = it.dst + (int64_t)y * (H + 1);
  for (int k = threadIdx.x; k <= H; k += blockDim.x) dst[k] = G[k];
}

// Series: one CTA per (group, channel).  acc = sum_i (sigma_i / Mx) F(U'_i) F(V'_i)
// then inverse, divide by w, NaN where w = 0.
template <typename T, typename TV>
__global__ void __launch_bounds__(512) k_rec1d(const Rec1Item<T, TV>* __restrict__ items, const Cx<T>* __restrict__ tw) {
  const Rec1Item<T, TV> it = items[blockIdx.x];
  extern __shared__ __align__(16) unsigned char smem[];
  const int log2H = it.log2Mx - 1, H = 1 << log2H;
  RSmem<T> sm(smem, H);
  load_octant(sm.tab, it.log2Mx, tw);
  for (int k = threadIdx.x; k <= H; k += blockDim.x) sm.C[k] = cx(T(0), T(0));
  __syncthreads();   // an empty group reads C right away below
  for (int c = 0; c < it.ncomp; ++c) {
    const int i = it.comps[c];
    rec_load_col<T, TV>(reinterpret_cast<T*>(sm.A), 2 * H, it.V + it.ldv * i, it.map, 0, sm.pre, sm.wt);
    Cx<T>* G = rec_forward(sm.A, sm.B, log2H, sm.tab, tw);
    const Cx<T>* gu = it.gu + it.ldgu * i;
    const T sc = (T)(it.sigma[i] * it.inv_norm);
    for (int k = threadIdx.x; k <= H; k += blockDim.x) sm.C[k] = sm.C[k] + sc * (gu[k] * G[k]);
    __syncthreads();
  }
  // inverse of the accumulated half spectrum (C), into A/C ping-pong
  for (int k = threadIdx.x; k < H; k += blockDim.x) sm.A[k] = twist_inv_s(sm.C, k, log2H, sm.tab);
  __syncthreads();
  Cx<T>* R = block_fft_s<T, true>(sm.A, sm.B, log2H, 1, sm.tab, log2H + 1);
  const T* r = reinterpret_cast<const T*>(R);
  for (int n = threadIdx.x; n < it.n; n += blockDim.x) {
    const int w = it.w[n];
    // FP32 sums: the division in FP32 (the sums carry FP32 error already),
    // one conversion -- an FP64 division per element ran on GB300's FP64 pipe
    if constexpr (std::is_same<T, float>::value)
      it.out[n] = (w > 0) ? (double)(r[n] / (float)w) : __longlong_as_double(0x7ff8000000000000ll);
    else
      it.out[n] = (w > 0) ? (double)r[n] / (double)w : __longlong_as_double(0x7ff8000000000000ll);
  }
}

// Images: inverse x-pass of the accumulated spectrum, divide by w.
template <typename T>
__global__ void __launch_bounds__(512) k_rec_xinv(const Rec2Item<T>* __restrict__ items, const Cx<T>* __restrict__ tw) {
  const Rec2Item<T> it = items[blockIdx.y];
  const int y = blockIdx.x;
  if (y >= it.ny) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int log2H = it.log2Mx - 1, H = 1 << log2H;
  RSmem<T> sm(smem, H);
  load_octant(sm.tab, it.log2Mx, tw);
  const Cx<T>* src = it.g2 + (int64_t)y * (H + 1);
  for (int k = threadIdx.x; k <= H; k += blockDim.x) sm.C[k] = src[k];
  __syncthreads();
  for (int k = threadIdx.x; k < H; k += blockDim.x) sm.A[k] = twist_inv_s(sm.C, k, log2H, sm.tab);
  __syncthreads();
  Cx<T>* R = block_fft_s<T, true>(sm.A, sm.B, log2H, 1, sm.tab, log2H + 1);
  const T* r = reinterpret_cast<const T*>(R);
  for (int x = threadIdx.x; x < it.nx; x += blockDim.x) {
    const int64_t g = x + (int64_t)it.nx * y;
    if (!it.w) { it.out[g] = (double)r[x] * it.inv_norm; continue; }   // raw sums (long series)
    const int w = it.w[g];
    if constexpr (std::is_same<T, float>::value)   // FP32 sums: FP32 division, one conversion
      it.out[g] = (w > 0) ? (double)(r[x] * (float)it.inv_norm / (float)w) : __longlong_as_double(0x7ff8000000000000ll);
    else
      it.out[g] = (w > 0) ? (double)r[x] * it.inv_norm / (double)w : __longlong_as_double(0x7ff8000000000000ll);
  }
}

// Long series: the diagonal sums of a group arrive as a segment image S
// (2B rows, one column per segment) whose column c holds the sums of the
// data elements cB .. cB + 2B - 2.  Element p gathers row p mod B of column
// p div B and row B + p mod B of the column before (overlap-add), then is
// divided by w.
__global__ void k_rec_fold(const RecFoldItem* __restrict__ items) {
  const RecFoldItem it = items[blockIdx.y];
  const int64_t B = it.B;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < it.n; p += (int64_t)gridDim.x * blockDim.x) {
    const int w = it.w[p];
    if (w <= 0) { it.out[p] = __longlong_as_double(0x7ff8000000000000ll); continue; }
    const int64_t c = p / B, i = p - c * B;
    double v = (c < it.ncols) ? it.S[i + 2 * B * c] : 0.0;
    if (c > 0 && i + B < 2 * B - 1) v += it.S[i + B + 2 * B * (c - 1)];
    it.out[p] = v / (double)w;
  }
}

// One warp per border element p: x~[p] = (1/w_p) sum over the anti-diagonal
// i + j = p of sum_{c in group} sigma_c U[i, c] V[j, c], summed directly
// (not through the FFT, whose absolute error the small w_p would magnify).
__global__ void __launch_bounds__(256) k_rec_border(const RecBorderItem* __restrict__ items) {
  const RecBorderItem it = items[blockIdx.y];
  const int lane = threadIdx.x & 31;
  const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);    // 0 .. 2W-1
  const int64_t N = (int64_t)it.L + it.K - 1;
  if (e >= 2 * REC_BORDER_W) return;
  const int64_t p = e < REC_BORDER_W ? e : N - 1 - (e - REC_BORDER_W);
  if (p < 0 || p >= N || (e >= REC_BORDER_W && p < REC_BORDER_W)) return;
  const int64_t i0 = p - it.K + 1 > 0 ? p - it.K + 1 : 0;
  const int64_t i1 = p < it.L - 1 ? p : it.L - 1;
  // FP32 products and sums of the FP32 vectors (at most 64 terms a
  // component: a relative error near 64 eps32 of the terms' magnitude, far
  // inside the form's tolerance); sigma converted once per component --
  // GB300 runs FP64 at about 1/70 of the FP32 rate
  float acc = 0.0f;
  for (int q = 0; q < it.ncomp; ++q) {
    const int c = it.comps[q];
    const float sg = (float)it.sigma[c];
    const float* uc = it.U + (int64_t)it.L * c;
    const float* vc = it.V + it.ldv * c;
    for (int64_t i = i0 + lane; i <= i1; i += 32) acc = fmaf(sg * uc[i], vc[p - i], acc);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) it.out[p] = (double)(acc / (float)(i1 - i0 + 1));
}

void launch_rec_border(const RecBorderItem* items, int n, cudaStream_t st) {
  if (n <= 0) return;
  const int warps = 8;
  k_rec_border<<<dim3((2 * REC_BORDER_W + warps - 1) / warps, n), 32 * warps, 0, st>>>(items); count_launch();
}

void launch_rec_fold(const RecFoldItem* items, int n, int64_t max_n, cudaStream_t st) {
  if (n <= 0) return;
  const unsigned bx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((max_n + 255) / 256, 1024));
  k_rec_fold<<<dim3(bx, n), 256, 0, st>>>(items); count_launch();
}

// residual = x - sum of the groups, on N' (NaN elsewhere), in FP64
__global__ void k_residual(const void* data, int data_double, const int32_t* w, int64_t n, const double* groups,
                           int64_t gstride, int ngroups, double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (w[i] <= 0) { out[i] = __longlong_as_double(0x7ff8000000000000ll); continue; }
    double v = data_double ? ((const double*)data)[i] : (double)((const float*)data)[i];
    for (int g = 0; g < ngroups; ++g) v -= groups[g * gstride + i];
    out[i] = v;
  }
}

__global__ void k_residual_batch(const ResItem* __restrict__ items) {
  const ResItem it = items[blockIdx.y];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < it.n; i += (int64_t)gridDim.x * blockDim.x) {
    if (it.w[i] <= 0) { it.out[i] = __longlong_as_double(0x7ff8000000000000ll); continue; }
    double v = it.data_double ? ((const double*)it.data)[i] : (double)((const float*)it.data)[i];
    for (int g = 0; g < it.ngroups; ++g) v -= it.groups[g * it.gstride + i];
    it.out[i] = v;
  }
}

void launch_residual_batch(const ResItem* items, int n, int64_t max_n, cudaStream_t st) {
  if (n <= 0) return;
  const unsigned bx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((max_n + 255) / 256, 1024));
  k_residual_batch<<<dim3(bx, n), 256, 0, st>>>(items); count_launch();
}

// ---------------------------------------------------------------- launchers
static inline size_t rsmem_bytes(int log2Mx, size_t csz) {
  const size_t H = size_t(1) << (log2Mx - 1);
  return (3 * (size_t)padded_len((int)H) + H / 4 + 1) * csz + ((2 * H) / 32 + 1 + 32) * sizeof(int32_t);
}

template <typename T, typename TV>
void launch_rec_col_fft(const RecColItem<T, TV>* items, int n, int max_log2Mx, int max_cols, const Cx<T>* tw,
                        cudaStream_t st) {
  if (n <= 0) return;
  size_t sm = rsmem_bytes(max_log2Mx, sizeof(Cx<T>));
  set_max_smem((const void*)k_rec_col_fft<T, TV>);
  k_rec_col_fft<T, TV><<<dim3(max_cols, n), 512, sm, st>>>(items, tw); count_launch();
}

template <typename T, typename TV>
void launch_rec1d(const Rec1Item<T, TV>* items, int n, int max_log2Mx, const Cx<T>* tw, cudaStream_t st) {
  if (n <= 0) return;
  size_t sm = rsmem_bytes(max_log2Mx, sizeof(Cx<T>));
  set_max_smem((const void*)k_rec1d<T, TV>);
  k_rec1d<T, TV><<<n, 512, sm, st>>>(items, tw); count_launch();
}

template <typename T>
void launch_rec_xinv(const Rec2Item<T>* items, int n, int max_log2Mx, int max_ny, const Cx<T>* tw,
                     cudaStream_t st) {
  if (n <= 0) return;
  size_t sm = rsmem_bytes(max_log2Mx, sizeof(Cx<T>));
  set_max_smem((const void*)k_rec_xinv<T>);
  k_rec_xinv<T><<<dim3(max_ny, n), 512, sm, st>>>(items, tw); count_launch();
}

void launch_residual(const void* data, int data_double, const int32_t* w, int64_t n, const double* groups,
                     int64_t gstride, int ngroups, double* out, cudaStream_t st) {
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
  if (blocks < 1) blocks = 1;
  k_residual<<<blocks, 256, 0, st>>>(data, data_double, w, n, groups, gstride, ngroups, out); count_launch();
}

#define INST(T, TV)                                                                                       \
  template void launch_rec_col_fft<T, TV>(const RecColItem<T, TV>*, int, int, int, const Cx<T>*, cudaStream_t); \
  template void launch_rec1d<T, TV>(const Rec1Item<T, TV>*, int, int, const Cx<T>*, cudaStream_t);
INST(float, float)
INST(double, float)
INST(double, double)
template void launch_rec_xinv<float>(const Rec2Item<float>*, int, int, int, const Cx<float>*, cudaStream_t);
template void launch_rec_xinv<double>(const Rec2Item<double>*, int, int, int, const Cx<double>*, cudaStream_t);

// ------------------------------------------------------------ w-correlations
// A block stages sqrt(w_k) y_i[k] for the m vectors over WGRAM_CH elements
// (zero where w_k = 0, which also drops the NaN outside N'), then each thread
// adds the chunk's products to its WGRAM_PT pairs; blocks stride over chunks.
__global__ void __launch_bounds__(WGRAM_NT) k_wgram(const double* __restrict__ Y, int64_t ldy, int n,
                                                    const void* __restrict__ x, int x_f64,
                                                    const int32_t* __restrict__ w, int64_t total,
                                                    const int2* __restrict__ pairs, int npair,
                                                    double* __restrict__ partials) {
  extern __shared__ __align__(16) double ys[];     // m x WGRAM_CH, then sqrt(w) (WGRAM_CH)
  const int m = n + 1;
  double* sw = ys + (size_t)m * WGRAM_CH;
  double acc[WGRAM_PT];
  int2 pr[WGRAM_PT];
#pragma unroll
  for (int q = 0; q < WGRAM_PT; ++q) {
    acc[q] = 0.0;
    const int p = threadIdx.x + q * WGRAM_NT;
    pr[q] = p < npair ? pairs[p] : make_int2(0, 0);
  }
  for (int64_t c0 = (int64_t)blockIdx.x * WGRAM_CH; c0 < total; c0 += (int64_t)gridDim.x * WGRAM_CH) {
    __syncthreads();                                  // the previous chunk has been used
    if (threadIdx.x < WGRAM_CH) {
      const int64_t k = c0 + threadIdx.x;
      const int32_t wk = k < total ? w[k] : 0;
      sw[threadIdx.x] = wk > 0 ? sqrt((double)wk) : 0.0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < m * WGRAM_CH; e += WGRAM_NT) {
      const int i = e / WGRAM_CH, t = e - i * WGRAM_CH;
      const int64_t k = c0 + t;
      double v = 0.0;
      const double s = sw[t];
      if (s != 0.0) {
        const double y = i < n ? Y[(int64_t)i * ldy + k]
                               : (x_f64 ? ((const double*)x)[k] : (double)((const float*)x)[k]);
        v = s * y;
      }
      ys[e] = v;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < WGRAM_PT; ++q) {
      if (threadIdx.x + q * WGRAM_NT < npair) {
        const double* yi = ys + pr[q].x * WGRAM_CH;
        const double* yj = ys + pr[q].y * WGRAM_CH;
        double s0 = acc[q], s1 = 0.0;
#pragma unroll 4
        for (int t = 0; t < WGRAM_CH; t += 2) { s0 = fma(yi[t], yj[t], s0); s1 = fma(yi[t + 1], yj[t + 1], s1); }
        acc[q] = s0 + s1;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < WGRAM_PT; ++q) {
    const int p = threadIdx.x + q * WGRAM_NT;
    if (p < npair) partials[(int64_t)blockIdx.x * npair + p] = acc[q];
  }
}

__global__ void __launch_bounds__(256) k_wcor_final(const double* __restrict__ partials, int nblk,
                                                    const int2* __restrict__ pairs, int npair, int n,
                                                    double* __restrict__ G, double* __restrict__ rho,
                                                    double* __restrict__ contrib) {
  const int m = n + 1;
  for (int p = threadIdx.x; p < npair; p += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partials[(int64_t)b * npair + p];
    const int2 ij = pairs[p];
    G[ij.x * m + ij.y] = s;
    G[ij.y * m + ij.x] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e - i * n;
    const double gi = G[i * m + i], gj = G[j * m + j];
    rho[e] = (gi > 0.0 && gj > 0.0) ? (i == j ? 1.0 : G[i * m + j] / (sqrt(gi) * sqrt(gj))) : 0.0;
  }
  const double xx = G[n * m + n];
  for (int i = threadIdx.x; i < n; i += blockDim.x) contrib[i] = xx > 0.0 ? G[i * m + i] / xx : 0.0;
}

void launch_wgram(const double* Y, int64_t ldy, int n, const void* x, int x_f64, const int32_t* w, int64_t total,
                  const int2* pairs, int npair, double* partials, int nblk, cudaStream_t st) {
  const size_t sm = sizeof(double) * (size_t)(n + 2) * WGRAM_CH;
  k_wgram<<<nblk, WGRAM_NT, sm, st>>>(Y, ldy, n, x, x_f64, w, total, pairs, npair, partials); count_launch();
}

void launch_wcor_final(const double* partials, int nblk, const int2* pairs, int npair, int n, double* G, double* rho,
                       double* contrib, cudaStream_t st) {
  k_wcor_final<<<1, 256, 0, st>>>(partials, nblk, pairs, npair, n, G, rho, contrib); count_launch();
}

// ------------------------------------------------------------ forecasting
template <typename T>
__global__ void __launch_bounds__(256) k_lrr(const T* __restrict__ U, int64_t L, const int32_t* __restrict__ idx,
                                             int nidx, double* __restrict__ R, double* __restrict__ nu2) {
  double n2 = 0.0;
  for (int j = 0; j < nidx; ++j) {
    const double pj = (double)U[(L - 1) + L * idx[j]];
    n2 = fma(pj, pj, n2);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *nu2 = n2;
  const double scale = n2 < 1.0 ? 1.0 / (1.0 - n2) : 0.0;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L - 1) return;
  double acc = 0.0;
  for (int j = 0; j < nidx; ++j) {
    const int64_t col = L * idx[j];
    acc = fma((double)U[(L - 1) + col], (double)U[i + col], acc);
  }
  R[i] = acc * scale;
}

__global__ void __launch_bounds__(256) k_forecast_rec(const double* __restrict__ rec, const int64_t* __restrict__ off,
                                                      const int64_t* __restrict__ len, int64_t L,
                                                      const double* __restrict__ R, int M, double* __restrict__ work,
                                                      int64_t ldw, double* __restrict__ out) {
  const int p = blockIdx.x;
  double* y = work + ldw * p;
  const int64_t n1 = L - 1;
  const double* src = rec + off[p] + len[p] - n1;      // the last L - 1 values of the series
  for (int64_t t = threadIdx.x; t < n1; t += blockDim.x) y[t] = src[t];
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int m = 0; m < M; ++m) {
    __syncthreads();                                    // y[m + L - 2] is in place
    double a = 0.0;
    for (int64_t t = threadIdx.x; t < n1; t += blockDim.x) a = fma(R[t], y[m + t], a);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) red[warp] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (int w = 0; w < nw; ++w) tot += red[w];     // fixed order
      y[m + n1] = tot;
      out[(int64_t)p * M + m] = tot;
    }
  }
}

template <typename T>
void launch_lrr(const T* U, int64_t L, const int32_t* idx, int nidx, double* R, double* nu2, cudaStream_t st) {
  const unsigned g = (unsigned)std::max<int64_t>(1, (L - 1 + 255) / 256);
  k_lrr<T><<<g, 256, 0, st>>>(U, L, idx, nidx, R, nu2); count_launch();
}
template void launch_lrr<float>(const float*, int64_t, const int32_t*, int, double*, double*, cudaStream_t);
template void launch_lrr<double>(const double*, int64_t, const int32_t*, int, double*, double*, cudaStream_t);

void launch_forecast_rec(const double* rec, const int64_t* off, const int64_t* len, int s, int64_t L,
                         const double* R, int M, double* work, int64_t ldw, double* out, cudaStream_t st) {
  k_forecast_rec<<<s, 256, 0, st>>>(rec, off, len, L, R, M, work, ldw, out); count_launch();
}

// ------------------------------------------------------------ vector forecast
__device__ __forceinline__ double vf_block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < nw; ++w) t += red[w];     // fixed order
  return t;
}

// G[a * nidx + b] = sum_{i < L-1} U[i, idx_a] U[i+1, idx_b]
template <typename T>
__global__ void __launch_bounds__(256) k_vf_gram(const T* __restrict__ U, int64_t L, const int32_t* __restrict__ idx,
                                                 int nidx, double* __restrict__ G) {
  __shared__ double red[32];
  const int a = blockIdx.x / nidx, b = blockIdx.x - a * nidx;
  const T* ua = U + L * idx[a];
  const T* ub = U + L * idx[b] + 1;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < L - 1; i += blockDim.x) acc = fma((double)ua[i], (double)ub[i], acc);
  const double t = vf_block_sum(acc, red);
  if (threadIdx.x == 0) G[blockIdx.x] = t;
}

// D = G + pi (pi^T G) / (1 - nu^2), nu^2 = |pi|^2 (written to *nu2)
template <typename T>
__global__ void __launch_bounds__(256) k_vf_shift(const T* __restrict__ U, int64_t L, const int32_t* __restrict__ idx,
                                                  int nidx, const double* __restrict__ G, double* __restrict__ D,
                                                  double* __restrict__ nu2) {
  double n2 = 0.0;
  for (int j = 0; j < nidx; ++j) {
    const double pj = (double)U[(L - 1) + L * idx[j]];
    n2 = fma(pj, pj, n2);
  }
  if (threadIdx.x == 0) *nu2 = n2;
  const double scale = n2 < 1.0 ? 1.0 / (1.0 - n2) : 0.0;
  for (int e = threadIdx.x; e < nidx * nidx; e += blockDim.x) {
    const int a = e / nidx, b = e - a * nidx;
    double pg = 0.0;                               // (pi^T G)_b
    for (int c = 0; c < nidx; ++c) pg = fma((double)U[(L - 1) + L * idx[c]], G[c * nidx + b], pg);
    D[e] = G[e] + (double)U[(L - 1) + L * idx[a]] * pg * scale;
  }
}

// c_0 = U_I^T (last L values of series p), then c_t = D c_{t-1}, t < M + L
template <typename T>
__global__ void __launch_bounds__(256) k_vf_coef(const T* __restrict__ U, int64_t L, const int32_t* __restrict__ idx,
                                                 int nidx, const void* __restrict__ x, int x_f64,
                                                 const int64_t* __restrict__ off, const int64_t* __restrict__ len,
                                                 int M, const double* __restrict__ D, double* __restrict__ cs) {
  __shared__ double red[32];
  const int p = blockIdx.x;
  double* c = cs + (int64_t)p * (M + L) * nidx;
  const int64_t x0 = off[p] + len[p] - L;
  for (int a = 0; a < nidx; ++a) {
    const T* ua = U + L * idx[a];
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < L; i += blockDim.x) {
      const double xv = x_f64 ? ((const double*)x)[x0 + i] : (double)((const float*)x)[x0 + i];
      acc = fma((double)ua[i], xv, acc);
    }
    const double t = vf_block_sum(acc, red);
    if (threadIdx.x == 0) c[a] = t;
  }
  for (int64_t t = 1; t < M + L; ++t) {
    __syncthreads();                               // c_{t-1} is complete
    const double* prev = c + (t - 1) * nidx;
    double* cur = c + t * nidx;
    for (int a = threadIdx.x; a < nidx; a += blockDim.x) {
      double acc = 0.0;
      for (int b = 0; b < nidx; ++b) acc = fma(D[a * nidx + b], prev[b], acc);
      cur[a] = acc;
    }
  }
}

// out[p * M + m] = (1 / L) sum_{i < L} sum_a U[i, idx_a] c_{L + m - i}[a]; block (m, p)
template <typename T>
__global__ void __launch_bounds__(256) k_vf_out(const T* __restrict__ U, int64_t L, const int32_t* __restrict__ idx,
                                                int nidx, int M, const double* __restrict__ cs, double* __restrict__ out) {
  __shared__ double red[32];
  const int m = blockIdx.x, p = blockIdx.y;
  const double* c = cs + (int64_t)p * (M + L) * nidx;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < L; i += blockDim.x) {
    const double* ct = c + (L + m - i) * nidx;
    for (int a = 0; a < nidx; ++a) acc = fma((double)U[i + L * idx[a]], ct[a], acc);
  }
  const double t = vf_block_sum(acc, red);
  if (threadIdx.x == 0) out[(int64_t)p * M + m] = t / (double)L;
}

template <typename T>
void launch_vector_forecast(const T* U, int64_t L, const int32_t* idx, int nidx, const void* x, int x_f64,
                            const int64_t* off, const int64_t* len, int s, int M, double* G, double* D, double* nu2,
                            double* cs, double* out, cudaStream_t st) {
  k_vf_gram<T><<<nidx * nidx, 256, 0, st>>>(U, L, idx, nidx, G); count_launch();
  k_vf_shift<T><<<1, 256, 0, st>>>(U, L, idx, nidx, G, D, nu2); count_launch();
  k_vf_coef<T><<<s, 256, 0, st>>>(U, L, idx, nidx, x, x_f64, off, len, M, D, cs); count_launch();
  k_vf_out<T><<<dim3(M, s), 256, 0, st>>>(U, L, idx, nidx, M, cs, out); count_launch();
}
template void launch_vector_forecast<float>(const float*, int64_t, const int32_t*, int, const void*, int,
                                            const int64_t*, const int64_t*, int, int, double*, double*, double*,
                                            double*, double*, cudaStream_t);
template void launch_vector_forecast<double>(const double*, int64_t, const int32_t*, int, const void*, int,
                                             const int64_t*, const int64_t*, int, int, double*, double*, double*,
                                             double*, double*, cudaStream_t);

// ------------------------------------------------------------ row forecasts
// Solve A X = B in place (A: n x n symmetric positive definite, B: n x q,
// row-major, global memory) by Gauss-Jordan without pivoting; one block.
__device__ void rf_solve_spd(double* A, double* B, int n, int q, int* fail) {
  __shared__ double piv;
  for (int k = 0; k < n; ++k) {
    __syncthreads();
    if (threadIdx.x == 0) {
      piv = A[k * n + k];
      if (!(piv > 0.0)) { *fail = 1; piv = 1.0; }
    }
    __syncthreads();
    const double ip = 1.0 / piv;
    for (int c = threadIdx.x; c < n + q; c += blockDim.x) {
      if (c < n) A[k * n + c] *= ip;
      else B[k * q + (c - n)] *= ip;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * (n + q); e += blockDim.x) {
      const int i = e / (n + q), c = e - i * (n + q);
      if (i == k) continue;
      const double f = A[i * n + k];
      if (c == k) continue;                        // column k of row i is cleared below
      if (c < n) A[i * n + c] -= f * A[k * n + c];
      else B[i * q + (c - n)] -= f * B[k * q + (c - n)];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      if (i != k) A[i * n + k] = 0.0;
  }
  __syncthreads();
}

// one block: S, then the system of the recurrent (A = I_s - S S^T, B = S,
// solution W: s x r) or the vector form (A = I_r - S^T S, B = Vbar^T V',
// solution D: r x r)
template <typename T>
__global__ void __launch_bounds__(256) k_rf_setup(int vector, const T* __restrict__ V, int64_t K,
                                                  const int32_t* __restrict__ idx, int nidx,
                                                  const int64_t* __restrict__ koff, const int64_t* __restrict__ kc,
                                                  int s, double* A, double* Bm, int* fail) {
  __shared__ double red[32];
  if (!vector) {
    for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
      const int p = e / s, q = e - p * s;
      double acc = 0.0;
      for (int j = 0; j < nidx; ++j) {
        const double sp = (double)V[koff[p] + kc[p] - 1 + K * idx[j]];
        const double sq = (double)V[koff[q] + kc[q] - 1 + K * idx[j]];
        acc = fma(sp, sq, acc);
      }
      A[e] = (p == q ? 1.0 : 0.0) - acc;
    }
    for (int e = threadIdx.x; e < s * nidx; e += blockDim.x) {
      const int p = e / nidx, j = e - p * nidx;
      Bm[e] = (double)V[koff[p] + kc[p] - 1 + K * idx[j]];
    }
    rf_solve_spd(A, Bm, s, nidx, fail);
  } else {
    for (int e = threadIdx.x; e < nidx * nidx; e += blockDim.x) {
      const int a = e / nidx, b = e - a * nidx;
      double acc = 0.0;
      for (int p = 0; p < s; ++p)
        acc = fma((double)V[koff[p] + kc[p] - 1 + K * idx[a]], (double)V[koff[p] + kc[p] - 1 + K * idx[b]], acc);
      A[e] = (a == b ? 1.0 : 0.0) - acc;
    }
    // Bm = Vbar^T V': sum over series p and rows t < kc[p] - 1 of V[t, a] V[t + 1, b]
    for (int e = 0; e < nidx * nidx; ++e) {
      const int a = e / nidx, b = e - a * nidx;
      double acc = 0.0;
      for (int p = 0; p < s; ++p) {
        const T* va = V + koff[p] + K * idx[a];
        const T* vb = V + koff[p] + 1 + K * idx[b];
        for (int64_t t = threadIdx.x; t < kc[p] - 1; t += blockDim.x) acc = fma((double)va[t], (double)vb[t], acc);
      }
      const double tot = vf_block_sum(acc, red);
      if (threadIdx.x == 0) Bm[e] = tot;
    }
    rf_solve_spd(A, Bm, nidx, nidx, fail);
  }
}

// recurrent row forecast: one block, M steps
template <typename T>
__global__ void __launch_bounds__(256) k_rf_rec(const T* __restrict__ V, int64_t K, const int32_t* __restrict__ idx,
                                                int nidx, const int64_t* __restrict__ koff,
                                                const int64_t* __restrict__ kc, const int64_t* __restrict__ off,
                                                const int64_t* __restrict__ len, int s, int M,
                                                const double* __restrict__ rec, const double* __restrict__ W,
                                                double* __restrict__ work, const int64_t* __restrict__ wo,
                                                double* __restrict__ out) {
  __shared__ double red[32];
  __shared__ double w[RF_MAXR];
  for (int p = 0; p < s; ++p) {                   // the last K_p - 1 reconstructed values
    const double* src = rec + off[p] + len[p] - (kc[p] - 1);
    for (int64_t t = threadIdx.x; t < kc[p] - 1; t += blockDim.x) work[wo[p] + t] = src[t];
  }
  for (int m = 0; m < M; ++m) {
    __syncthreads();
    for (int j = 0; j < nidx; ++j) {
      double acc = 0.0;
      for (int p = 0; p < s; ++p) {
        const T* vj = V + koff[p] + K * idx[j];
        const double* z = work + wo[p] + m;
        for (int64_t t = threadIdx.x; t < kc[p] - 1; t += blockDim.x) acc = fma((double)vj[t], z[t], acc);
      }
      const double tot = vf_block_sum(acc, red);
      if (threadIdx.x == 0) w[j] = tot;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < s; p += blockDim.x) {
      double nx = 0.0;
      for (int j = 0; j < nidx; ++j) nx = fma(W[p * nidx + j], w[j], nx);
      work[wo[p] + kc[p] - 1 + m] = nx;
      out[(int64_t)p * M + m] = nx;
    }
  }
}

// vector row forecast: c_{L-1} = V^T (row L-1 of X), c_i = D c_{i-1}; cs holds
// rows i = L-1 .. L-1 + M + kstar - 1 (ld nidx)
template <typename T>
__global__ void __launch_bounds__(256) k_rf_coef(const T* __restrict__ V, int64_t K, const int32_t* __restrict__ idx,
                                                 int nidx, const int64_t* __restrict__ koff,
                                                 const int64_t* __restrict__ kc, const int64_t* __restrict__ off,
                                                 int s, int64_t L, int M, int64_t kstar,
                                                 const void* __restrict__ x, int x_f64, const double* __restrict__ D,
                                                 double* __restrict__ cs) {
  __shared__ double red[32];
  for (int a = 0; a < nidx; ++a) {
    double acc = 0.0;
    for (int p = 0; p < s; ++p) {
      const T* va = V + koff[p] + K * idx[a];
      const int64_t x0 = off[p] + L - 1;          // row L-1 of series p's block: x_p[L-1 + t]
      for (int64_t t = threadIdx.x; t < kc[p]; t += blockDim.x) {
        const double xv = x_f64 ? ((const double*)x)[x0 + t] : (double)((const float*)x)[x0 + t];
        acc = fma((double)va[t], xv, acc);
      }
    }
    const double tot = vf_block_sum(acc, red);
    if (threadIdx.x == 0) cs[a] = tot;
  }
  for (int64_t t = 1; t < M + kstar; ++t) {
    __syncthreads();
    const double* prev = cs + (t - 1) * nidx;
    double* cur = cs + t * nidx;
    for (int a = threadIdx.x; a < nidx; a += blockDim.x) {
      double acc = 0.0;
      for (int b = 0; b < nidx; ++b) acc = fma(D[a * nidx + b], prev[b], acc);
      cur[a] = acc;
    }
  }
}

// out[p * M + m] = (1 / K_p) sum_{j < K_p} sum_a V[koff_p + j, a] c_{N_p + m - j}[a]; block (m, p)
template <typename T>
__global__ void __launch_bounds__(256) k_rf_out(const T* __restrict__ V, int64_t K, const int32_t* __restrict__ idx,
                                                int nidx, const int64_t* __restrict__ koff,
                                                const int64_t* __restrict__ kc, const int64_t* __restrict__ len,
                                                int64_t L, int M, const double* __restrict__ cs,
                                                double* __restrict__ out) {
  __shared__ double red[32];
  const int m = blockIdx.x, p = blockIdx.y;
  double acc = 0.0;
  for (int64_t j = threadIdx.x; j < kc[p]; j += blockDim.x) {
    const double* ct = cs + (len[p] + m - j - (L - 1)) * nidx;    // row N_p + m - j
    for (int a = 0; a < nidx; ++a) acc = fma((double)V[koff[p] + j + K * idx[a]], ct[a], acc);
  }
  const double tot = vf_block_sum(acc, red);
  if (threadIdx.x == 0) out[(int64_t)p * M + m] = tot / (double)kc[p];
}

template <typename T>
void launch_row_forecast(int vector, const T* V, int64_t K, const int32_t* idx, int nidx, const int64_t* koff,
                         const int64_t* kc, const int64_t* off, const int64_t* len, int s, int64_t L, int M,
                         int64_t kstar, const double* rec, const void* x, int x_f64, double* A, double* Bm,
                         double* work, const int64_t* wo, double* cs, double* out, int* fail, cudaStream_t st) {
  k_rf_setup<T><<<1, 256, 0, st>>>(vector, V, K, idx, nidx, koff, kc, s, A, Bm, fail); count_launch();
  if (!vector) {
    k_rf_rec<T><<<1, 256, 0, st>>>(V, K, idx, nidx, koff, kc, off, len, s, M, rec, Bm, work, wo, out); count_launch();
  } else {
    k_rf_coef<T><<<1, 256, 0, st>>>(V, K, idx, nidx, koff, kc, off, s, L, M, kstar, x, x_f64, Bm, cs); count_launch();
    k_rf_out<T><<<dim3(M, s), 256, 0, st>>>(V, K, idx, nidx, koff, kc, len, L, M, cs, out); count_launch();
  }
}
#define RF_INST(T)                                                                                          \
  template void launch_row_forecast<T>(int, const T*, int64_t, const int32_t*, int, const int64_t*,       \
                                       const int64_t*, const int64_t*, const int64_t*, int, int64_t, int,  \
                                       int64_t, const double*, const void*, int, double*, double*, double*, \
                                       const int64_t*, double*, double*, int*, cudaStream_t);
RF_INST(float)
RF_INST(double)

}  // namespace ssa
