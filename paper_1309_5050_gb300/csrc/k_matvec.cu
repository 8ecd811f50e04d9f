// Trajectory-matrix products by FFT (Sec. 6.1.2 Alg. hmul_u; Sec. 6.2.2, the
// quasi-Hankel product) and the data spectrum they share.
//
//   u = X v :  scatter v onto the grid at the origins K, transform, multiply by
//              the data spectrum times the conjugate, transform back, gather the
//              window positions L.  (X^T u swaps the roles of L and K.)
//
// Series (My == 1) run fused in one CTA per (problem, channel): load with
// scatter, length-H complex FFT of the packed real signal, half-spectrum
// product, inverse, gather -- all in shared memory.  Images run as three
// passes: x-pass (packed real FFT down every grid column, scatter fused),
// y-pass (complex FFT across columns, spectrum product, inverse, pruned to the
// output's columns), x-pass inverse (gather fused).
#include "fft_block.cuh"
#include "kernels.cuh"
#include <algorithm>
#include "launch.h"
#include "tma.cuh"

namespace ssa {

// ---------------------------------------------------------------- helpers
// Fill rb[0..Mx) with grid column y of a compact vector (zeros elsewhere).
template <typename T, typename TI>
__device__ void load_col(T* rb, int Mx, const TI* __restrict__ in, const MapDev& m, int y,
                         int32_t* s_pre, int32_t* s_wt, T scale = T(1)) {
  if (m.dense || y >= m.by) {
    const bool ok = (y < m.by);
    const int64_t base = (int64_t)y * m.bx;
    const int xe = ok ? (int)min((int64_t)m.bx, m.limit - base) : 0;   // entries of this column
    const TI* src = in + base;
    for (int x = threadIdx.x; x < Mx; x += blockDim.x)
      rb[x] = (x < xe) ? (T)src[x] * scale : T(0);
  } else {
    const uint32_t* wb = m.bits + (int64_t)y * m.words;
    block_popc_scan(wb, m.words, s_pre, s_wt);
    const TI* src = in + m.colbase[y];
    for (int x = threadIdx.x; x < Mx; x += blockDim.x) {
      T v = T(0);
      if (x < m.bx) {
        const uint32_t w = wb[x >> 5];
        const int b = x & 31;
        if ((w >> b) & 1u) v = (T)src[s_pre[x >> 5] + __popc(w & ((1u << b) - 1u))] * scale;
      }
      rb[x] = v;
    }
  }
}

// scale of the input column of a matvec item (deferred normalisation of the
// long Lanczos vectors), 1 when none
template <typename T>
__device__ __forceinline__ T in_scale_of(const MvItem<T>& it, int s) {
  if (!it.in_scale || !it.in.st) return T(1);
  return (T)it.in_scale[it.in.st->jc + s + it.in.jdelta];
}

// The series product's two scalars that come from FP64 state -- the input
// column's scale and, for the fused long step, alpha_j times v_j's column
// scale -- formed once per block by thread 0 into shared memory: GB300 runs
// FP64 arithmetic and FP64 -> FP32 conversions at about 1/70 of the FP32
// rate, and 512 threads forming each of them cost a measurable share of the
// product.
template <typename T, bool FUSED>
__device__ __forceinline__ void series_scalars(const MvItem<T>& it, int s, T* scal) {
  scal[0] = in_scale_of(it, s);
  scal[1] = T(0);
  if constexpr (FUSED) {
    const int j = it.st->jc + s;
    scal[1] = (T)(it.lB[j + (int64_t)it.lldb * j] * it.lcolscale[j]);
  }
}

// Write the map's positions of grid column y from rb into a compact vector.
template <typename T, typename TO>
__device__ void store_col(const T* rb, TO* __restrict__ out, const MapDev& m, int y,
                          int32_t* s_pre, int32_t* s_wt) {
  if (y >= m.by) return;
  if (m.dense) {
    const int64_t base = (int64_t)y * m.bx;
    const int xe = (int)min((int64_t)m.bx, m.limit - base);
    TO* dst = out + base;
    for (int x = threadIdx.x; x < xe; x += blockDim.x) dst[x] = (TO)rb[x];
  } else {
    const uint32_t* wb = m.bits + (int64_t)y * m.words;
    block_popc_scan(wb, m.words, s_pre, s_wt);
    TO* dst = out + m.colbase[y];
    for (int x = threadIdx.x; x < m.bx; x += blockDim.x) {
      const uint32_t w = wb[x >> 5];
      const int b = x & 31;
      if ((w >> b) & 1u) dst[s_pre[x >> 5] + __popc(w & ((1u << b) - 1u))] = (TO)rb[x];
    }
  }
}

template <typename T>
__device__ __forceinline__ bool item_skip(const LzState* st, int s) {
  return st && (!st->active || st->jc + s >= st->k || st->jc + s < 0);
}

// x-pass shared layout: two padded complex buffers (padded_len(H) >= H+1),
// the octant twiddle table of W_{2H} (it serves the length-H FFT, whose
// twiddles are the even powers, and the untwist / twist factors W_{2H}^k),
// optionally a 16-byte aligned staging buffer for the H+1 spectrum values,
// then scan scratch.
__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

template <typename T>
struct XSmem {
  Cx<T>* A; Cx<T>* B; Cx<T>* tab; Cx<T>* S; int32_t* pre; int32_t* wt;
  int log2H;
  __device__ XSmem(unsigned char* p, int H, int log2M_, const Cx<T>* tw, bool spec = false) : log2H(log2M_ - 1) {
    A = reinterpret_cast<Cx<T>*>(p);
    B = A + padded_len(H);
    tab = B + padded_len(H);
    size_t off = align16((size_t)(2 * padded_len(H) + (H >> 2) + 1) * sizeof(Cx<T>));
    S = reinterpret_cast<Cx<T>*>(p + off);
    if (spec) off += align16((size_t)(H + 1) * sizeof(Cx<T>));
    pre = reinterpret_cast<int32_t*>(p + off);
    wt = pre + ((2 * H) / 32 + 1);
    load_octant(tab, log2H + 1, tw);
  }
};

// Forward half of an x-pass: packed FFT of rb (viewed in A) and untwist into
// the other buffer.  Returns the half spectrum (H+1 values).
template <typename T>
__device__ Cx<T>* xpass_forward(XSmem<T>& sm, int log2H) {
  const int H = 1 << log2H;
  __syncthreads();
  Cx<T>* Z = block_fft_s<T, false>(sm.A, sm.B, log2H, 1, sm.tab, log2H + 1);
  Cx<T>* G = (Z == sm.A) ? sm.B : sm.A;
  for (int k = threadIdx.x; k <= H; k += blockDim.x) G[k] = untwist_fwd_s(Z, k, log2H, sm.tab);
  __syncthreads();
  return G;
}

// Inverse half of an x-pass: P (H+1 values, in one buffer) -> real signal
// (2H values) viewed in the returned buffer.
template <typename T>
__device__ T* xpass_inverse(XSmem<T>& sm, Cx<T>* P, int log2H) {
  const int H = 1 << log2H;
  Cx<T>* Q = (P == sm.A) ? sm.B : sm.A;
  for (int k = threadIdx.x; k < H; k += blockDim.x) Q[k] = twist_inv_s(P, k, log2H, sm.tab);
  __syncthreads();
  Cx<T>* R = block_fft_s<T, true>(Q, P, log2H, 1, sm.tab, log2H + 1);
  return reinterpret_cast<T*>(R);
}

// Polls of a bulk-copy wait before the kernel gives up and flags it.
constexpr int MBAR_POLL_LIMIT = 1 << 22;
__device__ int g_mv_async_timeouts;
__device__ int g_ypass_bad_tiles;      // y-pass blocks whose tile did not fit the launch's buffers

// The series product with the transform size a compile-time constant
// (H = 2^LOG2H complex points, NT threads) for dense maps -- the FP32 form's
// code paths 0 (X v), 5 (X^T u of the FP64 u, fused long step) and 20 (X^T u
// from the shared transform of u, fused long step).  Same arithmetic as the
// runtime form of k_mv1d, which calls it for the sizes of the series
// workloads; the index, padding and loop arithmetic folds to constants
// (about 30% fewer instructions per product at H = 4096).
template <typename T, int MODE, int LOG2H, int NT>
__device__ __forceinline__ void mv1d_ct_body(const MvItem<T>& it, int s, const Cx<T>* __restrict__ tw,
                                             unsigned char* smem, uint64_t& bar) {
  constexpr int H = 1 << LOG2H, LOG2TN = LOG2H + 1;
  constexpr bool IN_DOUBLE = (MODE & MV1_IN_DOUBLE) != 0;
  constexpr bool OUT_FUSED = (MODE & MV1_OUT_FUSED) != 0;
  constexpr bool IN_ZSPEC = (MODE & MV1_IN_ZSPEC) != 0;
  static_assert((MODE & (MV1_IN_MAPPED | MV1_OUT_MAPPED)) == 0, "dense maps only");
  typedef typename std::conditional<IN_DOUBLE, double, T>::type TI;
  Cx<T>* A = reinterpret_cast<Cx<T>*>(smem);
  Cx<T>* B = A + padded_len(H);
  Cx<T>* tab = B + padded_len(H);
  Cx<T>* S = reinterpret_cast<Cx<T>*>(smem + align16((size_t)(2 * padded_len(H) + H / 4 + 1) * sizeof(Cx<T>)));
  load_octant(tab, LOG2TN, tw);
  constexpr uint32_t bulk = (uint32_t)(H * sizeof(Cx<T>));
  constexpr int NST = (LOG2H + 2) / 3;            // stages of block_fft_io_ct
  Cx<T>* Z = (IN_ZSPEC || !(NST & 1)) ? A : B;
  Cx<T>* X = (Z == A) ? B : A;
  __shared__ T scal[2];                 // input scale, fused-step coefficient (see series_scalars)
  if (threadIdx.x == 0) {
    mbar_init(&bar);
    if constexpr (IN_ZSPEC) {
      mbar_arrive_expect(&bar, 2 * bulk);
      bulk_copy(S, it.xh, bulk, &bar);
      bulk_copy(Z, it.zin, bulk, &bar);
    } else {
      bulk_load(S, it.xh, bulk, &bar);
    }
    series_scalars<T, OUT_FUSED>(it, s, scal);
  }
  const Cx<T> last = it.xh[H];
  if constexpr (IN_ZSPEC) {
    __syncthreads();                    // twiddle table and barrier initialised
  } else {
    const int64_t ioff = vec_elem_off(it.in, s);
    const int64_t xe = imin64((int64_t)it.min.bx, it.min.limit);
    __syncthreads();                    // twiddle table, scalars
    const T isc = scal[0];
    const TI* src = (const TI*)it.in.base + ioff;
    auto in = [src, xe, isc](int j, int r, int nq) {
      const int64_t x = 2 * (int64_t)(j + r * nq);
      return cx(x < xe ? (T)src[x] * isc : T(0), x + 1 < xe ? (T)src[x + 1] * isc : T(0));
    };
    auto zout = [Z](int base, int stride, auto& v) {
      constexpr int R = sizeof(v) / sizeof(v[0]);
#pragma unroll
      for (int r = 0; r < R; ++r) Z[base + r * stride] = v[r];
    };
    block_fft_io_ct<T, false, LOG2H, NT, LOG2TN>(in, zout, A, B, tab);
  }
  if (!mbar_wait_bounded(&bar, 0, MBAR_POLL_LIMIT) && threadIdx.x == 0) atomicAdd(&g_mv_async_timeouts, 1);
  // G = untwist(Z); P = S conj(G); Q = twist(P), over the pairs (k, H - k)
#pragma unroll
  for (int k = threadIdx.x; k <= (H >> 1); k += NT) {
    const int k2 = H - k;
    const Cx<T> za = Z[k], zb = Z[k2 & (H - 1)];
    const Cx<T> w = tw_oct(tab, LOG2TN, k);             // W_2H^k
    const Cx<T> w2 = cx(-w.re, w.im);                    // W_2H^(H-k) = -conj(W_2H^k)
    const Cx<T> g1 = T(0.5) * (za + conj(zb)) + w * (T(0.5) * mul_mi(za - conj(zb)));
    const Cx<T> g2 = T(0.5) * (zb + conj(za)) + w2 * (T(0.5) * mul_mi(zb - conj(za)));
    const Cx<T> p1 = S[k] * conj(g1);
    const Cx<T> p2 = (k == 0 ? last : S[k2]) * conj(g2);
    X[k] = (p1 + conj(p2)) + mul_pi(conj(w) * (p1 - conj(p2)));
    if (k != 0 && k2 != k) X[k2] = (p2 + conj(p1)) + mul_pi(conj(w2) * (p2 - conj(p1)));
  }
  __syncthreads();
  const Cx<T>* Xc = X;
  auto qin = [Xc](int j, int r, int nq) { return Xc[j + r * nq]; };
  T* o = (T*)it.out.base + vec_elem_off(it.out, s);
  if constexpr (OUT_FUSED) {
    // fused long-side step: q = (X^T u) - alpha_j v_j into column j+1, partial |q|^2
    const int64_t xe = imin64((int64_t)it.mout.bx, it.mout.limit);
    const int j = it.st->jc + s;
    const T coef = scal[1];
    const T* vj = it.lV + it.lld * j + it.out.off;
    T* qn = it.lV + it.lld * (j + 1) + it.out.off;
    // v_j lands in the (now free) spectrum buffer while the inverse FFT runs:
    // each thread copies exactly the entries of its last-stage butterfly
    // (complex outputs t + r H / 8, t = thread index)
    T* vs = reinterpret_cast<T*>(S);
    constexpr int NS = H >> 3;
    if (threadIdx.x < NS) {
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int64_t x = 2 * (int64_t)(threadIdx.x + r * NS);
        if (x < xe) cp_async_elem<sizeof(T)>(vs + x, vj + x);
        if (x + 1 < xe) cp_async_elem<sizeof(T)>(vs + x + 1, vj + x + 1);
      }
    }
    T acc = T(0);
    auto st = [vs, qn, xe, coef, &acc](int base, int stride, auto& v) {
      constexpr int R = sizeof(v) / sizeof(v[0]);
      cp_async_wait_all();
      T a[2 * R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int64_t x = 2 * (int64_t)(base + r * stride);
        a[2 * r] = x < xe ? vs[x] : T(0);
        a[2 * r + 1] = x + 1 < xe ? vs[x + 1] : T(0);
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int64_t x = 2 * (int64_t)(base + r * stride);
        if (x < xe) { const T q = v[r].re - coef * a[2 * r]; qn[x] = q; acc = fma(q, q, acc); }
        if (x + 1 < xe) { const T q = v[r].im - coef * a[2 * r + 1]; qn[x + 1] = q; acc = fma(q, q, acc); }
      }
    };
    block_fft_io_ct<T, true, LOG2H, NT, LOG2TN>(qin, st, X, Z, tab);
    __shared__ double red[NT / 32];
    T wacc = acc;                   // threads without a butterfly add 0
    for (int o2 = 16; o2 > 0; o2 >>= 1) wacc += __shfl_down_sync(0xffffffffu, wacc, o2);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)wacc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < NT / 32; ++w) t += red[w];   // fixed order
      it.lnpart[it.lslot] = t;
    }
  } else {
    const int64_t xe = imin64((int64_t)it.mout.bx, it.mout.limit);
    auto st = [o, xe](int base, int stride, auto& v) {
      constexpr int R = sizeof(v) / sizeof(v[0]);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int64_t x = 2 * (int64_t)(base + r * stride);
        if (x < xe) o[x] = v[r].re;
        if (x + 1 < xe) o[x + 1] = v[r].im;
      }
    };
    block_fft_io_ct<T, true, LOG2H, NT, LOG2TN>(qin, st, X, Z, tab);
  }
}

// ---------------------------------------------------------------- kernels
// Series product, one CTA per (problem, channel):
//  * the data spectrum (H+1 values, contiguous) is brought into shared memory
//    by one bulk copy issued at entry, which lands during the forward FFT;
//  * the first forward stage reads the input column straight from global
//    memory (dense maps; a bit-mapped input is staged by load_col);
//  * untwist, product with the spectrum and twist run as one pass over the
//    pairs (k, H-k);
//  * the last inverse stage writes the output column straight to global
//    memory (dense maps; else through store_col).
// MODE (see mv1d_mode) selects one code path per instantiation: input type,
// input map, output form -- every item of a launch shares it.
template <typename T, int MODE>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 2 : 1) k_mv1d(const MvItem<T>* __restrict__ items, int s,
                                                 const Cx<T>* __restrict__ tw) {
  constexpr bool IN_DOUBLE = (MODE & MV1_IN_DOUBLE) != 0;
  constexpr bool IN_MAPPED = (MODE & MV1_IN_MAPPED) != 0;
  constexpr bool OUT_FUSED = (MODE & MV1_OUT_FUSED) != 0;
  constexpr bool OUT_MAPPED = (MODE & MV1_OUT_MAPPED) != 0;
  constexpr bool IN_ZSPEC = (MODE & MV1_IN_ZSPEC) != 0;
  typedef typename std::conditional<IN_DOUBLE, double, T>::type TI;
  const MvItem<T> it = items[blockIdx.x];
  if (item_skip<T>(it.st, s)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar;
  const int log2H = it.log2Mx - 1, H = 1 << log2H;
  if constexpr (std::is_same<T, float>::value && (MODE == 0 || MODE == 5 || MODE == 20)) {
    // the series workloads' sizes take the compile-time form (the layout of
    // the shared buffers is the same, so the launch's sizing fits it)
    if (log2H == 12) { mv1d_ct_body<T, MODE, 12, 512>(it, s, tw, smem, bar); return; }
    if (log2H == 11) { mv1d_ct_body<T, MODE, 11, 512>(it, s, tw, smem, bar); return; }
    if (log2H == 10) { mv1d_ct_body<T, MODE, 10, 512>(it, s, tw, smem, bar); return; }
  }
  XSmem<T> sm(smem, H, it.log2Mx, tw, true);
  // H complex values = a multiple of 16 bytes; the last value comes by a plain load
  const uint32_t bulk = (uint32_t)(H * sizeof(Cx<T>));
  const int nst = fft_io_stages(log2H);
  // forward result Z (written by the last forward stage, or copied in) and
  // the other buffer X (twisted product); a copied-in Z sits at the 16-byte
  // aligned start of the shared block
  Cx<T>* Z = (IN_ZSPEC || !(nst & 1)) ? sm.A : sm.B;
  Cx<T>* X = (Z == sm.A) ? sm.B : sm.A;
  __shared__ T scal[2];                 // input scale, fused-step coefficient (see series_scalars)
  if (threadIdx.x == 0) {
    mbar_init(&bar);
    if constexpr (IN_ZSPEC) {
      mbar_arrive_expect(&bar, 2 * bulk);
      bulk_copy(sm.S, it.xh, bulk, &bar);
      bulk_copy(Z, it.zin, bulk, &bar);
    } else {
      bulk_load(sm.S, it.xh, bulk, &bar);
    }
    series_scalars<T, OUT_FUSED>(it, s, scal);
  }
  const Cx<T> last = it.xh[H];
  auto zout = [Z](int base, int stride, auto& v) {
    constexpr int R = sizeof(v) / sizeof(v[0]);
#pragma unroll
    for (int r = 0; r < R; ++r) Z[base + r * stride] = v[r];
  };
  if constexpr (IN_ZSPEC) {
    __syncthreads();                    // twiddle table and barrier initialised
  } else if constexpr (!IN_MAPPED) {
    const int64_t ioff = vec_elem_off(it.in, s);
    const int64_t xe = imin64((int64_t)it.min.bx, it.min.limit);
    __syncthreads();                    // twiddle table, scalars
    const T isc = scal[0];
    const TI* src = (const TI*)it.in.base + ioff;
    auto in = [src, xe, isc](int i) {
      const int64_t x = 2 * (int64_t)i;
      return cx(x < xe ? (T)src[x] * isc : T(0), x + 1 < xe ? (T)src[x + 1] * isc : T(0));
    };
    block_fft_io<T, false>(in, zout, sm.A, sm.B, log2H, sm.tab, log2H + 1);
  } else {
    const int64_t ioff = vec_elem_off(it.in, s);
    const T isc = in_scale_of(it, s);
    load_col<T, TI>(reinterpret_cast<T*>(sm.A), 2 * H, (const TI*)it.in.base + ioff, it.min, 0, sm.pre, sm.wt, isc);
    __syncthreads();
    const Cx<T>* A = sm.A;
    auto in = [A](int i) { return A[i]; };
    block_fft_io<T, false>(in, zout, sm.A, sm.B, log2H, sm.tab, log2H + 1);
  }
  if (!mbar_wait_bounded(&bar, 0, MBAR_POLL_LIMIT) && threadIdx.x == 0) atomicAdd(&g_mv_async_timeouts, 1);
  // G = untwist(Z); P = S conj(G); Q = twist(P), over the pairs (k, H - k)
  for (int k = threadIdx.x; k <= (H >> 1); k += blockDim.x) {
    const int k2 = H - k;
    const Cx<T> za = Z[k], zb = Z[k2 & (H - 1)];
    const Cx<T> w = tw_oct(sm.tab, log2H + 1, k);      // W_2H^k
    const Cx<T> w2 = cx(-w.re, w.im);                    // W_2H^(H-k) = -conj(W_2H^k)
    const Cx<T> g1 = T(0.5) * (za + conj(zb)) + w * (T(0.5) * mul_mi(za - conj(zb)));
    const Cx<T> g2 = T(0.5) * (zb + conj(za)) + w2 * (T(0.5) * mul_mi(zb - conj(za)));
    const Cx<T> p1 = sm.S[k] * conj(g1);
    const Cx<T> p2 = (k == 0 ? last : sm.S[k2]) * conj(g2);
    X[k] = (p1 + conj(p2)) + mul_pi(conj(w) * (p1 - conj(p2)));
    if (k != 0 && k2 != k) X[k2] = (p2 + conj(p1)) + mul_pi(conj(w2) * (p2 - conj(p1)));
  }
  __syncthreads();
  const Cx<T>* Xc = X;
  auto qin = [Xc](int i) { return Xc[i]; };
  T* o = (T*)it.out.base + vec_elem_off(it.out, s);
  if constexpr (OUT_FUSED) {
    // fused long-side step: q = (X^T u) - alpha_j v_j into column j+1, partial |q|^2
    const int64_t xe = imin64((int64_t)it.mout.bx, it.mout.limit);
    const int j = it.st->jc + s;
    const T coef = scal[1];
    const T* vj = it.lV + it.lld * j + it.out.off;
    T* qn = it.lV + it.lld * (j + 1) + it.out.off;
    // v_j lands in the (now free) spectrum buffer while the inverse FFT runs:
    // each thread copies exactly the entries its last-stage butterflies use
    // (complex outputs b + r*Ns, b = thread index + multiples of the block)
    T* vs = reinterpret_cast<T*>(sm.S);
    {
      const int Ns = H >> 3;
      for (int b = threadIdx.x; b < Ns; b += blockDim.x)
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int64_t x = 2 * (int64_t)(b + r * Ns);
          if (x < xe) cp_async_elem<sizeof(T)>(vs + x, vj + x);
          if (x + 1 < xe) cp_async_elem<sizeof(T)>(vs + x + 1, vj + x + 1);
        }
    }
    // per-thread and per-warp partials of |q|^2 in T (a few dozen terms, then
    // 32), the sum of the warps' partials in double: FP64 per element or per
    // thread would cost more than the product on GB300
    T acc = T(0);
    auto st = [vs, qn, xe, coef, &acc](int base, int stride, auto& v) {
      constexpr int R = sizeof(v) / sizeof(v[0]);
      cp_async_wait_all();
      T a[2 * R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int64_t x = 2 * (int64_t)(base + r * stride);
        a[2 * r] = x < xe ? vs[x] : T(0);
        a[2 * r + 1] = x + 1 < xe ? vs[x + 1] : T(0);
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int64_t x = 2 * (int64_t)(base + r * stride);
        if (x < xe) { const T q = v[r].re - coef * a[2 * r]; qn[x] = q; acc = fma(q, q, acc); }
        if (x + 1 < xe) { const T q = v[r].im - coef * a[2 * r + 1]; qn[x + 1] = q; acc = fma(q, q, acc); }
      }
    };
    block_fft_io<T, true>(qin, st, X, Z, log2H, sm.tab, log2H + 1);
    __shared__ double red[16];
    T wacc = acc;
    for (int o2 = 16; o2 > 0; o2 >>= 1) wacc += __shfl_down_sync(0xffffffffu, wacc, o2);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)wacc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];   // fixed order
      it.lnpart[it.lslot] = t;
    }
  } else if constexpr (!OUT_MAPPED) {
    const int64_t xe = imin64((int64_t)it.mout.bx, it.mout.limit);
    auto st = [o, xe](int base, int stride, auto& v) {
      constexpr int R = sizeof(v) / sizeof(v[0]);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int64_t x = 2 * (int64_t)(base + r * stride);
        if (x < xe) o[x] = v[r].re;
        if (x + 1 < xe) o[x + 1] = v[r].im;
      }
    };
    block_fft_io<T, true>(qin, st, X, Z, log2H, sm.tab, log2H + 1);
  } else {
    Cx<T>* R = (nst & 1) ? Z : X;
    auto rout = [R](int base, int stride, auto& v) {
      constexpr int RR = sizeof(v) / sizeof(v[0]);
#pragma unroll
      for (int r = 0; r < RR; ++r) R[base + r * stride] = v[r];
    };
    block_fft_io<T, true>(qin, rout, X, Z, log2H, sm.tab, log2H + 1);
    store_col<T, T>(reinterpret_cast<const T*>(R), o, it.mout, 0, sm.pre, sm.wt);
  }
}

template <typename T>
__global__ void __launch_bounds__(512) k_mv_xfwd(const MvItem<T>* __restrict__ items, Tiles tl, int s,
                                                 const Cx<T>* __restrict__ tw) {
  int y;
  const MvItem<T> it = items[tile_of(tl, blockIdx.x, y)];
  if (y >= it.y_in_hi || item_skip<T>(it.st, s)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int log2H = it.log2Mx - 1, H = 1 << log2H;
  XSmem<T> sm(smem, H, it.log2Mx, tw);
  const int64_t ioff = vec_elem_off(it.in, s);
  const T isc = in_scale_of(it, s);
  if (it.in_type == 1)
    load_col<T, double>(reinterpret_cast<T*>(sm.A), 2 * H, (const double*)it.in.base + ioff, it.min, y, sm.pre, sm.wt, isc);
  else
    load_col<T, T>(reinterpret_cast<T*>(sm.A), 2 * H, (const T*)it.in.base + ioff, it.min, y, sm.pre, sm.wt, isc);
  Cx<T>* G = xpass_forward(sm, log2H);
  Cx<T>* dst = it.g1 + (int64_t)y * (H + 1);
  for (int k = threadIdx.x; k <= H; k += blockDim.x) dst[k] = G[k];
}

template <typename T>
__global__ void __launch_bounds__(512) k_mv_xinv(const MvItem<T>* __restrict__ items, Tiles tl, int s,
                                                 const Cx<T>* __restrict__ tw) {
  int y;
  const MvItem<T> it = items[tile_of(tl, blockIdx.x, y)];
  if (y >= it.y_out_hi || item_skip<T>(it.st, s)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int log2H = it.log2Mx - 1, H = 1 << log2H;
  XSmem<T> sm(smem, H, it.log2Mx, tw);
  const Cx<T>* src = it.g2 + (int64_t)y * (H + 1);
  for (int k = threadIdx.x; k <= H; k += blockDim.x) sm.A[k] = src[k];
  __syncthreads();
  T* r = xpass_inverse(sm, sm.A, log2H);
  __syncthreads();
  store_col<T, T>(r, (T*)it.out.base + vec_elem_off(it.out, s), it.mout, y, sm.pre, sm.wt);
}

// y-pass over a tile of TK consecutive x-frequencies (all My rows).
template <typename T>
__global__ void __launch_bounds__(512) k_ypass(const YItem<T>* __restrict__ items, Tiles tl, int mode, int s,
                                               int buf_elems, const Cx<T>* __restrict__ tw) {
  int b0;
  const YItem<T> it = items[tile_of(tl, blockIdx.x, b0)];
  if (item_skip<T>(it.st, s)) return;
  const int log2My = it.log2My;
  const int H = 1 << (it.log2Mx - 1), ld = H + 1;
  const int TK = it.tk;             // TK * padded_len(My) <= buf_elems (ypass_tk)
  const int k0 = b0 * TK;
  if (k0 > H) return;
  if (TK < 1 || (int64_t)TK * padded_len(1 << log2My) > buf_elems) {
    // a launch sized for a smaller tile: touch nothing, report it
    if (threadIdx.x == 0) atomicAdd(&g_ypass_bad_tiles, 1);
    return;
  }
  extern __shared__ __align__(16) unsigned char smem[];
  Cx<T>* A = reinterpret_cast<Cx<T>*>(smem);
  Cx<T>* B = A + buf_elems;
  Cx<T>* tab = B + buf_elems;
  const int log2N = log2My < 3 ? 3 : log2My;
  load_octant(tab, log2N, tw);
  const int n = TK << log2My;
  const Cx<T> zero = cx(T(0), T(0));
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int m = t / TK, b = t - m * TK, k = k0 + b;
    Cx<T> v = zero;
    if (m < it.in_hi && k <= H) v = it.src[k + (int64_t)ld * m];
    A[(b << log2My) + m] = v;
  }
  __syncthreads();
  Cx<T>* F = A;
  if (mode != Y_INV) F = block_fft_s<T, false>(A, B, log2My, TK, tab, log2N);
  Cx<T>* O = (F == A) ? B : A;
  if (mode == Y_FWD) {
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const int m = t / TK, b = t - m * TK, k = k0 + b;
      if (m < it.out_hi && k <= H) it.dst[k + (int64_t)ld * m] = F[(b << log2My) + m];
    }
    return;
  }
  if (mode == Y_CONVACC) {
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const int m = t / TK, b = t - m * TK, k = k0 + b;
      if (k <= H) {
        const int64_t g = k + (int64_t)ld * m;
        it.dst[g] = it.dst[g] + it.scale * (it.mul[g] * F[(b << log2My) + m]);
      }
    }
    return;
  }
  if (mode == Y_MULCONJ_INV) {
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const int m = t / TK, b = t - m * TK, k = k0 + b;
      const int i = (b << log2My) + m;
      F[i] = (k <= H) ? it.mul[k + (int64_t)ld * m] * conj(F[i]) : zero;
    }
    __syncthreads();
  }
  Cx<T>* R = block_fft_s<T, true>(F, O, log2My, TK, tab, log2N);
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int m = t / TK, b = t - m * TK, k = k0 + b;
    if (m < it.out_hi && k <= H) it.dst[k + (int64_t)ld * m] = R[(b << log2My) + m];
  }
}

// Data to half spectrum, x-pass: masked / missing samples enter as zero
// (they never reach the trajectory matrix); scaled by 1/(Mx My).
template <typename T>
__global__ void __launch_bounds__(512) k_spec_x(const SpecItem<T>* __restrict__ items, Tiles tl,
                                                const Cx<T>* __restrict__ tw) {
  int y;
  const SpecItem<T> it = items[tile_of(tl, blockIdx.x, y)];
  if (y >= it.ny) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int log2H = it.log2Mx - 1, H = 1 << log2H, Mx = 2 * H;
  XSmem<T> sm(smem, H, it.log2Mx, tw);
  T* rb = reinterpret_cast<T*>(sm.A);
  for (int x = threadIdx.x; x < Mx; x += blockDim.x) {
    T v = T(0);
    if (x < it.nx) {
      bool ok = true;
      if (it.obs) ok = (it.obs[(int64_t)y * it.obs_words + (x >> 5)] >> (x & 31)) & 1u;
      const int64_t g = x + it.ld * y;
      if (ok && g < it.n_lin) {
        double d = it.data_double ? ((const double*)it.data)[g] : (double)((const float*)it.data)[g];
        v = (T)d * it.scale;
      }
    }
    rb[x] = v;
  }
  Cx<T>* G = xpass_forward(sm, log2H);
  Cx<T>* dst = ((it.log2My == 0) ? it.xh : it.g1) + (int64_t)y * (H + 1);
  for (int k = threadIdx.x; k <= H; k += blockDim.x) dst[k] = G[k];
}

// ---------------------------------------------------------------- launchers
static inline size_t xsmem_bytes(int log2Mx, size_t csz, bool spec = false) {
  const size_t H = size_t(1) << (log2Mx - 1);
  return align16((2 * (size_t)padded_len((int)H) + H / 4 + 1) * csz) + (spec ? align16((H + 1) * csz) : 0) +
         ((2 * H) / 32 + 1 + 32) * sizeof(int32_t);
}

// y-pass blocks refused for a tile larger than their launch's buffers since
// the last call (read and reset; -1 on a CUDA error)
int ypass_bad_tiles(cudaStream_t st) {
  int h = 0, z = 0;
  if (cudaMemcpyFromSymbolAsync(&h, g_ypass_bad_tiles, sizeof(int), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return -1;
  if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
  if (h) cudaMemcpyToSymbolAsync(g_ypass_bad_tiles, &z, sizeof(int), 0, cudaMemcpyHostToDevice, st);
  return h;
}

// Bulk-copy waits that gave up since the last call (read and reset).
int mv_async_timeouts(cudaStream_t st) {
  int h = 0, z = 0;
  if (cudaMemcpyFromSymbolAsync(&h, g_mv_async_timeouts, sizeof(int), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return -1;
  if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
  if (h) cudaMemcpyToSymbolAsync(g_mv_async_timeouts, &z, sizeof(int), 0, cudaMemcpyHostToDevice, st);
  return h;
}

// Forward transform of u_j = U[:, jc + s] (window side, L FP64 values) on a
// 2^log2M grid, the H packed values before the untwist, straight to global
// memory from the last stage (one block per problem and grid size).
// k_uspec's transform with H = 2^LOG2H fixed at compile time (512 threads)
template <typename T, int LOG2H>
__device__ __forceinline__ void uspec_ct(const UzItem<T>& it, int s, const Cx<T>* __restrict__ tw,
                                         unsigned char* smem) {
  constexpr int H = 1 << LOG2H, LOG2TN = LOG2H + 1;
  Cx<T>* A = reinterpret_cast<Cx<T>*>(smem);
  Cx<T>* B = A + padded_len(H);
  Cx<T>* tab = B + padded_len(H);
  load_octant(tab, LOG2TN, tw);
  __syncthreads();
  const double* src = it.U + it.ldu * (int64_t)(it.st->jc + s);
  const int64_t xe = it.L;
  auto in = [src, xe](int j, int r, int nq) {
    const int64_t x = 2 * (int64_t)(j + r * nq);
    return cx(x < xe ? (T)src[x] : T(0), x + 1 < xe ? (T)src[x + 1] : T(0));
  };
  Cx<T>* z = it.z;
  auto out = [z](int base, int stride, auto& v) {
    constexpr int R = sizeof(v) / sizeof(v[0]);
#pragma unroll
    for (int r = 0; r < R; ++r) z[base + r * stride] = v[r];
  };
  block_fft_io_ct<T, false, LOG2H, 512, LOG2TN>(in, out, A, B, tab);
}

template <typename T>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 2 : 1) k_uspec(const UzItem<T>* __restrict__ items, int s,
                                                                        const Cx<T>* __restrict__ tw) {
  const UzItem<T> it = items[blockIdx.x];
  if (item_skip<T>(it.st, s)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int log2H = it.log2M - 1;
  if constexpr (std::is_same<T, float>::value) {
    // the series workloads' sizes: the transform with its size fixed at
    // compile time (the shared layout is the generic one's)
    if (log2H == 12) { uspec_ct<T, 12>(it, s, tw, smem); return; }
    if (log2H == 11) { uspec_ct<T, 11>(it, s, tw, smem); return; }
    if (log2H == 10) { uspec_ct<T, 10>(it, s, tw, smem); return; }
  }
  XSmem<T> sm(smem, 1 << log2H, it.log2M, tw, false);
  __syncthreads();
  const double* src = it.U + it.ldu * (int64_t)(it.st->jc + s);
  const int64_t xe = it.L;
  auto in = [src, xe](int i) {
    const int64_t x = 2 * (int64_t)i;
    return cx(x < xe ? (T)src[x] : T(0), x + 1 < xe ? (T)src[x + 1] : T(0));
  };
  Cx<T>* z = it.z;
  auto out = [z](int base, int stride, auto& v) {
    constexpr int R = sizeof(v) / sizeof(v[0]);
#pragma unroll
    for (int r = 0; r < R; ++r) z[base + r * stride] = v[r];
  };
  block_fft_io<T, false>(in, out, sm.A, sm.B, log2H, sm.tab, log2H + 1);
}

template <typename T>
void launch_uspec(const UzItem<T>* items, int n, int max_log2M, int s, const Cx<T>* tw, cudaStream_t st) {
  if (n <= 0) return;
  const size_t sm = xsmem_bytes(max_log2M, sizeof(Cx<T>));
  set_max_smem((const void*)k_uspec<T>);
  k_uspec<T><<<n, 512, sm, st>>>(items, s, tw); count_launch();
}

template <typename T, int MODE>
static void launch_mv1d_mode(const MvItem<T>* items, int n, size_t sm, int s, const Cx<T>* tw, cudaStream_t st) {
  set_max_smem((const void*)k_mv1d<T, MODE>);
  k_mv1d<T, MODE><<<n, 512, sm, st>>>(items, s, tw); count_launch();
}

template <typename T>
void launch_mv1d(const MvItem<T>* items, int n, int max_log2Mx, int s, const Cx<T>* tw, cudaStream_t st, int mode) {
  if (n <= 0) return;
  const size_t sm = xsmem_bytes(max_log2Mx, sizeof(Cx<T>), true);
  switch (mode) {
#define SSA_MV1(M) case M: launch_mv1d_mode<T, M>(items, n, sm, s, tw, st); break;
    SSA_MV1(0) SSA_MV1(1) SSA_MV1(2) SSA_MV1(3)
    SSA_MV1(4) SSA_MV1(5) SSA_MV1(6) SSA_MV1(7)
    SSA_MV1(8) SSA_MV1(9) SSA_MV1(10) SSA_MV1(11)
    SSA_MV1(16) SSA_MV1(20) SSA_MV1(24)
#undef SSA_MV1
    default: break;
  }
}

template <typename T>
void launch_mv2d(const MvItem<T>* items, const YItem<T>* yitems, int n, Tiles xf, Tiles yp, Tiles xi,
                 int max_log2Mx, int max_log2My, int s, const Cx<T>* tw, cudaStream_t st, int max_buf) {
  if (n <= 0) return;
  size_t sm = xsmem_bytes(max_log2Mx, sizeof(Cx<T>));
  set_max_smem((const void*)k_mv_xfwd<T>);
  set_max_smem((const void*)k_mv_xinv<T>);
  if (xf.total > 0) { k_mv_xfwd<T><<<xf.total, 512, sm, st>>>(items, xf, s, tw); count_launch(); }
  launch_ypass<T>(yitems, yp, Y_MULCONJ_INV, max_log2My, s, tw, st, max_buf);
  if (xi.total > 0) { k_mv_xinv<T><<<xi.total, 512, sm, st>>>(items, xi, s, tw); count_launch(); }
}

template <typename T>
void launch_ypass(const YItem<T>* items, Tiles tl, int mode, int max_log2My, int s, const Cx<T>* tw,
                  cudaStream_t st, int max_buf) {
  if (tl.total <= 0) return;
  const int buf = std::max(ypass_buf<T>(max_log2My), max_buf);
  const int N = 1 << (max_log2My < 3 ? 3 : max_log2My);
  const size_t sm = (2 * (size_t)buf + N / 8 + 1) * sizeof(Cx<T>);
  set_max_smem((const void*)k_ypass<T>);
  k_ypass<T><<<tl.total, 512, sm, st>>>(items, tl, mode, s, buf, tw); count_launch();
}

template <typename T>
void launch_spec(const SpecItem<T>* items, Tiles sx, const YItem<T>* yitems, Tiles sy, int max_log2Mx,
                 int max_log2My, const Cx<T>* tw, cudaStream_t st, int max_buf) {
  if (sx.total <= 0) return;
  size_t sm = xsmem_bytes(max_log2Mx, sizeof(Cx<T>));
  set_max_smem((const void*)k_spec_x<T>);
  k_spec_x<T><<<sx.total, 512, sm, st>>>(items, sx, tw); count_launch();
  if (max_log2My > 0) launch_ypass<T>(yitems, sy, Y_FWD, max_log2My, -1, tw, st, max_buf);
}

#define INST(T)                                                                                       \
  template void launch_mv1d<T>(const MvItem<T>*, int, int, int, const Cx<T>*, cudaStream_t, int);     \
  template void launch_uspec<T>(const UzItem<T>*, int, int, int, const Cx<T>*, cudaStream_t);          \
  template void launch_mv2d<T>(const MvItem<T>*, const YItem<T>*, int, Tiles, Tiles, Tiles, int, int,  \
                               int, const Cx<T>*, cudaStream_t, int);                                 \
  template void launch_ypass<T>(const YItem<T>*, Tiles, int, int, int, const Cx<T>*, cudaStream_t, int); \
  template void launch_spec<T>(const SpecItem<T>*, Tiles, const YItem<T>*, Tiles, int, int,           \
                               const Cx<T>*, cudaStream_t, int);
INST(float)
INST(double)

}  // namespace ssa
