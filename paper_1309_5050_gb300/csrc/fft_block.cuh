// Block-cooperative FFTs in shared memory, and the packed real-to-half-spectrum
// conversions used by every pass.
//
// Complex DFT convention (Sec. 6.1.1, eq. fft_def): Y_k = sum_n x_n W^{nk},
// W = exp(-2 pi i / n); the inverse uses W^{-1} and is left unnormalised here
// (all scale factors are folded into the precomputed data spectrum).
//
// block_fft runs the Stockham autosort algorithm (published by Stockham, in
// the GPU form of Govindaraju et al., SC'08): log2(n) is split into radix-8
// stages plus one radix-4 or radix-2 stage; each stage reads R values with
// stride n/R, multiplies by W_{Ns R}^{k r}, does an R-point DFT and writes
// them with stride Ns, ping-ponging between two shared buffers.
#pragma once
#include "common.cuh"

namespace ssa {

template <typename T, bool INV>
__device__ __forceinline__ void dft2(Cx<T>& a, Cx<T>& b) {
  Cx<T> t = a - b;
  a = a + b;
  b = t;
}

// multiply by the 4th root W_4 = -i (forward) or +i (inverse)
template <typename T, bool INV>
__device__ __forceinline__ Cx<T> rot4(Cx<T> a) { return INV ? mul_pi(a) : mul_mi(a); }

template <typename T, bool INV>
__device__ __forceinline__ void dft4(Cx<T>& v0, Cx<T>& v1, Cx<T>& v2, Cx<T>& v3) {
  Cx<T> t0 = v0 + v2, t1 = v0 - v2, t2 = v1 + v3, t3 = rot4<T, INV>(v1 - v3);
  v0 = t0 + t2;
  v2 = t0 - t2;
  v1 = t1 + t3;
  v3 = t1 - t3;
}

template <typename T, bool INV>
__device__ __forceinline__ void dft8(Cx<T>* v) {
  // split into even / odd 4-point DFTs, then combine with W_8^k
  dft4<T, INV>(v[0], v[2], v[4], v[6]);
  dft4<T, INV>(v[1], v[3], v[5], v[7]);
  const T h = T(0.70710678118654752440084436210485);
  Cx<T> o1 = v[3], o2 = v[5], o3 = v[7];
  // W_8^1 = (1 - i)/sqrt2, W_8^2 = -i, W_8^3 = (-1 - i)/sqrt2 (conjugates for INV)
  if (!INV) {
    o1 = cx(h * (o1.re + o1.im), h * (o1.im - o1.re));
    o2 = mul_mi(o2);
    o3 = cx(h * (o3.im - o3.re), -h * (o3.re + o3.im));
  } else {
    o1 = cx(h * (o1.re - o1.im), h * (o1.re + o1.im));
    o2 = mul_pi(o2);
    o3 = cx(-h * (o3.re + o3.im), h * (o3.re - o3.im));
  }
  Cx<T> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
  v[0] = e0 + o0; v[4] = e0 - o0;
  v[1] = e1 + o1; v[5] = e1 - o1;
  v[2] = e2 + o2; v[6] = e2 - o2;
  v[3] = e3 + o3; v[7] = e3 - o3;
}

template <typename T, bool INV, int LR>
__device__ __forceinline__ void stockham_stage(const Cx<T>* __restrict__ src, Cx<T>* __restrict__ dst,
                                               int log2n, int nb, int log2Ns, const Cx<T>* tw) {
  constexpr int R = 1 << LR;
  const int n = 1 << log2n;
  const int nq = n >> LR;            // butterflies per transform
  const int Ns = 1 << log2Ns;
  const int total = nq * nb;
  for (int jj = threadIdx.x; jj < total; jj += blockDim.x) {
    const int b = jj >> (log2n - LR);
    const int j = jj & (nq - 1);
    const Cx<T>* s = src + ((int64_t)b << log2n);
    Cx<T>* d = dst + ((int64_t)b << log2n);
    const int k = j & (Ns - 1);
    Cx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = s[j + r * nq];
    if (log2Ns > 0) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        Cx<T> w = twid(tw, log2Ns + LR, (int64_t)k * r);
        if (INV) w = conj(w);
        v[r] = v[r] * w;
      }
    }
    if (LR == 3) dft8<T, INV>(v);
    else if (LR == 2) dft4<T, INV>(v[0], v[1], v[2], v[3]);
    else dft2<T, INV>(v[0], v[1]);
    const int base = ((j - k) << LR) + k;
#pragma unroll
    for (int r = 0; r < R; ++r) d[base + r * Ns] = v[r];
  }
}

// nb independent transforms of length 2^log2n stored back to back in a.
// Returns the buffer (a or b) holding the result.  Caller syncs before.
template <typename T, bool INV>
__device__ Cx<T>* block_fft(Cx<T>* a, Cx<T>* b, int log2n, int nb, const Cx<T>* tw) {
  int done = 0;
  while (done < log2n) {
    int rem = log2n - done;
    if (rem >= 3) stockham_stage<T, INV, 3>(a, b, log2n, nb, done, tw), done += 3;
    else if (rem == 2) stockham_stage<T, INV, 2>(a, b, log2n, nb, done, tw), done += 2;
    else stockham_stage<T, INV, 1>(a, b, log2n, nb, done, tw), done += 1;
    __syncthreads();
    Cx<T>* t = a; a = b; b = t;
  }
  return a;
}

// ---------------------------------------------------------------- shared tables
// Octant twiddle table in shared memory: tab[m] = W_N^m for m in [0, N/8],
// N = 2^log2N >= 8, copied from the global table (correctly rounded values).
// Any W_N^j follows exactly: W_N^{qN/4 + m} = (-i)^q W_N^m, and for
// N/8 < m < N/4, W_N^m = -i conj(W_N^{N/4 - m}) -- sign changes and swaps only.
template <typename T>
__device__ __forceinline__ void load_octant(Cx<T>* tab, int log2N, const Cx<T>* __restrict__ tw) {
  const int n8 = (1 << log2N) >> 3;
  for (int m = threadIdx.x; m <= n8; m += blockDim.x) tab[m] = tw[(int64_t)m << (TW_LOG - log2N)];
}

template <typename T>
__device__ __forceinline__ Cx<T> tw_oct(const Cx<T>* tab, int log2N, int64_t j) {
  const int N = 1 << log2N;
  const int jj = (int)(j & (N - 1));
  const int q = jj >> (log2N - 2);
  const int m = jj & ((N >> 2) - 1);
  Cx<T> w;
  if (m <= (N >> 3)) {
    w = tab[m];
  } else {
    const Cx<T> t = tab[(N >> 2) - m];
    w = cx(-t.im, -t.re);
  }
  if (q == 1) w = cx(w.im, -w.re);
  else if (q == 2) w = cx(-w.re, -w.im);
  else if (q == 3) w = cx(-w.im, w.re);
  return w;
}

// Padded shared layout of the intermediate Stockham buffers: one spare slot
// per 16 elements, so the scattered stores of the early radix-8 stages hit
// distinct banks.  First-stage loads and last-stage stores stay unpadded
// (both are already contiguous across a warp).
__device__ __forceinline__ int padi(int i) { return i + (i >> 4); }
__host__ __device__ __forceinline__ int padded_len(int n) { return n + (n >> 4) + 1; }

template <typename T, bool INV, int LR, bool PIN, bool POUT>
__device__ __forceinline__ void stockham_stage_s(const Cx<T>* __restrict__ src, Cx<T>* __restrict__ dst,
                                                 int log2n, int nb, int sin, int sout, int log2Ns,
                                                 const Cx<T>* tab, int log2N) {
  constexpr int R = 1 << LR;
  const int n = 1 << log2n;
  const int nq = n >> LR;
  const int Ns = 1 << log2Ns;
  const int total = nq * nb;
  const int tshift = log2N - (log2Ns + LR);    // W_{Ns R}^a = W_N^{a << tshift}
  for (int jj = threadIdx.x; jj < total; jj += blockDim.x) {
    const int b = jj >> (log2n - LR);
    const int j = jj & (nq - 1);
    const Cx<T>* s = src + b * sin;
    Cx<T>* d = dst + b * sout;
    const int k = j & (Ns - 1);
    Cx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = j + r * nq;
      v[r] = s[PIN ? padi(i) : i];
    }
    if (log2Ns > 0) {
      // W^{k r} for r = 1..R-1 from one table value by products (a few
      // roundings more than separate lookups, far fewer instructions)
      Cx<T> w1 = tw_oct(tab, log2N, (int64_t)k << tshift);
      if (INV) w1 = conj(w1);
      Cx<T> w = w1;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        v[r] = v[r] * w;
        if (r + 1 < R) w = w * w1;
      }
    }
    if (LR == 3) dft8<T, INV>(v);
    else if (LR == 2) dft4<T, INV>(v[0], v[1], v[2], v[3]);
    else dft2<T, INV>(v[0], v[1]);
    const int base = ((j - k) << LR) + k;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = base + r * Ns;
      d[POUT ? padi(i) : i] = v[r];
    }
  }
}

// nb transforms of length 2^log2n.  Input: unpadded, transform b at a + b*n.
// Output (returned buffer): unpadded, transform b at out + b*n.  Both buffers
// must hold nb * padded_len(n) elements.  Twiddles from the octant table of
// W_N (N >= n, N >= 8).  Caller syncs before.
template <typename T, bool INV>
__device__ Cx<T>* block_fft_s(Cx<T>* a, Cx<T>* b, int log2n, int nb, const Cx<T>* tab, int log2N) {
  const int n = 1 << log2n;
  const int sp = padded_len(n);
  int done = 0;
  bool first = true;
  while (done < log2n) {
    const int rem = log2n - done;
    const int lr = rem >= 3 ? 3 : rem;
    const bool last = (done + lr == log2n);
    const int sin = first ? n : sp, sout = last ? n : sp;
#define SSA_STAGE(LRV, PI, PO) stockham_stage_s<T, INV, LRV, PI, PO>(a, b, log2n, nb, sin, sout, done, tab, log2N)
    if (lr == 3) {
      if (first && last) SSA_STAGE(3, false, false);
      else if (first) SSA_STAGE(3, false, true);
      else if (last) SSA_STAGE(3, true, false);
      else SSA_STAGE(3, true, true);
    } else if (lr == 2) {
      if (first && last) SSA_STAGE(2, false, false);
      else if (first) SSA_STAGE(2, false, true);
      else if (last) SSA_STAGE(2, true, false);
      else SSA_STAGE(2, true, true);
    } else {
      if (first && last) SSA_STAGE(1, false, false);
      else if (first) SSA_STAGE(1, false, true);
      else if (last) SSA_STAGE(1, true, false);
      else SSA_STAGE(1, true, true);
    }
#undef SSA_STAGE
    done += lr;
    first = false;
    __syncthreads();
    Cx<T>* t = a; a = b; b = t;
  }
  return a;
}

// One radix-2^LR Stockham stage of a single transform (nb = 1) whose input
// element i comes from in(i) and whose R outputs base + r * stride go to
// out(base, stride, v[R]) together (so an output functor can issue all its
// global loads before its stores): the first stage can read global memory and
// the last one write it directly.
template <typename T, bool INV, int LR, class In, class Out>
__device__ __forceinline__ void stage_io(In& in, Out& out, int log2n, int log2Ns, const Cx<T>* tab, int log2N) {
  constexpr int R = 1 << LR;
  const int nq = (1 << log2n) >> LR;
  const int Ns = 1 << log2Ns;
  const int tshift = log2N - (log2Ns + LR);
  for (int j = threadIdx.x; j < nq; j += blockDim.x) {
    const int k = j & (Ns - 1);
    Cx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in(j + r * nq);
    if (log2Ns > 0) {
      Cx<T> w1 = tw_oct(tab, log2N, (int64_t)k << tshift);
      if (INV) w1 = conj(w1);
      Cx<T> w = w1;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        v[r] = v[r] * w;
        if (r + 1 < R) w = w * w1;
      }
    }
    if (LR == 3) dft8<T, INV>(v);
    else if (LR == 2) dft4<T, INV>(v[0], v[1], v[2], v[3]);
    else dft2<T, INV>(v[0], v[1]);
    const int base = ((j - k) << LR) + k;
    out(base, Ns, v);
  }
}

// Stages of one transform of length 2^log2n: the first reads in(i), the last
// hands its outputs to out(base, stride, v), the ones between ping-pong through
// the padded buffers (the first stage writes b).  The first stage takes the
// 1..3 leftover bits and every later stage is radix 8, which keeps the number
// of stage bodies the compiler emits small.  A barrier follows every stage.
template <typename T, bool INV, class In, class Out>
__device__ void block_fft_io(In in, Out out, Cx<T>* a, Cx<T>* b, int log2n, const Cx<T>* tab, int log2N) {
  auto wr = [b](int base, int stride, auto& v) {
    constexpr int R = sizeof(v) / sizeof(v[0]);
#pragma unroll
    for (int r = 0; r < R; ++r) b[padi(base + r * stride)] = v[r];
  };
  const int lr0 = log2n - 3 * ((log2n - 1) / 3);   // 1..3
  if (lr0 == log2n) {                                // a single stage
    if (lr0 == 3) stage_io<T, INV, 3>(in, out, log2n, 0, tab, log2N);
    else if (lr0 == 2) stage_io<T, INV, 2>(in, out, log2n, 0, tab, log2N);
    else stage_io<T, INV, 1>(in, out, log2n, 0, tab, log2N);
    __syncthreads();
    return;
  }
  if (lr0 == 3) stage_io<T, INV, 3>(in, wr, log2n, 0, tab, log2N);
  else if (lr0 == 2) stage_io<T, INV, 2>(in, wr, log2n, 0, tab, log2N);
  else stage_io<T, INV, 1>(in, wr, log2n, 0, tab, log2N);
  __syncthreads();
  Cx<T>* src = b;
  Cx<T>* dst = a;
  for (int done = lr0; done < log2n; done += 3) {
    auto rd = [src](int i) { return src[padi(i)]; };
    if (done + 3 == log2n) {
      stage_io<T, INV, 3>(rd, out, log2n, done, tab, log2N);
    } else {
      auto wd = [dst](int base, int stride, auto& v) {
        constexpr int R = sizeof(v) / sizeof(v[0]);
#pragma unroll
        for (int r = 0; r < R; ++r) dst[padi(base + r * stride)] = v[r];
      };
      stage_io<T, INV, 3>(rd, wd, log2n, done, tab, log2N);
    }
    __syncthreads();
    Cx<T>* t = src; src = dst; dst = t;
  }
}

// ---------------------------------------------------------------- compile-time sizes
// The same Stockham transform with the length 2^LOG2N, the block size NT and
// the twiddle table order LOG2TN (octant table of W_{2^LOG2TN}) known at
// compile time: every index, stride, padding offset and loop count folds to
// constants, which removes most of the integer work of the runtime form (the
// series product is issue-bound).  Stage with LR = log2 radix after LOG2NS
// bits; its NQ = 2^(LOG2N - LR) butterflies are spread over the NT threads.
template <typename T, bool INV, int LR, int LOG2N, int LOG2NS, int NT, int LOG2TN, class In, class Out>
__device__ __forceinline__ void stage_ct(In& in, Out& out, const Cx<T>* tab) {
  constexpr int R = 1 << LR;
  constexpr int NQ = (1 << LOG2N) >> LR;
  constexpr int NS = 1 << LOG2NS;
  constexpr int TSHIFT = LOG2TN - (LOG2NS + LR);     // W_{NS R}^a = W_{2^LOG2TN}^{a << TSHIFT}
  constexpr int ITER = (NQ + NT - 1) / NT;
#pragma unroll
  for (int it = 0; it < ITER; ++it) {
    const int j = (int)threadIdx.x + it * NT;
    if (NQ % NT != 0 && j >= NQ) break;
    const int k = j & (NS - 1);
    Cx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in(j, r, NQ);      // element j + r NQ
    if (LOG2NS > 0) {
      Cx<T> w1 = tw_oct(tab, LOG2TN, (int64_t)k << TSHIFT);
      if (INV) w1 = conj(w1);
      Cx<T> w = w1;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        v[r] = v[r] * w;
        if (r + 1 < R) w = w * w1;
      }
    }
    if (LR == 3) dft8<T, INV>(v);
    else if (LR == 2) dft4<T, INV>(v[0], v[1], v[2], v[3]);
    else dft2<T, INV>(v[0], v[1]);
    out(((j - k) << LR) + k, NS, v);
  }
}

// radix-8 stages after the first DONE bits, ping-ponging between the padded
// buffers src and dst; the last one hands its outputs to out
// Padded element j + r nq with j < nq and 16 | nq: padi(j) + r (nq + nq / 16),
// a constant offset per r once nq is a compile-time constant.
template <typename T>
__device__ __forceinline__ Cx<T> padded_at(const Cx<T>* src, int j, int r, int nq) {
  return (nq & 15) ? src[padi(j + r * nq)] : src[padi(j) + r * (nq + (nq >> 4))];
}
// padded store of a butterfly's outputs base + r stride (16 | stride: constant offsets)
template <typename T, int R>
__device__ __forceinline__ void padded_put(Cx<T>* dst, int base, int stride, const Cx<T> (&v)[R]) {
  if (stride & 15) {
#pragma unroll
    for (int r = 0; r < R; ++r) dst[padi(base + r * stride)] = v[r];
  } else {
    const int pb = padi(base);
#pragma unroll
    for (int r = 0; r < R; ++r) dst[pb + r * (stride + (stride >> 4))] = v[r];
  }
}

template <typename T, bool INV, int LOG2N, int DONE, int NT, int LOG2TN, class Out>
__device__ __forceinline__ void stages8_ct(Cx<T>* src, Cx<T>* dst, Out& out, const Cx<T>* tab) {
  auto rd = [src](int j, int r, int nq) { return padded_at(src, j, r, nq); };
  if constexpr (DONE + 3 == LOG2N) {
    stage_ct<T, INV, 3, LOG2N, DONE, NT, LOG2TN>(rd, out, tab);
    __syncthreads();
  } else {
    auto wd = [dst](int base, int stride, auto& v) { padded_put(dst, base, stride, v); };
    stage_ct<T, INV, 3, LOG2N, DONE, NT, LOG2TN>(rd, wd, tab);
    __syncthreads();
    stages8_ct<T, INV, LOG2N, DONE + 3, NT, LOG2TN>(dst, src, out, tab);
  }
}

// block_fft_io with compile-time sizes (LOG2N >= 4): first stage of the 1..3
// leftover bits from in(j, r, nq) (element j + r nq), radix-8 stages after
// it, the last to out(base, stride, v).  A barrier follows every stage.
template <typename T, bool INV, int LOG2N, int NT, int LOG2TN, class In, class Out>
__device__ __forceinline__ void block_fft_io_ct(In in, Out out, Cx<T>* a, Cx<T>* b, const Cx<T>* tab) {
  static_assert(LOG2N >= 4, "compile-time form needs at least two stages");
  constexpr int LR0 = LOG2N - 3 * ((LOG2N - 1) / 3);   // 1..3
  auto wr = [b](int base, int stride, auto& v) { padded_put(b, base, stride, v); };
  stage_ct<T, INV, LR0, LOG2N, 0, NT, LOG2TN>(in, wr, tab);
  __syncthreads();
  stages8_ct<T, INV, LOG2N, LR0, NT, LOG2TN>(b, a, out, tab);
}

// number of stages block_fft_io runs for length 2^log2n
__host__ __device__ __forceinline__ int fft_io_stages(int log2n) { return (log2n + 2) / 3; }

template <typename T>
__device__ __forceinline__ Cx<T> untwist_fwd_s(const Cx<T>* Z, int k, int log2H, const Cx<T>* tab) {
  const int H = 1 << log2H;
  Cx<T> a = Z[k & (H - 1)];
  Cx<T> b = conj(Z[(H - k) & (H - 1)]);
  Cx<T> E = T(0.5) * (a + b);
  Cx<T> O = T(0.5) * mul_mi(a - b);
  return E + tw_oct(tab, log2H + 1, k) * O;
}

template <typename T>
__device__ __forceinline__ Cx<T> twist_inv_s(const Cx<T>* P, int k, int log2H, const Cx<T>* tab) {
  const int H = 1 << log2H;
  Cx<T> a = P[k];
  Cx<T> b = conj(P[H - k]);
  Cx<T> w = conj(tw_oct(tab, log2H + 1, k));
  return (a + b) + mul_pi(w * (a - b));
}

// Packed real transform, forward: z[n] = g[2n] + i g[2n+1] (length H) has
// been transformed to Z; produce the half spectrum G[k], k = 0..H, of the real
// length-2H signal g:  G[k] = E + W^k O,  E = (Z[k] + conj Z[H-k]) / 2,
// O = -i (Z[k] - conj Z[H-k]) / 2,  W = exp(-2 pi i / 2H).
template <typename T>
__device__ __forceinline__ Cx<T> untwist_fwd(const Cx<T>* Z, int k, int log2H, const Cx<T>* tw) {
  const int H = 1 << log2H;
  Cx<T> a = Z[k & (H - 1)];
  Cx<T> b = conj(Z[(H - k) & (H - 1)]);
  Cx<T> E = T(0.5) * (a + b);
  Cx<T> O = T(0.5) * mul_mi(a - b);
  return E + twid(tw, log2H + 1, k) * O;
}

// Packed real transform, inverse: from a half spectrum P[0..H] of a real
// signal r of length 2H, form Q[k] (k < H) whose unnormalised inverse
// length-H transform is r[2n] + i r[2n+1] times 2H:
// Q[k] = (P[k] + conj P[H-k]) + i W^{-k} (P[k] - conj P[H-k]).
template <typename T>
__device__ __forceinline__ Cx<T> twist_inv(const Cx<T>* P, int k, int log2H, const Cx<T>* tw) {
  const int H = 1 << log2H;
  Cx<T> a = P[k];
  Cx<T> b = conj(P[H - k]);
  Cx<T> w = conj(twid(tw, log2H + 1, k));
  return (a + b) + mul_pi(w * (a - b));
}

// Exclusive prefix of popcounts of n words (n <= 32 * blockDim.x), result in
// out[0..n).  Uses out as scratch; ends with __syncthreads.
__device__ __forceinline__ void block_popc_scan(const uint32_t* words, int n, int32_t* out,
                                                int32_t* warp_tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  for (int base = 0; base < n; base += blockDim.x) {
    int i = base + threadIdx.x;
    int v = (i < n) ? __popc(words[i]) : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
      int carry = (base == 0) ? 0 : out[base - 1] + __popc(words[base - 1]);
      for (int w = 0; w < nw; ++w) { int t = warp_tot[w]; warp_tot[w] = carry; carry += t; }
    }
    __syncthreads();
    if (i < n) out[i] = x - v + warp_tot[warp];
    __syncthreads();
  }
}

}  // namespace ssa
