// Shared device-side definitions of the SSA library (sm_103a).
//
// Layout conventions used by every kernel:
//  * A problem lives on a grid of Mx x My real samples (My = 1 for series),
//    column-major: sample (x, y) sits at x + Mx*y.  Mx, My are powers of two
//    with Mx >= Nx and My >= Ny, which keeps every window product inside one
//    period of the circulant (the L x K Hankel / quasi-Hankel matrix is a
//    sub-matrix of the Mx x My HbH circulant of the zero-padded data,
//    Sec. 6.1.2 and 6.2.2).
//  * Half spectra are stored per grid column y as H+1 complex values
//    (H = Mx/2): element (k, y) at k + (H+1)*y.
//  * A compact vector (a window vector U_i, a factor vector V_i, or one slice
//    of it) is mapped to grid positions by a MapDev: either a dense rectangle
//    [0,bx) x [0,by) in column-major order, or per-column bit masks with a
//    per-column prefix count (lexicographic order of Sec. 5.1).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ssa {

template <typename T> struct __align__(2 * sizeof(T)) Cx { T re, im; };

template <typename T> __device__ __forceinline__ Cx<T> cx(T r, T i) { Cx<T> c; c.re = r; c.im = i; return c; }
template <typename T> __device__ __forceinline__ Cx<T> operator+(Cx<T> a, Cx<T> b) { return cx(a.re + b.re, a.im + b.im); }
template <typename T> __device__ __forceinline__ Cx<T> operator-(Cx<T> a, Cx<T> b) { return cx(a.re - b.re, a.im - b.im); }
template <typename T> __device__ __forceinline__ Cx<T> operator*(Cx<T> a, Cx<T> b) {
  return cx(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T> __device__ __forceinline__ Cx<T> operator*(T s, Cx<T> a) { return cx(s * a.re, s * a.im); }
template <typename T> __device__ __forceinline__ Cx<T> conj(Cx<T> a) { return cx(a.re, -a.im); }
// multiply by -i / +i
template <typename T> __device__ __forceinline__ Cx<T> mul_mi(Cx<T> a) { return cx(a.im, -a.re); }
template <typename T> __device__ __forceinline__ Cx<T> mul_pi(Cx<T> a) { return cx(-a.im, a.re); }

// Twiddle table: tw[j] = exp(-2 pi i j / TW_N), j < TW_N, written once per
// device by the library (values computed in double, rounded for float).
constexpr int TW_LOG = 15;
constexpr int TW_N = 1 << TW_LOG;

template <typename T> struct Tw;
template <> struct Tw<float> { const Cx<float>* p; };
template <> struct Tw<double> { const Cx<double>* p; };

// W_n^m = exp(-2 pi i m / n) for n a power of two <= TW_N (m taken mod n).
template <typename T>
__device__ __forceinline__ Cx<T> twid(const Cx<T>* tw, int log2n, int64_t m) {
  int64_t idx = (m << (TW_LOG - log2n)) & (TW_N - 1);
  return tw[idx];
}

// Map between a compact vector and grid positions (see file comment).
struct MapDev {
  int32_t dense;           // 1: rectangle [0,bx) x [0,by), index x + bx*y
  int32_t bx, by;          // bounding box of the set
  int32_t words;           // 32-bit words per column (bit mode)
  const uint32_t* bits;    // by * words, bit x of column y at word x>>5, bit x&31
  const int32_t* colbase;  // by: number of set elements in columns < y
  int64_t limit;           // dense mode: only indices x + bx*y < limit belong to the set
};

// Batched launches over items of different sizes: item i owns the blocks
// [pre[i], pre[i+1]) of a one-dimensional grid (pre[n] = grid size).  Returns
// the item of block b and sets the block's index within it.
__device__ __forceinline__ int tile_item(const int32_t* __restrict__ pre, int n, int b, int& local) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(pre + mid) <= b) lo = mid;
    else hi = mid - 1;
  }
  local = b - __ldg(pre + lo);
  return lo;
}

// Error word written by kernels that detect bad input or a stalled wait.
enum : int { DEV_OK = 0, DEV_BAD_INPUT = 1 };

__device__ __forceinline__ int ilog2(int n) { return 31 - __clz(n); }
__device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

}  // namespace ssa
