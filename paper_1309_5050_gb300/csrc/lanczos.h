// Lanczos bidiagonalisation work items and launchers (internal).
//
// The operator A is the trajectory matrix or its transpose, oriented so that
// its rows are the shorter side ("short", length Ls) and its columns the longer
// ("long", length Kl).  Golub-Kahan-Lanczos steps build
//   A V_k = U_k B_k,   A^T U_k = V_k B_k^T + beta_k v_{k+1} e_k^T,
// with U (short side, FP64) fully re-orthogonalised by classical Gram-Schmidt
// applied twice, and V (long side, storage type T) left as the three-term
// recurrence makes it (one-sided re-orthogonalisation, as in Simon and Zha's
// and Baglama and Reichel's bidiagonalisation methods).  After k steps the
// small B is decomposed; if the r leading triples have not converged, the
// method restarts from the kk best Ritz vectors (thick / augmented restart).
#pragma once
#include <cuda_runtime.h>
#include "kernels.cuh"

namespace ssa {

constexpr int SHORT_RB = 256;   // rows per CTA on the short side
constexpr int LONG_RB = 2048;   // rows per CTA on the long side
constexpr int KMAX = 112;       // largest Krylov dimension (small SVD in shared memory)

struct ShortItem {
  LzState* st;
  double* U; int64_t ldu;                 // Ls x (k+1), FP64
  float* Uh; float* Ul; int64_t ldf;      // FP32 form: float-float copy of U as hi and lo parts
                                          // (ldf = Ls rounded up to a multiple of four, zero pad
                                          // rows: 16-byte aligned columns), else null
  const void* parts; int64_t part_ld;     // n_part partial products (type of the matvec)
  int32_t n_part; int32_t parts_double;
  double* p;                              // work vector, Ls
  double* B; int32_t ldb; int32_t nblk;   // B column-major, ldb = k
  double* cpa; double* cpb;               // nblk x (KMAX+1) partial dots
  double* npart;                          // nblk partial squared norms
  int64_t Ls;
  uint64_t seed;                          // seeds the replacement vectors after a breakdown
};

// Breakdown test.  A Lanczos coefficient at the rounding level of the
// products (alpha_j or beta_j <= the larger of LzState::bd_floor = 4 eps
// log2(grid) ||x|| -- one FFT product with a unit vector is exact to about
// eps log2 M ||x|| -- and BD_REL times the largest coefficient so far) means
// the Krylov space is invariant to working precision: the data has exact rank
// below k, or a multiple singular value whose other copies one start vector
// cannot reach.  Normalising that residual would feed rounding noise into the
// basis (the long side is not re-orthogonalised, so the bases lose
// orthogonality and B stops describing A).  Instead the coefficient is set to
// 0: on the short side u_j becomes a seeded random vector orthogonalised twice
// against U; on the long side v_{j+1} becomes the zero vector, so the next
// short step breaks down too and X^T of its random u starts the next block
// (orthogonal to V in exact arithmetic, see k_long_norm).  The bidiagonal
// splits into blocks and the process goes on in the rest of the space.  The floor follows the data's
// scale, not sigma_1: a long series with a steep trend has legitimate noise
// singular values near 1e-6 sigma_1, far above its products' rounding.
constexpr double BD_REL_FP64 = 1e-12;
constexpr double BD_REL_FP32 = 1e-9;

template <typename T>
struct LongItem {
  LzState* st;
  T* V; int64_t ldv;                      // Kl x (k+1), columns stored unnormalised
  double* colscale;                       // k+1: column c of V times colscale[c] is v_c
  const T* parts; int64_t part_ld; int32_t n_part; int32_t nblk;
  T* q;                                   // work vector, Kl
  double* npart;                          // partial squared norms
  double* B; int32_t ldb;
  int32_t nsum;                           // partial norms of a step (nblk, or the fused products' count)
  int64_t Kl;
  uint64_t seed;
};

// Shared memory of the small SVD for a k-row W of nc columns: the FP64 W
// (column stride cs = k | 1), V and E (nc x nc FP32, stride lv = nc | 1), and
// V' in FP64 (stride s0).  Region 0 (nc x s0 doubles) holds the FP32 copy of
// W0, then V'; region 1 (nc x lv floats twice) holds V and E, then the FP64 W;
// region 2 (k x k doubles, stride cs), when the launch gives room for it, a
// copy of B for the products with it (W0 V' and W0^T P), which otherwise read
// B from global memory.
struct BsvdLayout { int cs, lv, s0; size_t bytes, bytes_b; };
__host__ __device__ inline BsvdLayout bsvd_layout(int k, int nc) {
  BsvdLayout l;
  l.cs = k | 1;
  l.lv = nc | 1;
  l.s0 = l.cs > l.lv ? l.cs : l.lv;
  l.bytes = sizeof(double) * (size_t)nc * l.s0 + 2 * sizeof(float) * (size_t)nc * l.lv;
  l.bytes_b = l.bytes + sizeof(double) * (size_t)k * l.cs;
  return l;
}

struct SvdItem {
  LzState* st;
  double* B; int32_t ldb;
  int32_t ffpolish;                       // FP32 form: the polish in float-float (bsvd_tail_ff)
  double* colscale;                       // long-basis column scales (reset on restart)
  double* sig;                            // k singular values (descending)
  double* P;                              // k x k left vectors of B (ld k)
  double* Q;                              // k x k right vectors of B (ld k)
};

template <typename T>
struct RitzItem {
  LzState* st;
  double* U; int64_t ldu; int64_t Ls;     // short basis
  T* V; int64_t ldv; int64_t Kl;          // long basis (column scales below)
  double* colscale;
  const double* P; const double* Q;       // from the small SVD
  int32_t ldc; int32_t ldcs;              // their leading dimension (allocated k); row length of Cs
  T* Cs;                                  // long-side coefficients Q[i, c] * colscale[i] as T, row-major
  float* Uh; float* Ul; int64_t ldf;      // FP32 form: the short basis's float-float copy, else null
};
// row length of the scaled long-side coefficients for an allocated Krylov dimension k
inline int ritz_ldcs(int k) { return ((k + 63) / 64) * 64; }

template <typename T>
struct FinalItem {
  LzState* st;
  const double* U; int64_t ldu; int64_t Ls;   // short basis (Ritz vectors in the first r columns)
  const T* V; int64_t ldv; int64_t Kl;
  const double* sig;
  int32_t swapped;                            // 1: the short side is the K side
  int32_t r;
  T* Uo; T* Vo;                               // canonical outputs: L x r, K x r
  double* sigma_out;                          // r
  double* sgn;                                // r signs (scratch)
};

// Row-block launches are tile-mapped: item i owns blocks [tpre[i], tpre[i+1])
// (short side ceil(Ls / SHORT_RB), long side ceil(Kl / LONG_RB), Ritz
// ceil(rows / RITZ_RB_*)), tiles = tpre[n].
template <typename E>
constexpr int RITZ_RB() { return sizeof(E) == 8 ? 64 : 256; }   // rows per Ritz block
template <typename E>
constexpr int RITZ_CW() { return sizeof(E) == 8 ? 4 : 8; }      // columns per thread tile
constexpr int RITZ_RB_SHORT = RITZ_RB<double>();
// FP32 long side: the tensor-core kernel (k_ritz_tc.cu) takes 128-row tiles
constexpr int RITZ_TC_M = 128;
template <typename T>
constexpr int ritz_rb_long() { return sizeof(T) == 4 ? RITZ_TC_M : RITZ_RB<T>(); }
void launch_short_steps(const ShortItem* items, const int32_t* tpre, int n, int tiles, int s, cudaStream_t st);
// Problems whose short side has at most SHORT_FUSED_MAX rows: the whole
// short-side step in one block per problem (items: only those problems).
constexpr int SHORT_FUSED_MAX = 4096;
void launch_short_fused(const ShortItem* items, int n, int64_t max_ls, int s, cudaStream_t st);
// The same steps in float-float arithmetic on U's copy (Uh, Ul) (the FP32
// form; see ff.cuh): p, the Gram-Schmidt coefficients and the partial sums
// are float-float, u_j is written to U, Uh and Ul.
void launch_short_steps_ff(const ShortItem* items, const int32_t* tpre, int n, int tiles, int s, cudaStream_t st);
void launch_short_fused_ff(const ShortItem* items, int n, int64_t max_ls, int s, cudaStream_t st);
// (Uh, Ul)[:, 0:ncols[i]] <- U[:, 0:ncols[i]] of item i (after a restart or a
// resumed decomposition rewrote U in FP64)
void launch_uf_sync(const ShortItem* items, const int32_t* ncols, int n, cudaStream_t st);
// Bulk-copy waits of the float-float short side that gave up since the last call
// (read and reset; -1 on a CUDA error).
int short_tma_timeouts(cudaStream_t st);
// device address of that counter (current device), for a read-back that
// rides along with other copies; null on a CUDA error
int* short_tma_timeout_word();
template <typename T>
void launch_long_step(const LongItem<T>* items, const int32_t* tpre, int n, int tiles, int s, cudaStream_t st);
template <typename T>
void launch_long_init(const LongItem<T>* items, const int32_t* tpre, int n, int tiles, cudaStream_t st);
void launch_bsvd(const SvdItem* items, int n, int kmax, cudaStream_t st);
void launch_restart(const SvdItem* items, int n, cudaStream_t st);
// kmax / kkmax: largest Krylov dimension and largest number of kept columns
// (restart: kk; final pass: r) among the items
template <typename T>
void launch_ritz(const RitzItem<T>* items, int n, int kmax, int kkmax, const int32_t* pre_s, int tiles_s,
                 const int32_t* pre_l, int tiles_l, int final_pass, cudaStream_t st);
// FP32 long side on the tensor cores (k_ritz_tc.cu): 128-row tiles, tcgen05.mma
// kind::tf32 with each operand split into two TF32 parts
void launch_ritz_tc(const RitzItem<float>* items, int n, int kmax, int kkmax, const int32_t* pre, int tiles,
                    int final_pass, cudaStream_t st);
// bounded MMA-barrier waits of k_ritz_tc that gave up since the last call
// (read and reset; synchronises the stream; -1 on a CUDA error)
int ritz_tc_timeouts(cudaStream_t st);
// device address of k_ritz_tc's counter (current device), null on a CUDA
// error; and launches skipped for want of plan scratch since the last call
// (read and reset, host side)
int* ritz_tc_timeout_word();
int ritz_tc_plan_failures();
template <typename T>
void launch_finalize(const FinalItem<T>* items, int n, int max_r, int64_t max_rows, cudaStream_t st);

}  // namespace ssa
