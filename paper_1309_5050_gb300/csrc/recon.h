// Reconstruction work items and launchers (internal).
#pragma once
#include <cuda_runtime.h>
#include "kernels.cuh"

namespace ssa {

// x-pass transform of columns of one compact vector (U_i or V_i slice).
template <typename T, typename TV>
struct RecColItem {
  const TV* vec;         // compact vector
  MapDev map;            // its grid positions
  Cx<T>* dst;            // (H+1) x ncols half spectra
  int32_t log2Mx, ncols; // grid columns to transform
};

// Series reconstruction of one (group, channel).
template <typename T, typename TV>
struct Rec1Item {
  const TV* V; int64_t ldv;     // channel slice of the factor vectors (column i at V + ldv*i)
  MapDev map;                  // the channel's origin set
  const Cx<T>* gu; int64_t ldgu;  // F(U'_i) at gu + ldgu*i
  const double* sigma;         // device
  const int32_t* comps; int32_t ncomp;
  int32_t log2Mx;
  const int32_t* w; int32_t n; // weights of the channel grid, n = N_c
  double* out;                 // n values
  double inv_norm;             // 1 / Mx
};

// Image reconstruction, final inverse x-pass of one group.
template <typename T>
struct Rec2Item {
  const Cx<T>* g2;             // y-inverse of the accumulated spectrum
  const int32_t* w;            // Nx x Ny weights (null: write the raw sums, no division)
  double* out;                 // Nx x Ny
  int32_t log2Mx, nx, ny, pad_;
  double inv_norm;             // 1 / (Mx My)
};

template <typename T, typename TV>
void launch_rec_col_fft(const RecColItem<T, TV>* items, int n, int max_log2Mx, int max_cols, const Cx<T>* tw,
                        cudaStream_t st);
template <typename T, typename TV>
void launch_rec1d(const Rec1Item<T, TV>* items, int n, int max_log2Mx, const Cx<T>* tw, cudaStream_t st);
template <typename T>
void launch_rec_xinv(const Rec2Item<T>* items, int n, int max_log2Mx, int max_ny, const Cx<T>* tw,
                     cudaStream_t st);
// Complete series reconstructed with FP32 FFTs: the elements whose weight is
// below REC_BORDER_W (the first and last REC_BORDER_W of the series) are
// recomputed by direct FP64 summation over their anti-diagonal -- the FFT's
// absolute error, divided by a small weight, would dominate there.
constexpr int REC_BORDER_W = 64;
struct RecBorderItem {
  const float* U;              // L x r, column c at U + L c
  const float* V;              // the channel's slice of V: K x r, column c at V + ldv c
  int64_t ldv;
  const double* sigma;
  const int32_t* comps; int32_t ncomp;
  int32_t L, K;                // window length and the channel's K (N = L + K - 1)
  int32_t pad_;
  double* out;                 // the channel's N outputs of this group
};
void launch_rec_border(const RecBorderItem* items, int n, cudaStream_t st);

// w-correlations (Sec. 2.2, paragraph Separability): the Gram matrix
// G = Y^T diag(w) Y of m = n + 1 vectors over the data elements -- the n
// reconstructed components (FP64, ld ldy, NaN outside N') and, last, the data
// x (FP32 or FP64) -- with w_k = |A_k| (zero outside N').  k_wgram: each block
// sums the pairs listed in `pairs` (i <= j) over its chunks of elements into
// partials[block][pair]; k_wcor_final adds the blocks' partials in block order
// (deterministic) and writes rho (n x n, row-major; 0 where a norm is 0) and
// the contributions G_ii / G_mm.
constexpr int WGRAM_NT = 512;
constexpr int WGRAM_PT = 16;                 // pairs per thread
constexpr int WGRAM_CH = 32;                 // elements per staged chunk
constexpr int WCOR_MAX = 120;                // components: (n+1)(n+2)/2 <= WGRAM_NT * WGRAM_PT
void launch_wgram(const double* Y, int64_t ldy, int n, const void* x, int x_f64, const int32_t* w, int64_t total,
                  const int2* pairs, int npair, double* partials, int nblk, cudaStream_t st);
void launch_wcor_final(const double* partials, int nblk, const int2* pairs, int npair, int n, double* G, double* rho,
                       double* contrib, cudaStream_t st);

// Column recurrent forecast (Sec. 3.3, eq. Forec:ContMSSAL).  k_lrr: the
// recurrence R (L - 1 values) from the group's window-side vectors U[:, idx]
// (T, ld L), R = sum_j pi_j U'_j / (1 - nu^2), and nu^2 into *nu2 (the caller
// refuses nu^2 >= 1).  k_forecast_rec: one block per series p continues the
// reconstruction rec[off[p] .. off[p] + len[p]) by M values, each the dot
// product of R with the last L - 1 values (block sum in a fixed order), into
// out[p * M ..]; work holds the running series (ld ldw >= L - 1 + M).
template <typename T>
void launch_lrr(const T* U, int64_t L, const int32_t* idx, int nidx, double* R, double* nu2, cudaStream_t st);
void launch_forecast_rec(const double* rec, const int64_t* off, const int64_t* len, int s, int64_t L,
                         const double* R, int M, double* work, int64_t ldw, double* out, cudaStream_t st);

// Vector column forecast in the coefficients of the group's window space
// (Sec. 3.3, eqs. PGcolumn and V_FORcolumn; the fast form with a shift
// matrix).  Every continued lagged vector is U_I c_t with c_t = D c_{t-1},
// D = (I + pi pi^T / (1 - nu^2)) Ubar^T Uup (Ubar, Uup: U_I without its last,
// first row; pi its last row); c_0 = U_I^T (the last L values of the series);
// forecast m = (1 / L) sum_{i < L} (U_I c_{L + m - i})_i (diagonal averaging of
// the continued columns).  k_vf_gram: G = Ubar^T Uup, one block per entry;
// k_vf_shift: D and nu^2 (one block); k_vf_coef: c_0 .. c_{M+L-1} per series
// (one block each, stored in cs, ld nidx, per series (M + L) rows);
// k_vf_out: the M values of every series.
template <typename T>
void launch_vector_forecast(const T* U, int64_t L, const int32_t* idx, int nidx, const void* x, int x_f64,
                            const int64_t* off, const int64_t* len, int s, int M, double* G, double* D, double* nu2,
                            double* cs, double* out, cudaStream_t st);

// Row forecasts of an MSSA system (Sec. 3.3, eqs. Forec:ContMSSAK, PGrow,
// V_FORrow) from the group's origin-side vectors V[:, idx] (T, ld K; series p
// owns rows koff[p] .. koff[p] + kc[p]).  S = [mu(V_j)] (the last row of each
// series' block, s x r); Vbar / V': V without the last / first row of each
// block.  Recurrent: W = (I_s - S S^T)^-1 S, and each step appends
// W (Vbar^T z) to every series, z the last K_p - 1 values of each series
// (reconstruction rec, then the forecasts; work: per series kc[p] - 1 + M
// values at work + wo[p]).  Vector: D = (I_r - S^T S)^-1 Vbar^T V', the
// coefficients of the continued rows c_i = D c_{i-1} from c_{L-1} = V^T (row
// L - 1 of the trajectory matrix), and forecast m of series p
// = (1 / K_p) sum_{j < K_p} (V c_{N_p + m - j})[koff_p + j].  The dense solves
// (SPD matrices, no pivoting) run in one block on scratch in global memory;
// a non-positive pivot sets *fail.
constexpr int RF_MAXR = 128;                  // components of a row forecast
constexpr int RF_MAXS = 64;                   // series of a row forecast
template <typename T>
void launch_row_forecast(int vector, const T* V, int64_t K, const int32_t* idx, int nidx, const int64_t* koff,
                         const int64_t* kc, const int64_t* off, const int64_t* len, int s, int64_t L, int M,
                         int64_t kstar, const double* rec, const void* x, int x_f64, double* A, double* Bm,
                         double* work, const int64_t* wo, double* cs, double* out, int* fail, cudaStream_t st);
struct RecFoldItem {            // long series: segment-image sums -> one group's output
  const double* S;              // 2B x (segments), column-major
  const int32_t* w;             // n weights
  double* out;                  // n values
  int64_t B, n;
  int64_t ncols;                // columns of S (segments of the grid)
};
void launch_rec_fold(const RecFoldItem* items, int n, int64_t max_n, cudaStream_t st);
struct ResItem {                // residual x - sum of groups for one channel
  const void* data; int32_t data_double, ngroups;
  const int32_t* w; const double* groups; int64_t gstride, n;
  double* out;
};
void launch_residual_batch(const ResItem* items, int n, int64_t max_n, cudaStream_t st);
void launch_residual(const void* data, int data_double, const int32_t* w, int64_t n, const double* groups,
                     int64_t gstride, int ngroups, double* out, cudaStream_t st);

}  // namespace ssa
