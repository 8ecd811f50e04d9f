// Work-item descriptors shared by the kernels and the host orchestration.
#pragma once
#include "common.cuh"

namespace ssa {

// Per-problem Lanczos state kept in device memory.
struct LzState {
  int32_t jc;         // next Lanczos step of the current cycle (from 0, or kk after a restart);
                      // the cycle is complete when jc reaches k
  int32_t k;          // Krylov dimension
  int32_t r;          // wanted rank
  int32_t kk;         // vectors kept on restart
  int32_t active;     // 1 while the problem still iterates
  int32_t converged;  // set by the small-SVD kernel
  int32_t nconv;      // leading triples that pass the residual test
  int32_t breakdown;  // breakdowns met: coefficients at rounding level set to 0 and their vectors
                      // replaced by random ones orthogonal to the basis (k_lanczos.cu)
  int32_t restarts;   // restart cycles done
  int32_t max_restarts;
  int32_t full;       // k equals min(L, K): one cycle spans the whole space
  int32_t sweeps;     // FP64 Jacobi sweeps of the last small SVD
  int32_t svd_done;   // the small SVD of the completed cycle has run (cleared by a restart)
  int32_t sweeps32;   // FP32 Jacobi sweeps that preceded them
  double beta_k;      // coupling to the (k+1)-th long vector after k steps
  double anorm;       // largest Lanczos coefficient seen (scale for breakdown)
  double tol;         // residual tolerance relative to sigma_1
  double sigma1;      // current leading Ritz value
  double maxres;      // largest relative residual among the r wanted
  double bd_floor;    // rounding level of one product with a unit vector (breakdown test)
};

// A compact vector, possibly column (jc + s + jdelta) of a basis.
struct VecRef {
  void* base;
  int64_t off;              // element offset (channel slice or partial row)
  int64_t ld;               // column stride in elements
  const LzState* st;        // non-null: column chosen from the Lanczos step
  int32_t jdelta;
  int32_t pad_;
};

__device__ __forceinline__ int64_t vec_elem_off(const VecRef& v, int s) {
  int64_t o = v.off;
  if (v.st) o += (int64_t)(v.st->jc + s + v.jdelta) * v.ld;
  return o;
}

// One matvec job: a channel of one problem in one direction.
template <typename T>
struct MvItem {
  const Cx<T>* xh;          // channel spectrum, (H+1) x My, pre-scaled by 1/(Mx My)
  VecRef in, out;           // compact input / output
  const double* in_scale;   // non-null: input column c is scaled by in_scale[c]
  MapDev min, mout;         // their grid positions
  Cx<T>* g1;                // 2D scratch: after x-pass, (H+1) x My
  Cx<T>* g2;                // 2D scratch: after y-pass
  const LzState* st;        // non-null: skip when inactive or past k
  int32_t log2Mx, log2My;
  int32_t in_type;          // 0: T, 1: double
  int32_t y_in_hi;          // grid columns [0, y_in_hi) may hold input
  int32_t y_out_hi;         // grid columns [0, y_out_hi) hold output positions
  int32_t pad_;
  // Long-side Lanczos step fused into the store of X^T u (series whose long
  // side is the origin side): instead of the product slice, row o of the
  // output writes q = (X^T u)_o - alpha_j v_j[o] into column j+1 of lV,
  // alpha_j v_j = lB[j, j] lcolscale[j] lV[:, j] (j = jc + s), and the
  // block's partial sum of q^2 goes to lnpart[lslot].  lV == null: off.
  T* lV; int64_t lld;
  const double* lB; const double* lcolscale; double* lnpart;
  int32_t lldb, lslot;
  // Non-null: the input's forward transform (H values before the untwist),
  // computed once per problem and grid size by k_uspec, replaces the forward
  // FFT of this product.
  const Cx<T>* zin;
};

// Forward transform of the window-side vector u_j (column jc + s of the FP64
// short basis) on a grid of 2^log2M, shared by every channel of that size.
template <typename T>
struct UzItem {
  const double* U; int64_t ldu;
  const LzState* st;
  int32_t L, log2M;
  Cx<T>* z;                 // H values
};

// Code path of a series product (one k_mv1d instantiation per value): the
// input is double (else T), the input map is bit-mapped (else a dense range),
// the output is the fused long-side step, or bit-mapped (else a dense range).
// MV1_IN_ZSPEC: the input arrives as its precomputed forward transform.
enum : int { MV1_IN_DOUBLE = 1, MV1_IN_MAPPED = 2, MV1_OUT_FUSED = 4, MV1_OUT_MAPPED = 8, MV1_IN_ZSPEC = 16,
             MV1_MODES = 25 };
template <typename T>
inline int mv1d_mode(const MvItem<T>& m) {
  const int out = !m.mout.dense ? MV1_OUT_MAPPED : (m.lV ? MV1_OUT_FUSED : 0);
  if (m.zin) return MV1_IN_ZSPEC | out;
  return (m.in_type == 1 ? MV1_IN_DOUBLE : 0) | (m.min.dense ? 0 : MV1_IN_MAPPED) | out;
}

// Raw data to half spectrum (step 1 of the matvec algorithms, precomputed).
template <typename T>
struct SpecItem {
  const void* data;         // column y of the grid starts at data + ld*y (float or double)
  int64_t ld;               // column stride: nx for an image, the segment step for a long series
  int64_t n_lin;            // elements data[0, n_lin) exist; later ones read as zero
  const uint32_t* obs;      // observed bits, Ny columns x words (null = all)
  int32_t obs_words;
  int32_t data_double;
  int32_t nx, ny;
  int32_t log2Mx, log2My;
  Cx<T>* g1;                // x-pass result (2D)
  Cx<T>* xh;                // output spectrum (H+1) x My
  T scale;                  // 1/(Mx My)
};

enum YMode : int { Y_FWD = 0, Y_MULCONJ_INV = 1, Y_CONVACC = 2, Y_INV = 3 };

// One y-pass job (2D grids): a complex FFT along y of every x-frequency.
//  Y_FWD         dst = F_y(src)                     (rows m < in_hi nonzero)
//  Y_MULCONJ_INV dst = F_y^-1(mul . conj F_y(src))  (rows m < out_hi written)
//  Y_CONVACC     dst += scale * mul . F_y(src)      (all rows)
//  Y_INV         dst = F_y^-1(src)                  (rows m < out_hi written)
template <typename T>
struct YItem {
  const Cx<T>* src;
  Cx<T>* dst;
  const Cx<T>* mul;
  const LzState* st;
  int32_t log2Mx, log2My;
  int32_t in_hi, out_hi;
  T scale;
  int32_t tk;               // x-frequencies per block (ypass_tk), set by the host
};

// Block ranges of a batched launch: item i owns blocks [pre[i], pre[i+1]);
// pre == nullptr means one item owning every block.
struct Tiles {
  const int32_t* pre;
  int32_t n, total;
};
__device__ __forceinline__ int tile_of(const Tiles& t, int b, int& local) {
  if (!t.pre) { local = b; return 0; }
  return tile_item(t.pre, t.n, b, local);
}

}  // namespace ssa
