/*
 * ssa.h -- C ABI of the GB300 SSA library (libssa.so).
 *
 * Singular Spectrum Analysis of a series (SSA), a system of series (MSSA), an
 * image (2D-SSA) and a shaped / masked image (Shaped 2D-SSA), following
 * Golyandina, Korobeynikov, Shlemov and Usevich, "Multivariate and 2D
 * Extensions of Singular Spectrum Analysis with the Rssa Package":
 *   embedding (Sec. 2.1 Step 1; eqs. ssa_embedding, mssa_embedding,
 *   block_hankel_cols, qh_mat), truncated SVD of the trajectory matrix
 *   (Step 2, eq. mmexp), grouping (Step 3, eq. mmexp_g) and reconstruction by
 *   averaging over the sets A_k (Step 4, eq. res_decomp).
 * The trajectory matrix is never formed: its products with vectors and the
 * rank-one diagonal averaging go through FFTs (Sec. 6.1-6.2).
 *
 * Conventions for every entry point
 *  - Return value: SSA_OK (0) or a negative SSA_E* code; ssa_strerror() names
 *    it and ssa_last_error() gives a one-line detail for the calling thread.
 *  - Arrays are column-major.  Images are Nx x Ny with x (rows) running down
 *    and y (columns) right, the paper's orientation (Sec. 4.1.1).  Vectors
 *    over the window set L and the origin set K follow the lexicographic
 *    (column-major) order of Sec. 5.1.  Group and component indices are
 *    0-based (the paper's are 1-based).
 *  - Pointers marked "host or device" follow the call's on_device flag; all
 *    others are host pointers.  The library copies its inputs and never keeps
 *    a caller pointer; outputs go to caller-allocated buffers.
 *  - A context owns every byte of device memory it allocates and frees it in
 *    ssa_destroy().  All work of a context is ordered on its CUDA stream; one
 *    context must not be used from two threads at once.
 *  - Errors leave the context usable unless SSA_ECUDA is returned (then the
 *    CUDA context may be unusable and the caller should destroy it).
 */
#ifndef SSA_GB300_H
#define SSA_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  SSA_OK = 0,
  SSA_EINVAL = -1,       /* bad argument (sizes, window, Inf in the data, ...) */
  SSA_EEMPTY = -2,       /* no admissible window origin: K is empty */
  SSA_ERANK = -3,        /* rank r outside [1, min(L, K)] */
  SSA_ENOMEM = -4,       /* device allocation failed */
  SSA_ENOTCONV = -5,     /* restarts exhausted; results valid, residuals in ssa_info */
  SSA_ETIMEOUT = -6,     /* a bounded wait expired */
  SSA_ECUDA = -7,        /* CUDA runtime error */
  SSA_ESTATE = -8,       /* call out of order (e.g. reconstruct before decompose) */
  SSA_EUNSUPPORTED = -9  /* size outside what this build supports */
};

typedef enum { SSA_1D = 0, SSA_MSSA = 1, SSA_2D = 2 } ssa_kind;  /* SSA_2D covers shaped */
typedef enum { SSA_F32 = 0, SSA_F64 = 1 } ssa_dtype;
/* Precision forms: FFTs, matvecs and the long-side Lanczos basis in FP32; the
 * short basis stored in FP64 and re-orthogonalised in FP32 plus float-float
 * (about 48 significant bits); the small SVD's rotations found in FP32 and
 * polished in float-float; reconstruction sums in FP32 (complete series, the
 * low-weight ends summed directly) or FP64 -- the name keeps the form's
 * first definition, FP64 re-orthogonalisation; or all FP64. */
typedef enum { SSA_PREC_FP32FFT_FP64REORTH = 0, SSA_PREC_FP64 = 1 } ssa_prec;

typedef struct ssa_ctx ssa_ctx;

typedef struct {
  int32_t kind;            /* ssa_kind */
  int32_t dtype;           /* ssa_dtype of data */
  int32_t on_device;       /* data and mask are device (1) or host (0) pointers */
  int32_t n_series;        /* MSSA: number of series s (>= 1); ignored otherwise */
  const void* data;        /* host or device.  1D: n values.  MSSA: the s series
                              concatenated.  2D: nx*ny values, column-major.
                              NaN marks a missing value (Sec. 5.2) */
  int64_t n;               /* 1D: series length N */
  const int64_t* lengths;  /* MSSA: s lengths N_p (host) */
  int64_t nx, ny;          /* 2D: image size */
  const uint8_t* mask;     /* optional, host or device, same layout as data:
                              nonzero = observed; NULL = all observed */
} ssa_input;

typedef struct {
  int64_t L;               /* 1D / MSSA window length, 1 < L < N (MSSA: < min N_p) */
  int64_t lx, ly;          /* 2D window bounding box, 1 <= lx <= nx, 1 <= ly <= ny */
  const uint8_t* wmask;    /* optional 2D window shape, lx*ly column-major (host);
                              NULL = the full rectangle */
} ssa_window;

typedef struct {
  int32_t rank;            /* r >= 1: eigentriples wanted */
  int32_t krylov_dim;      /* k; 0 = min(2r + 16, 112, min(L, K)) */
  int32_t max_restarts;    /* 0 = 40 */
  int32_t prec;            /* ssa_prec */
  double tol;              /* residual tolerance relative to sigma_1;
                              0 = 1e-7 (FP32 form) / 1e-13 (FP64 form) */
  uint64_t seed;           /* start vector seed */
} ssa_params;

typedef struct {
  int64_t L, K;            /* trajectory matrix size */
  int64_t nx, ny;          /* grid of the (first) channel */
  int32_t n_channels;      /* s for MSSA, else 1 */
  int32_t rank;            /* r of the last decomposition (0 before) */
  int32_t krylov_dim;      /* k used */
  int32_t restarts;        /* restart cycles run */
  int32_t converged;       /* 1 if every wanted triple met the tolerance */
  int32_t prec;            /* precision form of the last decomposition */
  int64_t fft_mx, fft_my;  /* FFT grid */
  double max_residual;     /* max_i ||X^T u_i - sigma_i v_i|| / sigma_1 (Lanczos estimate) */
  int64_t device_bytes;    /* device memory held by the context */
  int32_t jacobi_sweeps;   /* FP64 sweeps of the last small SVD (one-sided Jacobi) */
  int32_t jacobi_sweeps_fp32;  /* FP32 sweeps that found its rotations first */
  int32_t breakdowns;      /* Lanczos coefficients found at the rounding level of the largest
                              one (an invariant subspace: exact rank below k, or a multiple
                              singular value): set to 0, the process went on from a random
                              vector orthogonal to the basis.  Results are not affected. */
  int32_t pad_;
} ssa_info;

/*
 * ssa_embed -- Step 1 (Sec. 2.1) and the shape calculus (Sec. 5.1, 6.2.4).
 * Validates the input, copies it to the device and computes, exactly in
 * integers, the origin set K = {kappa : L (+) {kappa} inside N} (eq. sh_Ks),
 * the reconstructable set N' = L (+) K and the weights w_k = |A_k|.  The data
 * spectrum (Sec. 6.1.2: "F(x) can be precomputed") is built on first use.
 * cuda_stream: a cudaStream_t to order the context's work on, or NULL for a
 * stream owned by the context.  On success *out receives a new context.
 * Series (1D and every series of an MSSA system) longer than 16384 samples
 * run in segment form: with B = 4096 the L x K Hankel matrix equals the
 * Hankel-block-Hankel matrix of the image S[i, c] = x[cB + i] (i < 2B - 1)
 * with window B x ceil(L/B) and origins B x ceil(K/B), rows and columns past
 * L and K absent (Sec. 6.2 applied to a 1D series), so the products and the
 * reconstruction use a 2B x My grid; such series must have no missing values.
 * Errors: SSA_EINVAL (sizes, window, +-Inf), SSA_EEMPTY (K empty),
 * SSA_EUNSUPPORTED (image grid above 16384 along x or 4096 along y; a
 * segment-form series with missing values or more than 4096 segments).
 */
int ssa_embed(const ssa_input* in, const ssa_window* win, void* cuda_stream, ssa_ctx** out);

/*
 * ssa_embed_batch -- ssa_embed for n inputs (ins[i] with window wins[i]) in
 * one pass: the shape kernels of all inputs are launched back to back and the
 * host waits twice for the whole batch.  outs (host array of n) receives the
 * contexts (NULL where an input failed); status (may be NULL) each code.
 * Returns the first non-OK code.  All contexts share cuda_stream (NULL: each
 * gets its own).
 */
int ssa_embed_batch(const ssa_input* ins, const ssa_window* wins, int32_t n, void* cuda_stream, ssa_ctx** outs,
                    int32_t* status);

/*
 * ssa_decompose -- Step 2 (Sec. 2.1, eq. mmexp): the r leading eigentriples
 * (sigma_i, U_i, V_i) of the trajectory matrix, by Golub-Kahan-Lanczos
 * bidiagonalisation on FFT products (Sec. 6.1.2 Alg. hmul_u; Sec. 6.2.2) with
 * thick restarts; the truncated-SVD role Rssa gives PROPACK / nu-TRLan
 * (Sec. 2.4).  Signs: each pair (U_i, V_i) is flipped so that the entry of
 * U_i with the largest magnitude is positive.
 * Errors: SSA_ERANK, SSA_ENOTCONV (results kept), SSA_ENOMEM, SSA_ECUDA.
 */
int ssa_decompose(ssa_ctx* ctx, const ssa_params* params);

/*
 * ssa_continue -- continue a decomposition to a larger rank (the
 * auto-continuation Rssa offers, Sec. 2.4): the previous run's r1 Ritz
 * triples, their couplings beta_k P[k-1, i] and the residual direction seed
 * the new Krylov space as after a thick restart that keeps them, so only the
 * new part of the space is built.  params: the new rank (above the previous
 * one and at most min(L, K)), the same precision form; krylov_dim, tol and
 * max_restarts as for ssa_decompose (seed unused).  A previous run that
 * spanned the whole space, broke down, did not converge or used the other
 * form is redone from a new start vector.  The results replace the previous
 * ones.
 * Errors: SSA_ESTATE (no decomposition), SSA_ERANK, SSA_ENOTCONV, SSA_ENOMEM,
 * SSA_ECUDA.
 */
int ssa_continue(ssa_ctx* ctx, const ssa_params* params);

/*
 * ssa_decompose_batch -- the same for n contexts at once: every kernel of the
 * Lanczos step is launched once for the whole batch (all problems advance in
 * lock-step).  params: n entries (one per context).  All contexts must live
 * on the current device; work is ordered on ctxs[0]'s stream.  status
 * (host, n entries, may be NULL) receives each context's code; the return
 * value is the first non-OK code.
 */
int ssa_decompose_batch(ssa_ctx* const* ctxs, int32_t n, const ssa_params* params, int32_t* status);

/* ssa_get_info -- sizes and solver statistics (host struct). */
int ssa_get_info(const ssa_ctx* ctx, ssa_info* info);

/* ssa_get_sigma -- the r singular values sqrt(lambda_i), descending, into
 * sigma (host, r doubles); r must not exceed the decomposed rank. */
int ssa_get_sigma(const ssa_ctx* ctx, double* sigma, int32_t r);

/*
 * ssa_get_vectors -- eigenvectors U (L x r) and factor vectors V (K x r),
 * column-major FP64, into host or device buffers (on_device).  Either pointer
 * may be NULL.  MSSA factor vectors stack the series' factor subvectors
 * (Sec. 3.2); image vectors list the window / origin sets lexicographically.
 */
int ssa_get_vectors(const ssa_ctx* ctx, double* U, double* V, int32_t on_device);

/*
 * ssa_reconstruct -- Steps 3-4 (Sec. 2.1; eq. res_decomp): for each group g the
 * component x~_g = T^-1 Pi^(H) sum_{i in g} sigma_i U_i V_i^T, computed by
 * rank-one FFT hankelization summed in frequency space (Sec. 6.1.3 Alg.
 * hankelization, Sec. 6.2.3 Alg. qhankelization / diagsums).
 * group_of: r entries (host), component i goes to group group_of[i] in
 * [0, n_groups), or -1 to leave it out.  residual: if nonzero one more output
 * x - sum_g x~_g is appended.  out (host or device): (n_groups + residual)
 * blocks of FP64 values in the input's layout (1D: N; MSSA: sum N_p, series
 * concatenated; 2D: nx*ny); NaN outside N' (values that never enter the
 * trajectory matrix, Sec. 5.1).
 */
int ssa_reconstruct(ssa_ctx* ctx, const int32_t* group_of, int32_t n_groups, int32_t residual, double* out,
                    int32_t on_device);

/*
 * ssa_reconstruct_batch -- ssa_reconstruct for n decomposed contexts; every
 * context uses the same grouping (group_of has the first context's r entries,
 * the others must have the same r).  out_ptrs: n pointers (host array) to
 * buffers as for ssa_reconstruct.
 */
int ssa_reconstruct_batch(ssa_ctx* const* ctxs, int32_t n, const int32_t* group_of, int32_t n_groups,
                          int32_t residual, double* const* out_ptrs, int32_t on_device);

/*
 * ssa_wcor -- w-correlations and contributions of reconstructed components
 * (Sec. 2.2, paragraph Separability).  With the weighted inner product
 * (Y, Z)_w = sum_k w_k y_k z_k (w_k = |A_k|, over every channel's elements):
 * wcor[i * n + j] = (X~_i, X~_j)_w / (||X~_i||_w ||X~_j||_w) for the
 * components X~_i of the n = n_groups groups of group_of (as for
 * ssa_reconstruct; group_of[i] = i gives the paper's w-correlation matrix of
 * the elementary components), means not subtracted, 0 where a norm is 0;
 * contrib[i] = ||X~_i||_w^2 / ||X||_w^2 (may be NULL).  wcor, contrib: host
 * buffers of n*n and n FP64 values.  The components are reconstructed on the
 * device and the weighted Gram matrix is summed there in FP64, in a fixed
 * order (repeatable results).
 * Errors: SSA_EINVAL (n_groups outside [1, 120], null pointers), SSA_ESTATE
 * (no decomposition), SSA_ENOMEM, SSA_ECUDA.
 */
int ssa_wcor(ssa_ctx* ctx, const int32_t* group_of, int32_t n_groups, double* wcor, double* contrib);

/*
 * ssa_forecast -- M-step recurrent column forecast of a series or of every
 * series of an MSSA system (Sec. 3.3, eq. Forec:ContMSSAL).  The component of
 * the n_idx components idx (0-based, below the decomposed rank) is
 * reconstructed on the device; the recurrence R = sum_j pi(U_j) U'_j /
 * (1 - nu^2), nu^2 = sum_j pi(U_j)^2 (pi: last coordinate, U': the others, of
 * the window-side vectors) is applied M times to the last L - 1 values of
 * each series' reconstruction -- one recurrence for all series, FP64 sums.
 * out (host): M values per series, series after series (s x M).
 * Errors: SSA_EINVAL (images, M < 1, an index out of range, nu^2 >= 1),
 * SSA_ESTATE (no decomposition), SSA_ENOMEM, SSA_ECUDA.  A series whose last
 * L - 1 values are missing gets NaN forecasts.
 */
int ssa_forecast(ssa_ctx* ctx, const int32_t* idx, int32_t n_idx, int32_t M, double* out);

/*
 * ssa_forecast_vector -- M-step vector column forecast of a series or of every
 * series of an MSSA system (Sec. 3.3, eqs. PGcolumn and V_FORcolumn).  The
 * last lagged vector of each series is projected on the window space of the
 * n_idx components idx, continued M + L - 1 times by the operator that drops
 * its first coordinate, projects the rest on the span of the U_j without
 * their last coordinate and appends the recurrence value, and the continued
 * lagged vectors are diagonally averaged.  On the device this runs in the
 * coefficients of the window space (c_t = D c_{t-1} with an n_idx x n_idx
 * shift matrix D), FP64 sums in a fixed order.  out (host): M values per
 * series, series after series.  M <= 65535.  Errors as for ssa_forecast.
 */
int ssa_forecast_vector(ssa_ctx* ctx, const int32_t* idx, int32_t n_idx, int32_t M, double* out);

/*
 * ssa_forecast_row -- M-step row forecast of a series or of every series of
 * an MSSA system (Sec. 3.3): recurrent (vector = 0, eq. Forec:ContMSSAK: each
 * step appends R_K z to every series, R_K = (I_s - S S^T)^-1 S Vbar^T, z the
 * last K_p - 1 reconstructed values of all series, S the last coordinates of
 * each series' block of the group's origin-side vectors) or vector
 * (vector = 1, eqs. PGrow and V_FORrow: the rows of the reconstructed matrix
 * continued by the row projector, in the coefficients of the group's row
 * space, then the MSSA diagonal averaging).  idx / n_idx / M / out as for
 * ssa_forecast.  At most 64 series and 128 components.
 * Errors as for ssa_forecast; SSA_EINVAL also when I - S S^T is singular.
 */
int ssa_forecast_row(ssa_ctx* ctx, const int32_t* idx, int32_t n_idx, int32_t M, int32_t vector, double* out);

/*
 * ssa_get_shape -- the shape calculus results (host buffers, any may be NULL):
 * L, K; origin_mask (uint8, input layout: 1 where an element is a window origin
 * kappa of K); weights (int32, input layout: w_k = |A_k|, 0 outside N').
 */
int ssa_get_shape(const ssa_ctx* ctx, int64_t* L, int64_t* K, uint8_t* origin_mask, int32_t* weights);

/*
 * ssa_matvec -- one product with the trajectory matrix by FFT: transpose = 0
 * gives u = X v (in: K values, out: L values), transpose = 1 gives
 * v = X^T u (in: L, out: K).  Sec. 6.1.2 Alg. hmul_u and Sec. 6.2.2.
 * prec selects the arithmetic (ssa_prec).  in/out: FP64, host or device.
 */
int ssa_matvec(ssa_ctx* ctx, int32_t transpose, int32_t prec, const double* in, double* out, int32_t on_device);

/*
 * Tuned plans (process-wide; no paper counterpart -- implementation tuning).
 * Two choices are otherwise derived from the sizes: the Krylov dimension k of
 * a decomposition (default min(2r + 16, 112, min(L, K))) and the y-pass tile
 * of 2D grids (x-frequencies transformed along y by one block; default from a
 * fixed shared-memory budget).  ssa_autotune times one decomposition of ctx
 * for each candidate -- k in {2/3, 1, 3/2, 2} x the default (clipped to
 * [r, min(112, L, K)]), then for 2D grids the tile in {1/2, 2, 4} x the
 * default that fit a block -- keeps the fastest converged one (a candidate
 * replaces the default, or the tile chosen so far, only when it is more than
 * 2% faster: smaller differences are within run-to-run noise) and records it
 * as the plan of its size class: k keyed by (precision form, kind, L,
 * ceil log2 K, r), the tile by (element size, grid).  Every later
 * decomposition with krylov_dim = 0 and every product on such a grid uses
 * the plans.  ctx ends decomposed with the chosen plan.  out (may be NULL):
 * the choice, candidates timed, and the default and best times (ms,
 * CUDA events on the context's stream).
 * ssa_plans_export writes the plans as text lines "kdim <key> <k>" /
 * "ytk <key> <tile>" into buf (cap bytes, NUL-terminated; *len = bytes
 * needed) so a caller can keep them in a file; ssa_plans_import reads such
 * text back.
 * Errors: SSA_EINVAL, SSA_ERANK; those of ssa_decompose.
 */
typedef struct {
  int32_t krylov_dim;      /* chosen k */
  int32_t ytk;             /* chosen y-pass tile (0: not a 2D grid) */
  int32_t n_tried;         /* candidates timed */
  int32_t pad_;
  double ms_default;       /* one decomposition with the default plan */
  double ms_best;          /* one decomposition with the chosen plan */
} ssa_tune_result;

int ssa_autotune(ssa_ctx* ctx, const ssa_params* params, ssa_tune_result* out);
int ssa_plans_export(char* buf, int64_t cap, int64_t* len);
int ssa_plans_import(const char* text);

/*
 * Profiling (process-wide; no paper counterpart -- measurement support).
 * Phases: 0 shapes and weights, 1 data spectrum, 2 trajectory products
 * (X v and X^T u), 3 short-side Lanczos (re-orthogonalisation), 4 long-side
 * Lanczos, 5 small SVD / Ritz vectors / restart, 6 reconstruction.
 * ssa_profile_enable(1) records CUDA events on the launching stream around
 * each phase; ssa_profile_read() waits for them and returns the summed device
 * milliseconds, the kernels launched and the phase instances since the last
 * reset.  Launch counts are kept even when timing is off.
 * ssa_kernel_launches() returns every kernel this library has launched.
 */
int ssa_profile_enable(int32_t on);
int ssa_profile_reset(void);
int ssa_profile_read(int32_t phase, double* ms, int64_t* launches, int64_t* calls);
int64_t ssa_kernel_launches(void);

/*
 * ssa_matvec_series_noalloc -- one Hankel trajectory-matrix product of a
 * single FP32 series, for callers that cannot allocate device memory at call
 * time (inside a captured CUDA graph region, hosts with a fixed memory budget,
 * plug-in hosts that keep the allocator to themselves).  The paper has no
 * counterpart: this is a deployment variant of the FFT product of ssa_matvec.
 *   x    device, n floats (the series, no missing values)
 *   L    window length, 1 < L < n; K = n - L + 1
 *   transpose 0: out = X in  (in: K floats, out: L floats, device)
 *   transpose 1: out = X^T in (in: L floats, out: K floats, device)
 *   cuda_stream  cudaStream_t the work is ordered on (NULL = default stream)
 * The only intermediate data (twiddle table and the series' half spectrum)
 * live in one fixed device array of about 320 KB that every GPU loading the
 * library holds until the process exits; n is limited to 16384 samples
 * (larger returns SSA_EUNSUPPORTED).  The first call on a device looks the
 * array up and fills its twiddle table (and waits for that): make it before
 * any stream capture.  Calls share the array, so calls whose work overlaps on
 * the GPU race; order them on one stream.  Nothing is allocated or freed.
 * Errors: SSA_EINVAL, SSA_EUNSUPPORTED, SSA_ECUDA; ssa_noalloc_last_error()
 * gives the detail (static buffer of the calling thread).
 */
int ssa_matvec_series_noalloc(const float* x, int64_t n, int64_t L, int32_t transpose, const float* in,
                              float* out, void* cuda_stream);
const char* ssa_noalloc_last_error(void);

/*
 * Serving: many independent decompositions in flight on one GPU.
 * The arithmetic of each request is that of ssa_embed + ssa_decompose +
 * ssa_reconstruct (Sec. 2.1, steps 1-4 of the basic algorithm, with the
 * products of Sec. 6.1 and the truncated SVD of Sec. 6.2); how requests
 * share the GPU has no paper counterpart.
 *
 * A server owns one stream.  ssa_server_submit copies a request (host data
 * only) into a FIFO queue and returns a ticket.  Each ssa_server_step
 *   1. admits queued requests in arrival order while the sum of the device
 *      bytes estimated for the live requests stays within memory_budget and
 *      fewer than max_live are live (a request larger than the whole budget
 *      finishes at once with SSA_ENOMEM);
 *   2. embeds the admitted ones together, builds their spectra and Lanczos
 *      workspaces and adds them to the live set;
 *   3. runs ONE thick-restart Lanczos cycle for every live request in shared
 *      launches (each request at its own cycle: continuous batching at
 *      restart granularity), then
 *   4. retires the converged ones -- final Ritz vectors, the requested
 *      grouped reconstruction, sigma and outputs copied to host memory owned
 *      by the server, device memory freed -- and restarts the others.
 * Series requests (1D, MSSA) and images (2D / shaped) iterate in two
 * separate sets on the same stream.  A request's result does not depend on
 * what else is in flight: every product, reduction and small SVD of a
 * request reads only that request's data, and its start vector comes from
 * its own seed.
 */
typedef struct ssa_server ssa_server;

typedef struct {
  int64_t memory_budget;   /* device bytes for live requests; <= 0: 40 GiB */
  int32_t max_live;        /* live requests at most; <= 0: 512 */
  int32_t prec;            /* SSA_PREC_*: precision of every request of this server */
} ssa_server_config;

typedef struct {
  int64_t ticket;
  int32_t status;          /* SSA_OK, or the error that ended the request */
  int32_t rank;
  int64_t out_len;         /* doubles in the reconstruction output: (n_groups + residual) x total */
  int32_t restarts;        /* restart cycles the request took */
  int32_t pad_;
  double max_residual;     /* largest relative residual among the wanted triples */
  double t_submit, t_admit, t_done;   /* seconds on the server's clock */
  int64_t device_bytes;    /* device bytes the request held */
  int64_t estimated_bytes; /* the estimate admission charged against the budget */
} ssa_server_result;

/* ssa_server_create -- cuda_stream: cudaStream_t to run on (NULL: the server
 * creates its own).  Errors: SSA_EINVAL (precision), SSA_ECUDA. */
int ssa_server_create(const ssa_server_config* cfg, void* cuda_stream, ssa_server** out);

/* ssa_server_submit -- queue one request.  in/win/p as for ssa_embed and
 * ssa_decompose (host data only; the server copies it, so the caller's
 * buffers may be reused at once; p->prec is replaced by the server's);
 * group_of / n_groups / residual as for ssa_reconstruct (n_groups = 0 and
 * residual = 0: no reconstruction).  *ticket names the request.
 * Errors: SSA_EINVAL (null or empty input, MSSA without lengths). */
int ssa_server_submit(ssa_server* s, const ssa_input* in, const ssa_window* win, const ssa_params* p,
                      const int32_t* group_of, int32_t n_groups, int32_t residual, int64_t* ticket);

/* ssa_server_step -- one admission + one restart cycle + retirement (above);
 * waits for the GPU.  *n_done (may be NULL): requests finished in this step.
 * A request-level failure ends only that request (its status says why); a
 * return other than SSA_OK is a failure of the server's stream itself. */
int ssa_server_step(ssa_server* s, int32_t* n_done);

/* ssa_server_stats -- queued, live and finished-but-not-taken requests, and
 * the device bytes charged to live requests.  Any pointer may be NULL. */
int ssa_server_stats(const ssa_server* s, int64_t* queued, int64_t* live, int64_t* finished, int64_t* bytes_live);

/* ssa_server_finished -- up to cap tickets of finished requests not taken
 * yet, in ticket order, into tickets[]; *n = how many were written. */
int ssa_server_finished(const ssa_server* s, int64_t* tickets, int32_t cap, int32_t* n);

/* ssa_server_take -- copy a finished request's result out and forget it.
 *   res    (may be NULL) summary above
 *   sigma  (may be NULL) host, rank doubles
 *   out    (may be NULL) host, out_len doubles, row-major (n_groups + residual) x total
 *          as ssa_reconstruct writes it (NaN outside the observed set)
 * Errors: SSA_ESTATE (unknown ticket or not finished yet). */
int ssa_server_take(ssa_server* s, int64_t ticket, ssa_server_result* res, double* sigma, double* out);

/* ssa_server_clock -- seconds since the server was created (its time base). */
double ssa_server_clock(const ssa_server* s);

/* ssa_server_destroy -- wait for the stream, free every request (queued,
 * live or finished) and the server (NULL is a no-op). */
void ssa_server_destroy(ssa_server* s);

/* ssa_synchronize -- wait for the context's stream. */
int ssa_synchronize(ssa_ctx* ctx);

/* ssa_destroy -- free the context and its device memory (NULL is a no-op). */
void ssa_destroy(ssa_ctx* ctx);

/* ssa_strerror -- static name of a return code. */
const char* ssa_strerror(int code);

/* ssa_last_error -- detail of the calling thread's last failure (static buffer). */
const char* ssa_last_error(void);

/* ssa_version -- library version string. */
const char* ssa_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SSA_GB300_H */
