// C ABI and host orchestration of the SSA library: contexts, shapes, spectra,
// the batched Lanczos driver, reconstruction.  Every arithmetic step runs in
// the kernels of k_*.cu; this file sizes buffers, builds work items and
// sequences launches on the context stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <climits>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <chrono>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/ssa.h"
#include "kernels.cuh"
#include "lanczos.h"
#include "launch.h"
#include "recon.h"
#include "shape.h"

using namespace ssa;

// ============================================================== errors
static thread_local char g_err[512] = "";

static int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

#define CU(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(e_ == cudaErrorMemoryAllocation ? SSA_ENOMEM : SSA_ECUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                     \
  } while (0)

#define TRY(expr)            \
  do {                       \
    int rc_ = (expr);        \
    if (rc_ != SSA_OK) return rc_; \
  } while (0)

// ============================================================== per-device setup
namespace ssa {

static std::mutex g_mu;

// ---------------------------------------------------------------- profiling
static std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches += n; }

struct Profiler {
  std::mutex mu;
  bool on = false;
  double ms[PH_COUNT] = {0};
  long long launches[PH_COUNT] = {0}, calls[PH_COUNT] = {0};
  struct Pend { int ph; cudaEvent_t a, b; };
  std::vector<Pend> pend;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
    cudaEvent_t e; cudaEventCreate(&e); return e;
  }
  void resolve() {   // caller holds mu
    for (auto& p : pend) {
      float t = 0.f;
      cudaEventSynchronize(p.b);
      if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) ms[p.ph] += t;
      pool.push_back(p.a); pool.push_back(p.b);
    }
    pend.clear();
  }
};
static Profiler g_prof;

PhaseScope::PhaseScope(int ph_, cudaStream_t st_) : ph(ph_), st(st_), a(nullptr), l0(g_launches.load()) {
  if (!g_prof.on) return;
  std::lock_guard<std::mutex> lk(g_prof.mu);
  cudaEvent_t e = g_prof.get();
  cudaEventRecord(e, st);
  a = (void*)e;
}
PhaseScope::~PhaseScope() {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  g_prof.launches[ph] += g_launches.load() - l0;
  g_prof.calls[ph] += 1;
  if (!a) return;
  cudaEvent_t b = g_prof.get();
  cudaEventRecord(b, st);
  g_prof.pend.push_back({ph, (cudaEvent_t)a, b});
  if (g_prof.pend.size() > 4096) g_prof.resolve();
}

void set_max_smem(const void* fn) {
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (done.count({fn, dev})) return;
  cudaFuncAttributes fa;
  int avail = device_max_smem();
  if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess) avail -= (int)fa.sharedSizeBytes;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, avail) != cudaSuccess)
    cudaGetLastError();  // leave no sticky error: the launch itself reports a too-large request
  done.insert({fn, dev});
}

int device_max_smem() {
  static std::map<int, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cache[dev] = v;
  return v;
}

__global__ void k_twiddles(Cx<float>* t32, Cx<double>* t64) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < TW_N; j += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(-2.0 * (double)j / (double)TW_N, &s, &c);
    t64[j] = cx(c, s);
    t32[j] = cx((float)c, (float)s);
  }
}

struct DevTables { Cx<float>* t32 = nullptr; Cx<double>* t64 = nullptr; };
static std::map<int, DevTables> g_tables;

static int ensure_tables(int dev) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_tables.count(dev)) return SSA_OK;
  DevTables t;
  // keep memory that contexts free cached in this process's stream-ordered
  // pool (the default releases it at every synchronisation, and mapping it
  // again costs milliseconds per context)
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  CU(cudaMalloc(&t.t32, sizeof(Cx<float>) * TW_N));
  CU(cudaMalloc(&t.t64, sizeof(Cx<double>) * TW_N));
  k_twiddles<<<64, 256>>>(t.t32, t.t64); count_launch();
  CU(cudaGetLastError());
  CU(cudaDeviceSynchronize());
  g_tables[dev] = t;
  return SSA_OK;
}

template <> const Cx<float>* twiddles<float>(int dev) { return g_tables[dev].t32; }
template <> const Cx<double>* twiddles<double>(int dev) { return g_tables[dev].t64; }

// ---------------------------------------------------------------- tuned plans
// A plan fixes two choices the library otherwise derives from the sizes: the
// Krylov dimension of a decomposition (keyed by precision form, kind, L,
// ceil log2 K and rank) and the y-pass tile -- the x-frequencies a block
// transforms along y -- of 2D grids (keyed by element size and grid).
// ssa_autotune times candidates on a real problem and records the fastest;
// later decompositions and products of the same class use them.
struct PlanTable {
  std::mutex mu;
  std::map<std::string, int> kdim;
  std::map<std::string, int> ytk;
};
static PlanTable g_plans;

static std::string kdim_key(int prec, int kind, int64_t L, int64_t K, int r) {
  int lk = 0;
  while ((int64_t(1) << lk) < K) ++lk;
  char b[96];
  snprintf(b, sizeof(b), "p%d.k%d.L%lld.K%d.r%d", prec, kind, (long long)L, lk, r);
  return b;
}
static std::string ytk_key(int esz, int log2Mx, int log2My) {
  char b[48];
  snprintf(b, sizeof(b), "e%d.x%d.y%d", esz, log2Mx, log2My);
  return b;
}
static int plan_kdim(int prec, int kind, int64_t L, int64_t K, int r) {
  std::lock_guard<std::mutex> lk(g_plans.mu);
  auto it = g_plans.kdim.find(kdim_key(prec, kind, L, K, r));
  return it == g_plans.kdim.end() ? 0 : it->second;
}
// y-pass tile of a grid: the tuned one, else the default from the buffer
// budget.  Keyed by the size of the complex element (8 for the FP32 form's
// transforms, 16 for FP64), as ssa_autotune records it.
template <typename T>
static int tuned_ytk(int log2Mx, int log2My) {
  std::lock_guard<std::mutex> lk(g_plans.mu);
  auto it = g_plans.ytk.find(ytk_key((int)sizeof(Cx<T>), log2Mx, log2My));
  return it == g_plans.ytk.end() ? ypass_tk<T>(log2My) : it->second;
}

// small helper kernels of the driver
// bd_scale = 4 eps_T log2(grid points): with ||x|| it is a few times the rounding
// error of one product with a unit vector (FFT error ~ eps log2 M ||x|| ||v||); a
// Lanczos coefficient below it is noise (the breakdown test of k_lanczos.cu).
__global__ void k_state_init(LzState* st, int k, int r, int kk, double tol, int max_restarts, int full,
                             const double* xnorm, double bd_scale) {
  st->bd_floor = bd_scale * *xnorm;
  st->full = full; st->sweeps = 0; st->sweeps32 = 0;
  st->jc = 0; st->svd_done = 0; st->k = k; st->r = r; st->kk = kk; st->active = 1; st->converged = 0;
  st->nconv = 0; st->breakdown = 0; st->restarts = 0; st->max_restarts = max_restarts;
  st->beta_k = 0.0; st->anorm = 0.0; st->tol = tol; st->sigma1 = 0.0; st->maxres = 0.0;
}

// A batch's workspace initialisation in one launch (one block per problem):
// B and the channel partial-product buffers zeroed, the state as
// k_state_init -- instead of three memsets and a launch per problem.
struct WsInit {
  LzState* st; double* B; int64_t bn;
  void* parts_s; int64_t bytes_s; void* parts_l; int64_t bytes_l;
  int32_t k, r, kk, maxr, full, pad_;
  double tol; const double* xnorm; double bd_scale;
};

__device__ __forceinline__ void zero_bytes(void* p, int64_t bytes) {
  // p is 256-byte aligned (arena), bytes a multiple of 4
  uint4* q = reinterpret_cast<uint4*>(p);
  const int64_t n16 = bytes >> 4;
  for (int64_t e = threadIdx.x; e < n16; e += blockDim.x) q[e] = make_uint4(0u, 0u, 0u, 0u);
  uint32_t* t = reinterpret_cast<uint32_t*>(p);
  for (int64_t e = (n16 << 2) + threadIdx.x; e < (bytes >> 2); e += blockDim.x) t[e] = 0u;
}

__global__ void __launch_bounds__(256) k_ws_init_batch(const WsInit* __restrict__ items) {
  const WsInit it = items[blockIdx.x];
  zero_bytes(it.B, it.bn * (int64_t)sizeof(double));
  zero_bytes(it.parts_s, it.bytes_s);
  zero_bytes(it.parts_l, it.bytes_l);
  if (threadIdx.x == 0) {
    LzState* st = it.st;
    st->bd_floor = it.bd_scale * *it.xnorm;
    st->full = it.full; st->sweeps = 0; st->sweeps32 = 0;
    st->jc = 0; st->svd_done = 0; st->k = it.k; st->r = it.r; st->kk = it.kk; st->active = 1; st->converged = 0;
    st->nconv = 0; st->breakdown = 0; st->restarts = 0; st->max_restarts = it.maxr;
    st->beta_k = 0.0; st->anorm = 0.0; st->tol = it.tol; st->sigma1 = 0.0; st->maxres = 0.0;
  }
}

// Continuation: the new cycle starts as after a thick restart that keeps the
// r1 Ritz triples of the previous decomposition -- B = diag(sigma_1..r1)
// with the column rho_i = beta_k P[k1-1, i] at r1, unit scales for the Ritz
// columns and the previous residual direction (scale cres) at column r1.
__global__ void k_state_resume(LzState* st, double* B, int k2, double* colscale, const double* sig,
                               const double* P1, int k1, const LzState* old, const double* cres, int r1) {
  for (int e = threadIdx.x; e < k2 * k2; e += blockDim.x) {
    const int c = e / k2, i = e - c * k2;
    double v = 0.0;
    if (c == i && c < r1) v = sig[c];
    else if (c == r1 && i < r1) v = old->beta_k * P1[(k1 - 1) + (int64_t)k1 * i];
    B[e] = v;
  }
  for (int c = threadIdx.x; c < k2 + 2; c += blockDim.x) colscale[c] = c < r1 ? 1.0 : (c == r1 ? *cres : 0.0);
  if (threadIdx.x == 0) {
    st->jc = r1;
    st->anorm = old->anorm;
  }
}

template <typename T>
__global__ void k_sum_parts_to_double(const T* parts, int nparts, int64_t ld, int64_t n, double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int p = 0; p < nparts; ++p) a += (double)parts[p * ld + i];
    out[i] = a;
  }
}

template <typename TO, typename TI>
__global__ void k_convert(const TI* in, TO* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (TO)in[i];
}

// Device error counters of the Lanczos kernels that an engine checks at the
// end of a chunk; their values ride along with the states' read-back (no
// extra synchronisation).
constexpr int N_ERR_WORDS = 2;
enum { EW_RITZ_TC = 0, EW_SHORT_TMA = 1 };
struct ErrWords { int* w[N_ERR_WORDS]; };

__global__ void k_gather_states(LzState* const* src, int n, LzState* dst, ErrWords ew) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = *src[i];
  if (blockIdx.x == 0 && threadIdx.x < N_ERR_WORDS) {
    const int* w = ew.w[threadIdx.x];
    reinterpret_cast<int*>(dst + n)[threadIdx.x] = w ? *w : 0;
  }
}

__global__ void k_kmask(const uint32_t* kbits, int kwords, int cx, int cy, int nx, int ny, uint8_t* out) {
  const int y = blockIdx.y;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nx; x += gridDim.x * blockDim.x) {
    uint8_t v = 0;
    if (x < cx && y < cy) v = (kbits[(int64_t)y * kwords + (x >> 5)] >> (x & 31)) & 1u;
    out[x + (int64_t)nx * y] = v;
  }
}

}  // namespace ssa

static unsigned grid1(int64_t n, int threads = 256) {
  int64_t b = (n + threads - 1) / threads;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 8192));
}

static int ilog2_ceil(int64_t n) {
  int l = 0;
  while ((int64_t(1) << l) < n) ++l;
  return l;
}

// ============================================================== context
struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
};

struct ShapeSet {          // a set of grid points as per-column bit rows
  bool dense = true;       // rectangle [0,bx) x [0,by)
  int bx = 0, by = 0, words = 0;
  uint32_t* bits = nullptr;     // device
  int32_t* colbase = nullptr;   // device, by + 1
  int32_t* cnt = nullptr;       // device scratch, by + 1
  int64_t count = 0;
  MapDev dev() const {
    MapDev m;
    m.dense = dense ? 1 : 0; m.bx = bx; m.by = by; m.words = words;
    m.bits = bits; m.colbase = colbase;
    m.limit = INT64_MAX;
    return m;
  }
};

// Long series (FFT grid above the single-CTA limit) are handled in segment
// form: with block length B, the L x K Hankel matrix is the Hankel-block-
// Hankel matrix of the "segment image" S[i, c] = x[cB + i] (0 <= i < 2B-1):
// window B x ceil(L/B), origins B x ceil(K/B), window element (i, a) <-> row
// aB + i, origin (j, b) <-> column bB + j, so X_{aB+i, bB+j} = x[(a+b)B + i + j]
// = S[i + j, a + b].  Rows and columns past L and K are absent (zero input,
// output dropped), which is what MapDev::limit expresses.
constexpr int FOLD_B = 4096;
constexpr int DECOMP_SPLIT_MIN = 64;   // batches at least this large run as two interleaved halves           // segment length: grid 2B = 8192 along x
constexpr int FOLD_MIN_LOG2 = 15;      // series needing a 2^15 grid or longer are folded

static MapDev fold_map(int B, int nb, int64_t count) {
  MapDev m;
  m.dense = 1; m.bx = B; m.by = nb; m.words = 0; m.bits = nullptr; m.colbase = nullptr; m.limit = count;
  return m;
}

// Segment-form geometry of complete series of lengths n[] with window L.
struct FoldGeom {
  int B = FOLD_B, lb = 0, log2My = 0;
  std::vector<int> kb, fy;
};
static FoldGeom fold_geometry(const std::vector<int64_t>& n, int64_t L) {
  FoldGeom g;
  g.lb = (int)((L + g.B - 1) / g.B);
  int fmax = 1;
  for (int64_t np : n) {
    const int64_t K = std::max<int64_t>(np - L + 1, 1);
    const int kb = (int)((K + g.B - 1) / g.B);
    g.kb.push_back(kb);
    g.fy.push_back(g.lb + kb - 1);
    fmax = std::max(fmax, g.lb + kb - 1);
  }
  g.log2My = std::max(ilog2_ceil(fmax), 1);
  return g;
}

struct Channel {
  int64_t nx = 0, ny = 0;
  int log2M = 0;               // FFT length along x of this channel's products
  int64_t data_off = 0;        // element offset of the channel's data
  ShapeSet K;                  // origins (bounding grid cx x cy)
  int cx = 0, cy = 0;
  int64_t koff = 0;            // offset of the channel's slice in K-vectors
  int32_t* w = nullptr;        // nx*ny weights
  uint32_t* obs = nullptr;     // observed bits, ny x nwords
  int32_t* kpre = nullptr;     // origin bits: word prefix counts per column (run-shaped windows)
  int nwords = 0;
  void* xh32 = nullptr;        // spectra
  void* xh64 = nullptr;
  int kb = 0, fy = 0;          // segment form: origin blocks ceil(K_p/B), segments lb + kb - 1
  double* sq = nullptr;        // sums of squares of the observation kernel's blocks (nsq)
  int64_t nsq = 0;
};

// leading dimension of the FP32 form's float-float short basis: rows rounded
// up to a multiple of four (16-byte aligned FP32 columns for the bulk copies)
static inline int64_t ldf_ff(int64_t Ls) { return (Ls + 3) & ~int64_t(3); }

struct Workspace {             // Lanczos + results, per precision
  int prec = -1, r = 0, k = 0, kk = 0;
  bool swapped = false;
  int64_t Ls = 0, Kl = 0;
  int nblk_s = 0, nblk_l = 0;
  LzState* st = nullptr;
  double* U = nullptr; void* V = nullptr;
  float* Uf = nullptr;         // FP32 form: float-float copy of U for the short side, hi
                               // parts then lo parts (ldf_ff(Ls) x (k+1) each)
  double* p = nullptr; void* q = nullptr;
  void* parts_s = nullptr; void* parts_l = nullptr;
  int n_part_s = 1, n_part_l = 1;
  double* B = nullptr; double* P = nullptr; double* Q = nullptr; double* sig = nullptr;
  double* colscale = nullptr;
  void* uz = nullptr;          // forward transforms of u_j per channel grid size (fused members)
  int64_t uz_off[32] = {};     // element offset of the transform for grid 2^log2M (-1: none)
  void* Cs = nullptr;          // scaled long-side Ritz coefficients, (k + 2) x ritz_ldcs(k) of T
  double* cpa = nullptr; double* cpb = nullptr; double* np_s = nullptr; double* np_l = nullptr;
  void* g1 = nullptr; void* g2 = nullptr;
  void* Uo = nullptr; void* Vo = nullptr;
  double* sigma = nullptr; double* sgn = nullptr;
  bool done = false;
  LzState host_st;
};

struct ssa_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int kind = 0, dtype = 0;
  std::vector<Channel> ch;
  int64_t total = 0;           // data elements
  void* data = nullptr;        // device copy of the input (dtype)
  double* xnorm = nullptr;     // device: ||x||_2 over the observed values (scale of the products' rounding)
  int log2Mx = 0, log2My = 0;
  int fold_B = 0, lb = 0;      // segment form of long series (0: off), window blocks ceil(L/B)
  ShapeSet Lset;               // window set (bounding box ex x ey)
  int ex = 0, ey = 0;
  int32_t* wint = nullptr;     // window columns as runs a, b (null: some column is not a run)
  uint32_t* wrows = nullptr;   // window rows (bits), ey x wwords
  uint32_t* rrows = nullptr;   // reversed window rows
  int wwords = 0;
  int64_t L = 0, K = 0;
  Workspace ws;
  std::vector<std::pair<void*, size_t>> allocs;   // device allocations owned
  int64_t bytes = 0;
  // Buffers with one lifetime are carved from one allocation (an arena):
  // many small stream-ordered allocations per context cost far more than the
  // work they hold.  A request that does not fit falls back to its own block.
  struct Arena { char* base = nullptr; size_t cap = 0, used = 0; };
  Arena embed_arena, spec_arena[2], ws_arena;
  Arena* cur = nullptr;

  int raw_alloc(void** p, size_t n) {
    if (n == 0) n = 16;
    cudaError_t e = cudaMallocAsync(p, n, stream);
    if (e != cudaSuccess) return fail(e == cudaErrorMemoryAllocation ? SSA_ENOMEM : SSA_ECUDA,
                                      "device allocation of %zu bytes: %s", n, cudaGetErrorString(e));
    allocs.push_back({*p, n});
    bytes += (int64_t)n;
    return SSA_OK;
  }
  int make_arena(Arena& a, size_t cap) {
    if (a.base) release(a.base);
    a = Arena();
    TRY(raw_alloc((void**)&a.base, cap));
    a.cap = cap;
    return SSA_OK;
  }
  int alloc(void** p, size_t n) {
    n = (std::max<size_t>(n, 16) + 255) & ~size_t(255);
    if (cur && cur->base && cur->used + n <= cur->cap) {
      *p = cur->base + cur->used;
      cur->used += n;
      return SSA_OK;
    }
    return raw_alloc(p, n);
  }
  template <typename X> int allocT(X** p, size_t count) { return alloc((void**)p, count * sizeof(X)); }
  void release(void* p) {   // arena pieces are freed with their arena
    for (size_t i = 0; i < allocs.size(); ++i)
      if (allocs[i].first == p) {
        cudaFreeAsync(p, stream);
        bytes -= (int64_t)allocs[i].second;
        allocs.erase(allocs.begin() + i);
        return;
      }
  }
};

static inline size_t rnd256(size_t n) { return ((n ? n : 16) + 255) & ~size_t(255); }

// Small host-to-device uploads (work items, window rows) go through a pinned
// ring buffer: a copy from pageable memory would make the driver wait for the
// stream, serialising every context set-up behind the work queued before it.
// A region of the ring is rewritten only after the event recorded behind its
// previous copy has completed.
struct PinnedRing {
  char* base = nullptr;
  size_t cap = 0, head = 0;
  struct Use { size_t a, b; cudaEvent_t ev; };
  std::vector<Use> inflight;      // oldest first
  std::vector<cudaEvent_t> spare;
  ~PinnedRing() {
    for (auto& u : inflight) cudaEventDestroy(u.ev);
    for (auto e : spare) cudaEventDestroy(e);
    if (base) cudaFreeHost(base);
  }
  int copy(void* dst, const void* src, size_t n, cudaStream_t st) {
    if (n == 0) return SSA_OK;
    const size_t need = (n + 255) & ~size_t(255);
    if (!base || need > cap) {
      if (need > (size_t(8) << 20))   // large: plain copy
        return cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, st) == cudaSuccess ? SSA_OK : SSA_ECUDA;
      if (!base) {
        cap = size_t(32) << 20;
        if (cudaHostAlloc((void**)&base, cap, cudaHostAllocDefault) != cudaSuccess) {
          base = nullptr; cap = 0;
          return cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, st) == cudaSuccess ? SSA_OK : SSA_ECUDA;
        }
      }
    }
    if (head + need > cap) head = 0;
    const size_t a = head, b = head + need;
    while (!inflight.empty()) {       // wait for older copies still reading [a, b)
      const Use& u = inflight.front();
      if (u.b <= a || u.a >= b) break;
      cudaEventSynchronize(u.ev);
      spare.push_back(u.ev);
      inflight.erase(inflight.begin());
    }
    std::memcpy(base + a, src, n);
    if (cudaMemcpyAsync(dst, base + a, n, cudaMemcpyHostToDevice, st) != cudaSuccess) return SSA_ECUDA;
    cudaEvent_t ev;
    if (!spare.empty()) { ev = spare.back(); spare.pop_back(); }
    else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return SSA_ECUDA;
    cudaEventRecord(ev, st);
    inflight.push_back({a, b, ev});
    head = b;
    return SSA_OK;
  }
};
static thread_local PinnedRing g_ring;

// upload a small host array into ctx-owned device memory
template <typename X>
static int upload(ssa_ctx* c, const std::vector<X>& h, X** d) {
  TRY(c->allocT(d, std::max<size_t>(h.size(), 1)));
  if (!h.empty() && g_ring.copy(*d, h.data(), h.size() * sizeof(X), c->stream) != SSA_OK)
    return fail(SSA_ECUDA, "upload of %zu bytes failed", h.size() * sizeof(X));
  return SSA_OK;
}

// ============================================================== shapes
// Shapes for a batch of contexts: stage 1 launches the observed bits, origin
// bits and their per-column counts for every channel of every context (one
// launch per kernel kind), stage 2 reads the totals and launches the weights,
// stage 3 checks the error flags -- two host waits for the whole batch.
struct EmbedBatch {
  std::vector<ObsItem> obs;
  std::vector<NormItem> norms;
  std::vector<PrefixItem> opre, kpre;
  int max_opre_cols = 1, max_kpre_cols = 1;
  std::vector<OriginItem> org;
  std::vector<CountItem> cnt;
  std::vector<WeightItem> wts;
  int max_nx = 1, max_ny = 1, max_cx = 0, max_cy = 0, max_cols = 1;
  std::vector<int> cnt_slot_L;                    // per context: count slot of its window set
  std::vector<std::vector<int>> cnt_slot_K;       // per context and channel (-1: empty)
};

static int embed_stage1(ssa_ctx* c, const ssa_window* win, EmbedBatch& eb, int ci, int32_t* d_totals,
                        int* d_err) {
  int ex, ey;
  std::vector<uint8_t> wm;
  if (c->kind == SSA_2D) {
    ex = (int)win->lx; ey = (int)win->ly;
    wm.assign((size_t)ex * ey, 1);
    if (win->wmask) std::memcpy(wm.data(), win->wmask, wm.size());
  } else {
    ex = (int)win->L; ey = 1;
    wm.assign((size_t)ex, 1);
  }
  const int ldm = ex;
  // the window mask's bounding box must start at its first row and column
  int x0 = ex, x1 = -1, y0 = ey, y1 = -1;
  for (int y = 0; y < ey; ++y)
    for (int x = 0; x < ex; ++x)
      if (wm[x + (size_t)ldm * y]) { x0 = std::min(x0, x); x1 = std::max(x1, x); y0 = std::min(y0, y); y1 = std::max(y1, y); }
  if (x1 < 0) return fail(SSA_EINVAL, "window mask is empty");
  if (x0 != 0 || y0 != 0) return fail(SSA_EINVAL, "window mask must touch its first row and column");
  ex = x1 + 1; ey = y1 + 1;
  bool full = true;
  for (int y = 0; y < ey; ++y)
    for (int x = 0; x < ex; ++x) full &= wm[x + (size_t)ldm * y] != 0;
  c->ex = ex; c->ey = ey;
  c->wwords = (ex + 31) / 32;
  std::vector<uint32_t> rows((size_t)ey * c->wwords, 0u), rrows((size_t)ey * c->wwords, 0u);
  for (int y = 0; y < ey; ++y)
    for (int x = 0; x < ex; ++x)
      if (wm[x + (size_t)ldm * y]) {
        rows[(size_t)y * c->wwords + (x >> 5)] |= 1u << (x & 31);
        const int xr = ex - 1 - x;
        rrows[(size_t)y * c->wwords + (xr >> 5)] |= 1u << (xr & 31);
      }
  TRY(upload(c, rows, &c->wrows));
  TRY(upload(c, rrows, &c->rrows));
  // window columns as runs [a, b] where they are (rectangles, discs, triangles)
  std::vector<int32_t> wint((size_t)2 * ey, -1);
  bool runs = true;
  for (int y = 0; y < ey; ++y) {
    int a = -1, b = -1, n = 0;
    for (int x = 0; x < ex; ++x)
      if (wm[x + (size_t)ldm * y]) { if (a < 0) a = x; b = x; ++n; }
    if (a >= 0 && n != b - a + 1) runs = false;
    wint[2 * y] = a; wint[2 * y + 1] = b;
  }
  int32_t* d_wint = nullptr;
  if (runs) TRY(upload(c, wint, &d_wint));
  c->wint = d_wint;
  ShapeSet& Ls = c->Lset;
  Ls.bx = ex; Ls.by = ey; Ls.words = c->wwords;
  Ls.dense = full;
  Ls.bits = c->wrows;
  TRY(c->allocT(&Ls.cnt, (size_t)Ls.by + 1));
  TRY(c->allocT(&Ls.colbase, (size_t)Ls.by + 1));
  eb.cnt_slot_L[ci] = (int)eb.cnt.size();
  eb.cnt.push_back({Ls.bits, Ls.words, Ls.by, Ls.cnt, Ls.colbase, d_totals + eb.cnt.size()});
  eb.max_cols = std::max(eb.max_cols, Ls.by);
  const size_t esz = c->dtype == SSA_F64 ? 8 : 4;
  eb.cnt_slot_K[ci].assign(c->ch.size(), -1);
  // the observation kernel's block sums of squares, one array for all channels
  int64_t nsq = 0;
  for (auto& h : c->ch) nsq += ((h.nx + 255) >> 8) * h.ny;
  double* sq = nullptr;
  TRY(c->allocT(&sq, (size_t)nsq));
  TRY(c->allocT(&c->xnorm, 1));
  eb.norms.push_back({sq, nsq, c->xnorm});
  for (size_t q = 0; q < c->ch.size(); ++q) {
    Channel& h = c->ch[q];
    h.nwords = (int)((h.nx + 31) / 32);
    TRY(c->allocT(&h.obs, (size_t)h.ny * h.nwords));
    h.sq = sq;
    h.nsq = ((h.nx + 255) >> 8) * h.ny;
    sq += h.nsq;
    const void* dptr = (const char*)c->data + h.data_off * esz;
    eb.obs.push_back({dptr, c->dtype == SSA_F64, (int)h.nx, (int)h.ny, h.nwords, h.obs, d_err + ci, h.sq});
    int32_t* opre = nullptr;
    if (runs) {
      TRY(c->allocT(&opre, (size_t)h.ny * (h.nwords + 1)));
      eb.opre.push_back({h.obs, h.nwords, (int)h.ny, opre});
      eb.max_opre_cols = std::max(eb.max_opre_cols, (int)h.ny);
    }
    eb.max_nx = std::max(eb.max_nx, (int)h.nx);
    eb.max_ny = std::max(eb.max_ny, (int)h.ny);
    h.cx = (int)(h.nx - ex + 1);
    h.cy = (int)(h.ny - ey + 1);
    ShapeSet& ks = h.K;
    if (h.cx <= 0 || h.cy <= 0) {
      ks.bx = 0; ks.by = 0; ks.words = 0; ks.count = 0; ks.dense = true;
    } else {
      ks.bx = h.cx; ks.by = h.cy; ks.words = (h.cx + 31) / 32;
      TRY(c->allocT(&ks.bits, (size_t)ks.by * ks.words));
      TRY(c->allocT(&ks.cnt, (size_t)ks.by + 1));
      TRY(c->allocT(&ks.colbase, (size_t)ks.by + 1));
      eb.org.push_back({h.obs, h.nwords, c->wwords, c->wrows, ey, h.cx, h.cy, ks.words, ks.bits, opre, d_wint,
                        runs ? 1 : 0, 0});
      if (runs) {
        TRY(c->allocT(&h.kpre, (size_t)ks.by * (ks.words + 1)));
        eb.kpre.push_back({ks.bits, ks.words, ks.by, h.kpre});
        eb.max_kpre_cols = std::max(eb.max_kpre_cols, ks.by);
      }
      eb.max_cx = std::max(eb.max_cx, h.cx);
      eb.max_cy = std::max(eb.max_cy, h.cy);
      eb.cnt_slot_K[ci][q] = (int)eb.cnt.size();
      eb.cnt.push_back({ks.bits, ks.words, ks.by, ks.cnt, ks.colbase, d_totals + eb.cnt.size()});
      eb.max_cols = std::max(eb.max_cols, ks.by);
    }
    TRY(c->allocT(&h.w, (size_t)(h.nx * h.ny)));
  }
  return SSA_OK;
}

static int embed_stage2(ssa_ctx* c, EmbedBatch& eb, int ci, const int32_t* totals) {
  c->L = totals[eb.cnt_slot_L[ci]];
  c->K = 0;
  for (size_t q = 0; q < c->ch.size(); ++q) {
    Channel& h = c->ch[q];
    ShapeSet& ks = h.K;
    const int slot = eb.cnt_slot_K[ci][q];
    ks.count = slot >= 0 ? totals[slot] : 0;
    if (ks.by > 0) ks.dense = (ks.count == (int64_t)h.cx * h.cy);
    h.koff = c->K;
    c->K += ks.count;
    uint32_t* nb = nullptr;
    TRY(c->allocT(&nb, (size_t)h.ny * h.nwords));
    if (ks.count > 0) {
      eb.wts.push_back({ks.bits, ks.words, ks.by, c->rrows, c->wwords, c->ex, c->ey, (int)h.nx, (int)h.ny,
                        h.nwords, h.w, nb, h.kpre, c->wint, c->wint ? 1 : 0, 0});
    } else {
      CU(cudaMemsetAsync(h.w, 0, sizeof(int32_t) * h.nx * h.ny, c->stream));
    }
  }
  return SSA_OK;
}

static int embed_stage3(ssa_ctx* c, int err) {
  c->cur = nullptr;
  if (err) return fail(SSA_EINVAL, "input holds +-Inf at an observed position");
  if (c->K <= 0) return fail(SSA_EEMPTY, "no window origin keeps the whole window inside the observed set");
  if (c->fold_B)
    for (auto& h : c->ch)
      if (!h.K.dense || h.K.count != h.nx - c->L + 1)
        return fail(SSA_EUNSUPPORTED, "series longer than %d samples must have no missing values", 1 << (FOLD_MIN_LOG2 - 1));
  return SSA_OK;
}

// growable pinned staging buffer (per host thread)
static int32_t* pinned_slots(size_t n) {
  static thread_local int32_t* buf = nullptr;
  static thread_local size_t cap = 0;
  if (n > cap) {
    if (buf) cudaFreeHost(buf);
    size_t nc = std::max<size_t>(n, 1024);
    if (cudaHostAlloc((void**)&buf, nc * sizeof(int32_t), cudaHostAllocDefault) != cudaSuccess) {
      buf = nullptr; cap = 0;
      return nullptr;
    }
    cap = nc;
  }
  return buf;
}

// ============================================================== spectrum
// Data spectra (Sec. 6.1.2: F(x) is computed once and reused by every
// product) for every channel of every context that lacks them, in one launch.
template <typename T>
static int ensure_spectra(ssa_ctx* const* cs, int n, cudaStream_t st) {
  const bool f32 = std::is_same<T, float>::value;
  std::vector<SpecItem<T>> items;
  std::vector<YItem<T>> yitems;
  std::vector<int32_t> sx_pre{0}, sy_pre{0};
  std::vector<std::pair<ssa_ctx*, void*>> scratch;
  int max_ny = 1, max_log2Mx = 1, max_log2My = 0;
  for (int i = 0; i < n; ++i) {
    ssa_ctx* c = cs[i];
    bool have = true;
    for (auto& h : c->ch) have &= (f32 ? h.xh32 : h.xh64) != nullptr;
    if (have) continue;
    cudaStream_t keep = c->stream;
    c->stream = st;
    const int H = 1 << (c->log2Mx - 1), My = 1 << c->log2My;
    void* g1 = nullptr;
    if (c->log2My > 0) {
      TRY(c->raw_alloc(&g1, sizeof(Cx<T>) * (size_t)(H + 1) * My * c->ch.size()));
      scratch.push_back({c, g1});
    }
    ssa_ctx::Arena& ar = c->spec_arena[f32 ? 0 : 1];
    size_t need = 0;
    for (auto& h : c->ch) need += rnd256(sizeof(Cx<T>) * (size_t)((1 << (h.log2M - 1)) + 1) * My);
    TRY(c->make_arena(ar, need));
    ssa_ctx::Arena* keep_cur = c->cur;
    c->cur = &ar;
    const size_t esz = c->dtype == SSA_F64 ? 8 : 4;
    for (size_t q = 0; q < c->ch.size(); ++q) {
      Channel& h = c->ch[q];
      const int Hc = 1 << (h.log2M - 1);
      void* xh = nullptr;
      TRY(c->alloc(&xh, sizeof(Cx<T>) * (size_t)(Hc + 1) * My));
      (f32 ? h.xh32 : h.xh64) = xh;
      SpecItem<T> sp;
      sp.data = (const char*)c->data + h.data_off * esz;
      sp.obs = h.obs; sp.obs_words = h.nwords;
      sp.data_double = c->dtype == SSA_F64;
      sp.nx = (int)h.nx; sp.ny = (int)h.ny;
      sp.ld = h.nx; sp.n_lin = h.nx * h.ny;
      if (c->fold_B) {
        // segment image: column s is x[sB .. sB + 2B - 2] (complete series)
        sp.obs = nullptr; sp.obs_words = 0;
        sp.nx = 2 * c->fold_B - 1; sp.ny = h.fy;
        sp.ld = c->fold_B; sp.n_lin = h.nx;
      }
      sp.log2Mx = h.log2M; sp.log2My = c->log2My;
      sp.g1 = g1 ? (Cx<T>*)g1 + q * (size_t)(H + 1) * My : nullptr;
      sp.xh = (Cx<T>*)xh;
      sp.scale = (T)(1.0 / ((double)(2 * Hc) * (double)My));
      items.push_back(sp);
      sx_pre.push_back(sx_pre.back() + sp.ny);
      if (c->log2My > 0) {
        YItem<T> y;
        y.src = sp.g1; y.dst = sp.xh; y.mul = nullptr; y.st = nullptr;
        y.log2Mx = c->log2Mx; y.log2My = c->log2My; y.in_hi = sp.ny; y.out_hi = My; y.scale = T(0);
        y.tk = tuned_ytk<T>(c->log2Mx, c->log2My);
        yitems.push_back(y);
        sy_pre.push_back(sy_pre.back() + ypass_blocks(c->log2Mx, y.tk));
      }
      max_ny = std::max(max_ny, sp.ny);
    }
    max_log2Mx = std::max(max_log2Mx, c->log2Mx);
    max_log2My = std::max(max_log2My, c->log2My);
    c->cur = keep_cur;
    c->stream = keep;
  }
  if (items.empty()) return SSA_OK;
  PhaseScope ps_(PH_SPECTRUM, st);
  SpecItem<T>* di = nullptr;
  YItem<T>* dy = nullptr;
  if (cudaMallocAsync((void**)&di, sizeof(SpecItem<T>) * items.size(), st) != cudaSuccess ||
      cudaMallocAsync((void**)&dy, sizeof(YItem<T>) * std::max<size_t>(yitems.size(), 1), st) != cudaSuccess)
    return fail(SSA_ENOMEM, "spectrum items");
  if (g_ring.copy(di, items.data(), sizeof(SpecItem<T>) * items.size(), st) != SSA_OK ||
      (!yitems.empty() && g_ring.copy(dy, yitems.data(), sizeof(YItem<T>) * yitems.size(), st) != SSA_OK))
    return fail(SSA_ECUDA, "spectrum item upload");
  int32_t *dpx = nullptr, *dpy = nullptr;
  if (cudaMallocAsync((void**)&dpx, sizeof(int32_t) * sx_pre.size(), st) != cudaSuccess ||
      cudaMallocAsync((void**)&dpy, sizeof(int32_t) * sy_pre.size(), st) != cudaSuccess)
    return fail(SSA_ENOMEM, "spectrum tiles");
  if (g_ring.copy(dpx, sx_pre.data(), sizeof(int32_t) * sx_pre.size(), st) != SSA_OK ||
      g_ring.copy(dpy, sy_pre.data(), sizeof(int32_t) * sy_pre.size(), st) != SSA_OK)
    return fail(SSA_ECUDA, "spectrum tile upload");
  (void)max_ny;
  int max_buf = 0;                  // every item's own tk x padded column must fit
  for (auto& y : yitems) max_buf = std::max(max_buf, (int)y.tk * padded_len(1 << y.log2My));
  launch_spec<T>(di, Tiles{dpx, (int)items.size(), sx_pre.back()}, dy,
                 Tiles{dpy, (int)yitems.size(), sy_pre.back()}, max_log2Mx, max_log2My, twiddles<T>(cs[0]->device), st,
                 max_buf);
  CU(cudaGetLastError());
  cudaFreeAsync(di, st);
  cudaFreeAsync(dy, st);
  cudaFreeAsync(dpx, st);
  cudaFreeAsync(dpy, st);
  for (auto& sc : scratch) {
    cudaStream_t keep = sc.first->stream;
    sc.first->stream = st;
    sc.first->release(sc.second);
    sc.first->stream = keep;
  }
  return SSA_OK;
}

template <typename T>
static int ensure_spectrum(ssa_ctx* c) { return ensure_spectra<T>(&c, 1, c->stream); }

// ============================================================== matvec items
// Direction "X" maps K -> L (sum over channels); "XT" maps L -> K (slices).
template <typename T>
struct MvSet {
  // series on one FFT grid (fused single-CTA products) and grids with a y
  // extent (images, segment-form series: x-pass, y-pass, x-pass)
  // items1[mode]: series products of one k_mv1d code path (mv1d_mode)
  std::vector<MvItem<T>> items1[MV1_MODES], items2;
  std::vector<YItem<T>> yitems2;
  MvItem<T>* d1[MV1_MODES] = {};
  MvItem<T>* d2 = nullptr;
  YItem<T>* dy2 = nullptr;
  int32_t *t_xf = nullptr, *t_yp = nullptr, *t_xi = nullptr;   // block ranges of the 2D launches
  int n_xf = 0, n_yp = 0, n_xi = 0;
  int max_y_in = 0, max_y_out = 0, max_buf = 0;
  int lx1[MV1_MODES] = {}, lx2 = 1, ly2 = 0;   // largest log2 grid sizes of each list
  void add(const MvItem<T>& m) {
    if (m.log2My == 0) {
      const int md = mv1d_mode(m);
      items1[md].push_back(m);
      lx1[md] = std::max(lx1[md], (int)m.log2Mx);
    } else {
      items2.push_back(m);
      lx2 = std::max(lx2, (int)m.log2Mx);
      ly2 = std::max(ly2, (int)m.log2My);
      max_y_in = std::max(max_y_in, (int)m.y_in_hi);
      max_y_out = std::max(max_y_out, (int)m.y_out_hi);
    }
  }
  size_t n1() const {
    size_t n = 0;
    for (auto& v : items1) n += v.size();
    return n;
  }
  size_t size() const { return n1() + items2.size(); }
};

template <typename T>
static MvItem<T> make_mv(ssa_ctx* c, const Channel& h, bool XT, VecRef in, int in_type, VecRef out,
                         Cx<T>* g1, Cx<T>* g2, const LzState* st) {
  MvItem<T> m;
  m.xh = (const Cx<T>*)(std::is_same<T, float>::value ? h.xh32 : h.xh64);
  m.in = in; m.out = out;
  m.in_scale = nullptr;
  m.min = XT ? c->Lset.dev() : h.K.dev();
  m.mout = XT ? h.K.dev() : c->Lset.dev();
  m.g1 = g1; m.g2 = g2; m.st = st;
  m.lV = nullptr; m.lld = 0; m.lB = nullptr; m.lcolscale = nullptr; m.lnpart = nullptr; m.lldb = 0; m.lslot = 0;
  m.zin = nullptr;
  m.log2Mx = h.log2M; m.log2My = c->log2My;
  m.in_type = in_type;
  m.y_in_hi = XT ? c->ey : h.cy;
  m.y_out_hi = XT ? h.cy : c->ey;
  if (c->fold_B) {
    const MapDev wl = fold_map(c->fold_B, c->lb, c->L), ko = fold_map(c->fold_B, h.kb, h.K.count);
    m.min = XT ? wl : ko;
    m.mout = XT ? ko : wl;
    m.y_in_hi = XT ? c->lb : h.kb;
    m.y_out_hi = XT ? h.kb : c->lb;
  }
  m.pad_ = 0;
  return m;
}

template <typename T>
static YItem<T> ymv(const MvItem<T>& m) {
  YItem<T> y;
  y.src = m.g1; y.dst = m.g2; y.mul = m.xh; y.st = m.st;
  y.log2Mx = m.log2Mx; y.log2My = m.log2My;
  y.in_hi = m.y_in_hi; y.out_hi = m.y_out_hi; y.scale = T(0);
  y.tk = tuned_ytk<T>(m.log2Mx, m.log2My);
  return y;
}

// y-pass items of the set's grids, then both lists to the device (uploader
// up(vector, device pointer) of the caller's choosing)
template <typename T, typename Up>
static int finish_set(MvSet<T>& s, Up&& up) {
  s.yitems2.clear();
  std::vector<int32_t> xf{0}, yp{0}, xi{0};
  for (auto& m : s.items2) {
    s.yitems2.push_back(ymv(m));
    s.max_buf = std::max(s.max_buf, (int)s.yitems2.back().tk * padded_len(1 << s.yitems2.back().log2My));
    xf.push_back(xf.back() + m.y_in_hi);
    yp.push_back(yp.back() + ypass_blocks(m.log2Mx, s.yitems2.back().tk));
    xi.push_back(xi.back() + m.y_out_hi);
  }
  for (int md = 0; md < MV1_MODES; ++md)
    if (!s.items1[md].empty()) TRY(up(s.items1[md], &s.d1[md]));
  if (!s.items2.empty()) {
    TRY(up(s.items2, &s.d2));
    TRY(up(s.yitems2, &s.dy2));
    TRY(up(xf, &s.t_xf)); TRY(up(yp, &s.t_yp)); TRY(up(xi, &s.t_xi));
    s.n_xf = xf.back(); s.n_yp = yp.back(); s.n_xi = xi.back();
  }
  return SSA_OK;
}

// the set's products, on stream st of device dev
template <typename T>
static void run_mv(int dev, const MvSet<T>& s, int step, cudaStream_t st) {
  PhaseScope ps_(PH_MATVEC, st);
  for (int md = 0; md < MV1_MODES; ++md)
    if (!s.items1[md].empty())
      launch_mv1d<T>(s.d1[md], (int)s.items1[md].size(), s.lx1[md], step, twiddles<T>(dev), st, md);
  if (!s.items2.empty()) {
    const int n2 = (int)s.items2.size();
    launch_mv2d<T>(s.d2, s.dy2, n2, Tiles{s.t_xf, n2, s.n_xf}, Tiles{s.t_yp, n2, s.n_yp},
                   Tiles{s.t_xi, n2, s.n_xi}, s.lx2, s.ly2, step, twiddles<T>(dev), st, s.max_buf);
  }
}

// ============================================================== decompose (batched)
static int default_k(int r, int64_t L, int64_t K, int req) {
  int64_t mn = std::min(L, K);
  int64_t k = req > 0 ? req : 2 * r + 16;
  k = std::min<int64_t>(k, KMAX);
  k = std::min<int64_t>(k, mn);
  k = std::max<int64_t>(k, r);
  return (int)k;
}

// The long-side step runs inside the X^T u series products (and u's forward
// transform is shared by the channels) when the long side is the origin side
// (each channel's product is its own slice of the long vector) and every
// slice is a dense range.
static size_t uz_bound(const ssa_ctx* c) {     // complex values of all distinct grids
  bool seen[32] = {};
  size_t t = 0;
  for (auto& h : c->ch)
    if (!seen[h.log2M]) { seen[h.log2M] = true; t += size_t(1) << (h.log2M - 1); }
  return t;
}

static bool member_fuses_long(const ssa_ctx* c, bool swapped) {
  if (swapped || c->log2My != 0) return false;
  for (auto& h : c->ch)
    if (!h.K.dense) return false;
  return true;
}

template <typename T>
static int alloc_ws(ssa_ctx* c, const ssa_params& p, Workspace& w, std::vector<WsInit>* batch = nullptr) {
  w = Workspace();
  w.prec = p.prec;
  w.r = p.rank;
  w.k = default_k(p.rank, c->L, c->K, p.krylov_dim ? p.krylov_dim : plan_kdim(p.prec, c->kind, c->L, c->K, p.rank));
  w.kk = std::max(w.r, std::min(w.k - 2, w.r + std::max(8, w.r / 2)));
  w.swapped = c->L > c->K;
  w.Ls = w.swapped ? c->K : c->L;
  w.Kl = w.swapped ? c->L : c->K;
  w.nblk_s = (int)((w.Ls + SHORT_RB - 1) / SHORT_RB);
  w.nblk_l = (int)((w.Kl + LONG_RB - 1) / LONG_RB);
  const int nch = (int)c->ch.size();
  w.n_part_s = w.swapped ? 1 : nch;
  w.n_part_l = w.swapped ? nch : 1;
  const size_t k1 = (size_t)w.k + 1;
  {
    const size_t cz = std::is_same<T, float>::value ? 4 : 8;
    size_t need = rnd256(sizeof(LzState)) + rnd256(8 * w.Ls * k1) + rnd256(cz * w.Kl * k1) + rnd256(8 * w.Ls) +
                  rnd256(cz * w.Kl) + rnd256(cz * w.Ls * w.n_part_s) + rnd256(cz * w.Kl * w.n_part_l) +
                  3 * rnd256(8 * k1 * k1) + 2 * rnd256(8 * (k1 + 1)) + 2 * rnd256(8 * (size_t)w.nblk_s * (KMAX + 1)) +
                  rnd256(8 * (size_t)w.nblk_s) + rnd256(8 * (size_t)std::max<int64_t>(w.nblk_l, (int64_t)c->ch.size())) + rnd256(cz * c->L * w.r) +
                  rnd256(cz * c->K * w.r) + 2 * rnd256(8 * (size_t)w.r) + rnd256(cz * (k1 + 1) * ritz_ldcs(w.k)) +
                  rnd256(2 * cz * uz_bound(c)) + (std::is_same<T, float>::value ? rnd256(8 * (size_t)ldf_ff(w.Ls) * k1) : 0);
    if (c->log2My > 0) {
      const size_t hs = (size_t)((1 << (c->log2Mx - 1)) + 1) << c->log2My;
      need += 2 * rnd256(2 * cz * hs * c->ch.size());
    }
    TRY(c->make_arena(c->ws_arena, need));
  }
  ssa_ctx::Arena* keep_cur = c->cur;
  c->cur = &c->ws_arena;
  TRY(c->allocT(&w.st, 1));
  TRY(c->allocT(&w.U, (size_t)w.Ls * k1));
  w.Uf = nullptr;
  if (std::is_same<T, float>::value) TRY(c->allocT(&w.Uf, 2 * (size_t)ldf_ff(w.Ls) * k1));
  TRY(c->alloc(&w.V, sizeof(T) * (size_t)w.Kl * k1));
  TRY(c->allocT(&w.p, (size_t)w.Ls));
  TRY(c->alloc(&w.q, sizeof(T) * (size_t)w.Kl));
  TRY(c->alloc(&w.parts_s, sizeof(T) * (size_t)w.Ls * w.n_part_s));
  TRY(c->alloc(&w.parts_l, sizeof(T) * (size_t)w.Kl * w.n_part_l));
  TRY(c->allocT(&w.B, (size_t)w.k * w.k));
  TRY(c->allocT(&w.P, (size_t)w.k * w.k));
  TRY(c->allocT(&w.Q, (size_t)(w.k + 1) * w.k));
  TRY(c->allocT(&w.sig, (size_t)w.k));
  TRY(c->allocT(&w.colscale, (size_t)w.k + 2));
  for (auto& o : w.uz_off) o = -1;
  if (member_fuses_long(c, w.swapped)) {
    int64_t tot = 0;
    for (auto& h : c->ch)
      if (w.uz_off[h.log2M] < 0) { w.uz_off[h.log2M] = tot; tot += int64_t(1) << (h.log2M - 1); }
    TRY(c->alloc(&w.uz, sizeof(Cx<T>) * (size_t)tot));
  }
  TRY(c->alloc(&w.Cs, sizeof(T) * (k1 + 1) * ritz_ldcs(w.k)));
  TRY(c->allocT(&w.cpa, (size_t)w.nblk_s * (KMAX + 1)));
  TRY(c->allocT(&w.cpb, (size_t)w.nblk_s * (KMAX + 1)));
  TRY(c->allocT(&w.np_s, (size_t)w.nblk_s));
  TRY(c->allocT(&w.np_l, (size_t)std::max<int64_t>(w.nblk_l, (int64_t)c->ch.size())));
  if (c->log2My > 0) {
    const size_t hs = (size_t)((1 << (c->log2Mx - 1)) + 1) << c->log2My;
    TRY(c->alloc(&w.g1, sizeof(Cx<T>) * hs * nch));
    TRY(c->alloc(&w.g2, sizeof(Cx<T>) * hs * nch));
  }
  TRY(c->alloc(&w.Uo, sizeof(T) * (size_t)c->L * w.r));
  TRY(c->alloc(&w.Vo, sizeof(T) * (size_t)c->K * w.r));
  TRY(c->allocT(&w.sigma, (size_t)w.r));
  TRY(c->allocT(&w.sgn, (size_t)w.r));
  if (!batch) {
    CU(cudaMemsetAsync(w.B, 0, sizeof(double) * w.k * w.k, c->stream));
    CU(cudaMemsetAsync(w.parts_s, 0, sizeof(T) * (size_t)w.Ls * w.n_part_s, c->stream));
    CU(cudaMemsetAsync(w.parts_l, 0, sizeof(T) * (size_t)w.Kl * w.n_part_l, c->stream));
  }
  double tol = p.tol > 0 ? p.tol : (std::is_same<T, float>::value ? 1e-7 : 1e-13);
  int maxr = p.max_restarts > 0 ? p.max_restarts : 40;
  c->cur = keep_cur;
  int lg = 0;
  for (auto& h : c->ch) lg = std::max(lg, h.log2M);
  const double eps_t = std::is_same<T, float>::value ? 5.9604644775390625e-08 : 1.1102230246251565e-16;
  const double bd_scale = 4.0 * eps_t * (double)(lg + c->log2My);
  const int full = w.k == std::min(c->L, c->K) ? 1 : 0;
  if (batch) {
    WsInit wi;
    wi.st = w.st; wi.B = w.B; wi.bn = (int64_t)w.k * w.k;
    wi.parts_s = w.parts_s; wi.bytes_s = (int64_t)sizeof(T) * w.Ls * w.n_part_s;
    wi.parts_l = w.parts_l; wi.bytes_l = (int64_t)sizeof(T) * w.Kl * w.n_part_l;
    wi.k = w.k; wi.r = w.r; wi.kk = w.kk; wi.maxr = maxr; wi.full = full; wi.pad_ = 0;
    wi.tol = tol; wi.xnorm = c->xnorm; wi.bd_scale = bd_scale;
    batch->push_back(wi);
    return SSA_OK;
  }
  k_state_init<<<1, 1, 0, c->stream>>>(w.st, w.k, w.r, w.kk, tol, maxr, full, c->xnorm, bd_scale); count_launch();
  CU(cudaGetLastError());
  return SSA_OK;
}

// Lanczos engine: a set of problems (contexts with a workspace) that advance
// together, one launch per kernel kind for all of them.  Each member keeps its
// own position (LzState::jc) in its own restart cycle: a chunk of steps moves
// every member that is inside a cycle, the small SVD runs for the members
// whose cycle just ended, and the host then retires or restarts exactly those.
// Members can be added and removed between chunks -- the batched
// decomposition and the server use the same engine.
template <typename T>
struct LzEngine {
  cudaStream_t st = nullptr;
  int device = 0;
  std::vector<ssa_ctx*> live;
  std::vector<uint64_t> seed;
  std::vector<bool> fresh;        // not started yet (no start vector)
  std::vector<LzState> hst;       // host copy after the last chunk (kept current for restarts)
  bool dirty = true;              // membership changed since the item arrays were built
  // device item arrays for the current membership
  ShortItem* d_sh = nullptr; LongItem<T>* d_lg = nullptr; SvdItem* d_sv = nullptr;
  RitzItem<T>* d_rz = nullptr; LzState** d_stp = nullptr; LzState* d_stg = nullptr;
  // block ranges of the members in the row-block launches
  int32_t *t_sh = nullptr, *t_lg = nullptr, *t_rs = nullptr, *t_rl = nullptr;
  int n_sh = 0, n_lg = 0, n_rs = 0, n_rl = 0;
  ShortItem* d_shf = nullptr;      // members whose short step runs in one block
  int n_shf = 0;
  int64_t max_ls_f = 1;
  UzItem<T>* d_uz = nullptr;       // shared forward transforms of u_j
  int n_uz = 0, max_uz_log2 = 1;
  bool share_u = false;            // X^T u products take u's transform from k_uspec
  MvSet<T> mvA, mvAT;
  int max_blk_s = 1, max_blk_l = 1, max_k = 1, max_kk = 1, max_r = 1;
  int64_t max_Ls = 1, max_Kl = 1, max_rows = 1;
  int max_log2Mx = 1, max_log2My = 0;
  std::vector<void*> dev_tmp;
  LzState* h_st = nullptr;
  int h_cap = 0;

  ~LzEngine() { release_items(); if (h_st) cudaFreeHost(h_st); }

  std::vector<void*> chunk_tmp;   // per-chunk item arrays, freed by the next chunk
  void release_chunk() {
    for (void* p : chunk_tmp) cudaFreeAsync(p, st);
    chunk_tmp.clear();
  }
  void release_items() {
    release_chunk();
    for (void* p : dev_tmp) cudaFreeAsync(p, st);
    dev_tmp.clear();
    mvA = MvSet<T>(); mvAT = MvSet<T>();
  }

  template <typename X>
  int up(const std::vector<X>& h, X** d) {
    if (cudaMallocAsync((void**)d, sizeof(X) * std::max<size_t>(h.size(), 1), st) != cudaSuccess)
      return fail(SSA_ENOMEM, "engine items");
    dev_tmp.push_back(*d);
    if (!h.empty() && g_ring.copy(*d, h.data(), sizeof(X) * h.size(), st) != SSA_OK)
      return fail(SSA_ECUDA, "engine item upload");
    return SSA_OK;
  }

  // prefix of per-member block counts, uploaded; *total = grid size
  template <typename F>
  int tiles(const std::vector<ssa_ctx*>& cs, F&& per, int32_t** d, int* total) {
    std::vector<int32_t> p{0};
    for (ssa_ctx* c : cs) p.push_back(p.back() + (int32_t)per(c));
    *total = p.back();
    return up(p, d);
  }
  static int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
  int ritz_tiles(const std::vector<ssa_ctx*>& cs, int32_t** ds, int* ns, int32_t** dl, int* nl) {
    TRY(tiles(cs, [](ssa_ctx* c) { return cdiv(c->ws.Ls, RITZ_RB_SHORT); }, ds, ns));
    TRY(tiles(cs, [](ssa_ctx* c) { return cdiv(c->ws.Kl, ritz_rb_long<T>()); }, dl, nl));
    return SSA_OK;
  }

  // The long-side step runs inside the X^T u series products when the long
  // side is the origin side (each channel's product is its own slice of the
  // long vector) and every slice is a dense range.
  static bool fuse_long(ssa_ctx* c) { return member_fuses_long(c, c->ws.swapped); }

  // The whole short-side step in one block per problem pays off when the
  // problems fill the GPU; a few problems with a long short side (an image
  // with a 64 x 64 window: 4096 rows) would leave most SMs idle for a step
  // that is FP64-bound, so they take the row-block kernels instead.
  int sm_count = 0;
  bool fused_short(ssa_ctx* c) {
    if (c->ws.Ls > SHORT_FUSED_MAX) return false;
    if (!sm_count && cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
      sm_count = 1;
    return c->ws.Ls <= 512 || (int)live.size() >= sm_count;
  }

  ShortItem short_item(ssa_ctx* c, uint64_t sd) {
    Workspace& w = c->ws;
    ShortItem s;
    s.seed = sd;
    s.st = w.st; s.U = w.U; s.ldf = ldf_ff(w.Ls); s.ldu = w.Ls;
    s.Uh = w.Uf; s.Ul = w.Uf ? w.Uf + (size_t)s.ldf * (w.k + 1) : nullptr; s.parts = w.parts_s; s.part_ld = w.Ls; s.n_part = w.n_part_s;
    s.parts_double = std::is_same<T, double>::value; s.p = w.p; s.B = w.B; s.ldb = w.k; s.nblk = w.nblk_s;
    s.cpa = w.cpa; s.cpb = w.cpb; s.npart = w.np_s; s.Ls = w.Ls;
    return s;
  }
  LongItem<T> long_item(ssa_ctx* c, uint64_t sd) {
    Workspace& w = c->ws;
    LongItem<T> l;
    l.st = w.st; l.V = (T*)w.V; l.ldv = w.Kl; l.colscale = w.colscale; l.parts = (const T*)w.parts_l;
    l.part_ld = w.Kl; l.n_part = w.n_part_l; l.nblk = w.nblk_l; l.q = (T*)w.q; l.npart = w.np_l; l.B = w.B;
    l.ldb = w.k; l.Kl = w.Kl; l.seed = sd;
    l.nsum = fuse_long(c) ? (int)c->ch.size() : w.nblk_l;
    return l;
  }
  SvdItem svd_item(ssa_ctx* c) {
    Workspace& w = c->ws;
    SvdItem v;
    v.st = w.st; v.B = w.B; v.ldb = w.k; v.ffpolish = std::is_same<T, float>::value; v.colscale = w.colscale; v.sig = w.sig; v.P = w.P; v.Q = w.Q;
    return v;
  }
  RitzItem<T> ritz_item(ssa_ctx* c) {
    Workspace& w = c->ws;
    RitzItem<T> z;
    z.st = w.st; z.U = w.U; z.ldu = w.Ls; z.Ls = w.Ls; z.V = (T*)w.V; z.ldv = w.Kl; z.Kl = w.Kl;
    z.colscale = w.colscale; z.P = w.P; z.Q = w.Q; z.ldc = w.k; z.ldcs = ritz_ldcs(w.k); z.Cs = (T*)w.Cs;
    z.ldf = ldf_ff(w.Ls);
    z.Uh = w.Uf; z.Ul = w.Uf ? w.Uf + (size_t)z.ldf * (w.k + 1) : nullptr;
    return z;
  }
  FinalItem<T> final_item(ssa_ctx* c) {
    Workspace& w = c->ws;
    FinalItem<T> f;
    f.st = w.st; f.U = w.U; f.ldu = w.Ls; f.Ls = w.Ls; f.V = (const T*)w.V; f.ldv = w.Kl; f.Kl = w.Kl;
    f.sig = w.sig; f.swapped = w.swapped; f.r = w.r; f.Uo = (T*)w.Uo; f.Vo = (T*)w.Vo; f.sigma_out = w.sigma;
    f.sgn = w.sgn;
    return f;
  }

  void add(ssa_ctx* c, uint64_t sd) {
    live.push_back(c); seed.push_back(sd); fresh.push_back(true);
    LzState z{};
    z.k = c->ws.k; z.kk = c->ws.kk; z.r = c->ws.r; z.jc = 0; z.active = 1;
    hst.push_back(z);
    dirty = true;
  }
  // a member whose bases already hold jc vectors (a continued decomposition)
  void add_resumed(ssa_ctx* c, int jc) {
    add(c, 0);
    fresh.back() = false;
    hst.back().jc = jc;
    if (std::is_same<T, float>::value) uf_pending.push_back({c, jc});
  }
  // Uf[:, 0:n] <- U[:, 0:n] of the given members (their float-float copy
  // after U was written in FP64)
  std::vector<std::pair<ssa_ctx*, int>> uf_pending;
  int sync_uf(const std::vector<std::pair<ssa_ctx*, int>>& ms) {
    std::vector<ShortItem> it;
    std::vector<int32_t> nc;
    for (auto& m : ms)
      if (m.second > 0) { it.push_back(short_item(m.first, 0)); nc.push_back(m.second); }
    if (it.empty()) return SSA_OK;
    ShortItem* d_i = nullptr;
    int32_t* d_n = nullptr;
    const size_t keep = dev_tmp.size();
    TRY(up(it, &d_i));
    TRY(up(nc, &d_n));
    chunk_tmp.insert(chunk_tmp.end(), dev_tmp.begin() + keep, dev_tmp.end());
    dev_tmp.resize(keep);
    launch_uf_sync(d_i, d_n, (int)it.size(), st);
    return SSA_OK;
  }

  // rebuild the device item arrays for the current members (when they changed)
  int build() {
    if (!dirty) return SSA_OK;
    dirty = false;
    release_items();
    // one extra launch per step pays off once enough products share it
    share_u = live.size() >= 32;
    std::vector<ShortItem> sh; std::vector<LongItem<T>> lg; std::vector<SvdItem> sv;
    std::vector<RitzItem<T>> rz; std::vector<LzState*> stp;
    max_blk_s = max_blk_l = max_k = max_kk = max_r = 1;
    max_Ls = max_Kl = max_rows = 1;
    max_log2Mx = 1; max_log2My = 0;
    for (size_t i = 0; i < live.size(); ++i) {
      ssa_ctx* c = live[i];
      Workspace& w = c->ws;
      sh.push_back(short_item(c, seed[i])); lg.push_back(long_item(c, seed[i])); sv.push_back(svd_item(c));
      rz.push_back(ritz_item(c)); stp.push_back(w.st);
      const size_t hs = c->log2My > 0 ? ((size_t)((1 << (c->log2Mx - 1)) + 1) << c->log2My) : 0;
      for (size_t q = 0; q < c->ch.size(); ++q) {
        const Channel& h = c->ch[q];
        Cx<T>* g1 = hs ? (Cx<T>*)w.g1 + q * hs : nullptr;
        Cx<T>* g2 = hs ? (Cx<T>*)w.g2 + q * hs : nullptr;
        VecRef vin{}, vout{};
        if (!w.swapped) {
          // A v = X v : K -> L partial per channel
          vin.base = w.V; vin.off = h.koff; vin.ld = w.Kl; vin.st = w.st; vin.jdelta = 0;
          vout.base = w.parts_s; vout.off = (int64_t)q * w.Ls; vout.ld = 0; vout.st = nullptr;
          MvItem<T> m = make_mv<T>(c, h, false, vin, 0, vout, g1, g2, w.st);
          m.in_scale = w.colscale;
          mvA.add(m);
          // A^T u = X^T u : L -> K slice
          vin.base = w.U; vin.off = 0; vin.ld = w.Ls; vin.st = w.st;
          vout.base = w.parts_l; vout.off = h.koff; vout.st = nullptr;
          MvItem<T> mt = make_mv<T>(c, h, true, vin, 1, vout, g1, g2, w.st);
          if (fuse_long(c)) {
            mt.lV = (T*)w.V; mt.lld = w.Kl; mt.lB = w.B; mt.lcolscale = w.colscale; mt.lnpart = w.np_l;
            mt.lldb = w.k; mt.lslot = (int32_t)q;
            if (share_u) mt.zin = (const Cx<T>*)w.uz + w.uz_off[h.log2M];
          }
          mvAT.add(mt);
        } else {
          // A v = X^T v : L -> K slice
          vin.base = w.V; vin.off = 0; vin.ld = w.Kl; vin.st = w.st;
          vout.base = w.parts_s; vout.off = h.koff; vout.st = nullptr;
          MvItem<T> m = make_mv<T>(c, h, true, vin, 0, vout, g1, g2, w.st);
          m.in_scale = w.colscale;
          mvA.add(m);
          // A^T u = X u : K -> L partial
          vin.base = w.U; vin.off = h.koff; vin.ld = w.Ls; vin.st = w.st;
          vout.base = w.parts_l; vout.off = (int64_t)q * w.Kl; vout.st = nullptr;
          mvAT.add(make_mv<T>(c, h, false, vin, 1, vout, g1, g2, w.st));
        }
      }
      max_blk_s = std::max(max_blk_s, w.nblk_s);
      max_blk_l = std::max(max_blk_l, w.nblk_l);
      max_k = std::max(max_k, w.k);
      max_kk = std::max(max_kk, w.kk);
      max_r = std::max(max_r, w.r);
      max_Ls = std::max(max_Ls, w.Ls);
      max_Kl = std::max(max_Kl, w.Kl);
      max_rows = std::max(max_rows, std::max(c->L, c->K));
      max_log2Mx = std::max(max_log2Mx, c->log2Mx);
      max_log2My = std::max(max_log2My, c->log2My);
    }
    if (live.empty()) return SSA_OK;
    if (!uf_pending.empty()) {
      TRY(sync_uf(uf_pending));
      uf_pending.clear();
    }
    TRY(up(sh, &d_sh)); TRY(up(lg, &d_lg)); TRY(up(sv, &d_sv)); TRY(up(rz, &d_rz)); TRY(up(stp, &d_stp));
    TRY(tiles(live, [this](ssa_ctx* c) { return fused_short(c) ? 0 : c->ws.nblk_s; }, &t_sh, &n_sh));
    {
      std::vector<UzItem<T>> uz;
      max_uz_log2 = 1;
      for (ssa_ctx* c : live) {
        if (!share_u || !fuse_long(c)) continue;
        Workspace& w = c->ws;
        for (int lg = 0; lg < 32; ++lg)
          if (w.uz_off[lg] >= 0) {
            UzItem<T> z;
            z.U = w.U; z.ldu = w.Ls; z.st = w.st; z.L = (int32_t)c->L; z.log2M = lg;
            z.z = (Cx<T>*)w.uz + w.uz_off[lg];
            uz.push_back(z);
            max_uz_log2 = std::max(max_uz_log2, lg);
          }
      }
      n_uz = (int)uz.size();
      d_uz = nullptr;
      if (n_uz) TRY(up(uz, &d_uz));
    }
    {
      std::vector<ShortItem> shf;
      max_ls_f = 1;
      for (size_t i = 0; i < live.size(); ++i) {
        ssa_ctx* c = live[i];
        if (fused_short(c)) { shf.push_back(short_item(c, seed[i])); max_ls_f = std::max(max_ls_f, c->ws.Ls); }
      }
      n_shf = (int)shf.size();
      d_shf = nullptr;
      if (n_shf) TRY(up(shf, &d_shf));
    }
    TRY(tiles(live, [](ssa_ctx* c) { return fuse_long(c) ? 0 : c->ws.nblk_l; }, &t_lg, &n_lg));
    TRY(ritz_tiles(live, &t_rs, &n_rs, &t_rl, &n_rl));
    auto upl = [&](auto& v, auto** d) { return up(v, d); };
    TRY(finish_set(mvA, upl));
    TRY(finish_set(mvAT, upl));
    if (cudaMallocAsync((void**)&d_stg, sizeof(LzState) * live.size() + sizeof(int) * N_ERR_WORDS, st) !=
        cudaSuccess)
      return fail(SSA_ENOMEM, "engine state buffer");
    dev_tmp.push_back(d_stg);
    if ((int)live.size() > h_cap) {
      if (h_st) cudaFreeHost(h_st);
      h_cap = std::max((int)live.size(), 256);
      if (cudaHostAlloc((void**)&h_st, sizeof(LzState) * h_cap + sizeof(int) * N_ERR_WORDS, cudaHostAllocDefault) !=
          cudaSuccess) {
        h_st = nullptr; h_cap = 0;
        return fail(SSA_ENOMEM, "pinned state buffer");
      }
    }
    return SSA_OK;
  }

  // start vectors of the members not started yet
  int start_fresh() {
    std::vector<LongItem<T>> lg;
    std::vector<ssa_ctx*> cs;
    for (size_t i = 0; i < live.size(); ++i)
      if (fresh[i]) { lg.push_back(long_item(live[i], seed[i])); cs.push_back(live[i]); fresh[i] = false; }
    if (lg.empty()) return SSA_OK;
    LongItem<T>* d = nullptr;
    int32_t* tp = nullptr;
    int nt = 0;
    TRY(up(lg, &d));
    TRY(tiles(cs, [](ssa_ctx* c) { return c->ws.nblk_l; }, &tp, &nt));
    PhaseScope ps_(PH_LONG, st);
    launch_long_init<T>(d, tp, (int)lg.size(), nt, st);
    CU(cudaGetLastError());
    return SSA_OK;
  }

  // One chunk: every member inside a cycle advances up to `steps` Lanczos
  // steps (its own jc); members whose cycle is complete get their small SVD;
  // the states are read back.  The chunk runs until the member closest to the
  // end of its cycle gets there (at least 8 steps when others have that many
  // left), so no member waits for a whole cycle of another.
  // number of steps of the next chunk (0 when no member is inside a cycle)
  int plan_steps() {
    release_chunk();
    int rmin = INT32_MAX, rmax = 0;
    for (size_t i = 0; i < live.size(); ++i) {
      const LzState& h = hst[i];
      if (!h.active || h.svd_done || h.jc >= h.k) continue;
      rmin = std::min(rmin, h.k - h.jc);
      rmax = std::max(rmax, h.k - h.jc);
    }
    return rmax == 0 ? 0 : std::min(rmax, std::max(rmin, 8));
  }
  // one Lanczos step for every member inside a cycle
  void issue_step() {
    const int nl = (int)live.size();
    run_mv<T>(device, mvA, 0, st);
    {
      PhaseScope ps_(PH_SHORT, st);
      if (std::is_same<T, float>::value) {
        launch_short_steps_ff(d_sh, t_sh, nl, n_sh, 0, st);
        launch_short_fused_ff(d_shf, n_shf, max_ls_f, 0, st);
      } else {
        launch_short_steps(d_sh, t_sh, nl, n_sh, 0, st);
        launch_short_fused(d_shf, n_shf, max_ls_f, 0, st);
      }
    }
    {
      PhaseScope ps_(PH_MATVEC, st);
      launch_uspec<T>(d_uz, n_uz, max_uz_log2, 0, twiddles<T>(device), st);
    }
    run_mv<T>(device, mvAT, 0, st);
    { PhaseScope ps_(PH_LONG, st); launch_long_step<T>(d_lg, t_lg, nl, n_lg, 0, st); }
  }
  // Small SVDs of the members whose cycle ended, then their thick restarts
  // (Ritz vectors, new B) -- launched over every member: the kernels pick the
  // members on the device (active, small SVD done), so the restart needs no
  // read-back first -- and the state read-back (async).
  int finish_chunk_async() {
    const int nl = (int)live.size();
    {
      PhaseScope ps_(PH_RITZ, st);
      launch_bsvd(d_sv, nl, max_k, st);
      launch_ritz<T>(d_rz, nl, max_k, max_kk, t_rs, n_rs, t_rl, n_rl, 0, st);
      launch_restart(d_sv, nl, st);
    }
    CU(cudaGetLastError());
    ErrWords ew;
    ew.w[EW_RITZ_TC] = ritz_tc_timeout_word();
    ew.w[EW_SHORT_TMA] = short_tma_timeout_word();
    for (int q = 0; q < N_ERR_WORDS; ++q)
      if (!ew.w[q]) return fail(SSA_ECUDA, "device error counters unavailable");
    k_gather_states<<<1, 128, 0, st>>>(d_stp, nl, d_stg, ew); count_launch();
    CU(cudaMemcpyAsync(h_st, d_stg, sizeof(LzState) * nl + sizeof(int) * N_ERR_WORDS, cudaMemcpyDeviceToHost, st));
    return SSA_OK;
  }
  // after the states' read-back: the chunk's error counters (nonzero ones are
  // reset on the device and reported); the series products' counters are
  // read (and reset) by their own calls
  int finish_chunk_sync() {
    const int nl = (int)live.size();
    CU(cudaStreamSynchronize(st));
    for (int i = 0; i < nl; ++i) hst[i] = h_st[i];
    const int* err = reinterpret_cast<const int*>(h_st + nl);
    if (err[EW_RITZ_TC] || err[EW_SHORT_TMA]) {
      const int e_rt = err[EW_RITZ_TC], e_sh = err[EW_SHORT_TMA];
      const int z = 0;
      int* words[N_ERR_WORDS] = {ritz_tc_timeout_word(), short_tma_timeout_word()};
      for (int q = 0; q < N_ERR_WORDS; ++q)
        if (err[q] && words[q]) cudaMemcpyAsync(words[q], &z, sizeof(int), cudaMemcpyHostToDevice, st);
      cudaStreamSynchronize(st);
      if (e_rt) return fail(SSA_ETIMEOUT, "a tensor-core Ritz update did not complete");
      if (e_sh) return fail(SSA_ETIMEOUT, "a bulk copy of the short-side basis did not complete");
    }
    if ((mvA.n1() || mvAT.n1()) && mv_async_timeouts(st) != 0)
      return fail(SSA_ETIMEOUT, "a bulk copy of a data spectrum did not complete");
    if (max_log2My > 0 && ypass_bad_tiles(st) != 0)
      return fail(SSA_ECUDA, "a y-pass tile did not fit its launch's buffers");
    if (std::is_same<T, float>::value && ritz_tc_plan_failures() != 0)
      return fail(SSA_ENOMEM, "no scratch for a tensor-core Ritz update's tile plan");
    return SSA_OK;
  }
  // One chunk: every member inside a cycle advances up to `steps` Lanczos
  // steps (its own jc); members whose cycle is complete get their small SVD;
  // the states are read back.  The chunk runs until the member closest to the
  // end of its cycle gets there (at least 8 steps when others have that many
  // left), so no member waits for a whole cycle of another.
  int run_chunk() {
    if (live.empty()) return SSA_OK;
    const int steps = plan_steps();
    for (int s = 0; s < steps; ++s) issue_step();
    TRY(finish_chunk_async());
    return finish_chunk_sync();
  }
  bool any_active() const {
    for (auto& h : hst) if (h.active) return true;
    return false;
  }

  // final Ritz vectors and outputs of the given members
  int retire(const std::vector<int>& idx) {
    if (idx.empty()) return SSA_OK;
    std::vector<RitzItem<T>> rz; std::vector<FinalItem<T>> fi;
    std::vector<ssa_ctx*> cs;
    int mk = 1, mr = 1;
    int64_t mls = 1, mkl = 1, mrows = 1;
    for (int i : idx) {
      ssa_ctx* c = live[i];
      cs.push_back(c);
      rz.push_back(ritz_item(c)); fi.push_back(final_item(c));
      mk = std::max(mk, c->ws.k); mr = std::max(mr, c->ws.r);
      mls = std::max(mls, c->ws.Ls); mkl = std::max(mkl, c->ws.Kl);
      mrows = std::max(mrows, std::max(c->L, c->K));
    }
    RitzItem<T>* d_r = nullptr; FinalItem<T>* d_f = nullptr;
    int32_t *ts = nullptr, *tl = nullptr;
    int ns = 0, nl = 0;
    TRY(up(rz, &d_r)); TRY(up(fi, &d_f));
    TRY(ritz_tiles(cs, &ts, &ns, &tl, &nl));
    PhaseScope ps_(PH_RITZ, st);
    launch_ritz<T>(d_r, (int)idx.size(), mk, mr, ts, ns, tl, nl, 1, st);
    launch_finalize<T>(d_f, (int)idx.size(), mr, mrows, st);
    CU(cudaGetLastError());
    for (int i : idx) {
      Workspace& w = live[i]->ws;
      w.host_st = hst[i];
      w.done = true;
    }
    return SSA_OK;
  }

  // drop members (after retire)
  void remove(const std::vector<int>& idx) {
    std::vector<bool> drop(live.size(), false);
    for (int i : idx) drop[i] = true;
    std::vector<ssa_ctx*> l2; std::vector<uint64_t> s2; std::vector<bool> f2; std::vector<LzState> h2;
    for (size_t i = 0; i < live.size(); ++i)
      if (!drop[i]) { l2.push_back(live[i]); s2.push_back(seed[i]); f2.push_back(fresh[i]); h2.push_back(hst[i]); }
    live.swap(l2); seed.swap(s2); fresh.swap(f2); hst.swap(h2);
    if (!idx.empty()) dirty = true;
  }
};

// Admission of problems into an engine: spectra and workspaces.
template <typename T>
static int prepare_members(ssa_ctx* const* cs, int n, const ssa_params* ps, cudaStream_t st, std::vector<int>& rc) {
  rc.assign(n, SSA_OK);
  std::vector<ssa_ctx*> need;
  for (int i = 0; i < n; ++i) {
    if (ps[i].rank < 1 || ps[i].rank > std::min(cs[i]->L, cs[i]->K))
      rc[i] = fail(SSA_ERANK, "rank %d outside [1, min(L, K) = %lld]", ps[i].rank,
                   (long long)std::min(cs[i]->L, cs[i]->K));
    else need.push_back(cs[i]);
  }
  if (!need.empty()) TRY(ensure_spectra<T>(need.data(), (int)need.size(), st));
  std::vector<WsInit> init;
  for (int i = 0; i < n; ++i) {
    if (rc[i] != SSA_OK) continue;
    ssa_ctx* c = cs[i];
    cudaStream_t keep = c->stream;
    c->stream = st;
    rc[i] = alloc_ws<T>(c, ps[i], c->ws, &init);
    c->stream = keep;
  }
  if (!init.empty()) {
    WsInit* d = nullptr;
    if (cudaMallocAsync((void**)&d, sizeof(WsInit) * init.size(), st) != cudaSuccess)
      return fail(SSA_ENOMEM, "workspace init items");
    if (g_ring.copy(d, init.data(), sizeof(WsInit) * init.size(), st) != SSA_OK)
      return fail(SSA_ECUDA, "workspace init item upload");
    k_ws_init_batch<<<(unsigned)init.size(), 256, 0, st>>>(d); count_launch();
    CU(cudaGetLastError());
    cudaFreeAsync(d, st);
  }
  return SSA_OK;
}

template <typename T>
static int decompose_batch_T(ssa_ctx* const* cs, int n, const ssa_params* ps, int32_t* status) {
  ssa_ctx* c0 = cs[0];
  cudaStream_t st = c0->stream;
  // make every context's prior work visible on the batch stream
  std::vector<cudaEvent_t> evs;
  for (int i = 1; i < n; ++i)
    if (cs[i]->stream != st) {
      cudaEvent_t e;
      CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      CU(cudaEventRecord(e, cs[i]->stream));
      CU(cudaStreamWaitEvent(st, e, 0));
      evs.push_back(e);
    }
  std::vector<int> rc;
  TRY(prepare_members<T>(cs, n, ps, st, rc));
  // Large batches run as two engines on two streams whose launches are issued
  // alternately: one half's FP64-bound kernels (Gram-Schmidt, small SVD) then
  // share the SMs with the other half's FP32 products.  Each problem's
  // arithmetic is the same either way.
  int nok = 0;
  for (int i = 0; i < n; ++i) nok += rc[i] == SSA_OK;
  const int ng = nok >= DECOMP_SPLIT_MIN ? 2 : 1;
  LzEngine<T> engs[2];
  cudaStream_t gst[2] = {st, st};
  cudaEvent_t ready = nullptr;
  if (ng == 2) {
    CU(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    CU(cudaEventRecord(ready, st));
    for (int g = 0; g < 2; ++g) {
      CU(cudaStreamCreateWithFlags(&gst[g], cudaStreamNonBlocking));
      CU(cudaStreamWaitEvent(gst[g], ready, 0));
    }
  }
  int placed = 0;
  for (int i = 0; i < n; ++i) {
    if (status) status[i] = rc[i];
    if (rc[i] == SSA_OK) {
      LzEngine<T>& e = engs[(ng == 2 && placed >= nok / 2) ? 1 : 0];
      e.add(cs[i], ps[i].seed);
      ++placed;
    } else {
      cs[i]->ws.done = false;
    }
  }
  int rc_all = SSA_OK;
  int rc_run = SSA_OK;
  auto run = [&]() -> int {
    for (int g = 0; g < ng; ++g) {
      engs[g].st = gst[g];
      engs[g].device = c0->device;
      if (engs[g].live.empty()) continue;
      TRY(engs[g].build());
      TRY(engs[g].start_fresh());
    }
    // Each engine runs its chunks on its own stream: as soon as one engine's
    // chunk is read back, its next chunk is issued, while the other engine's
    // chunk still runs (the GPU does not drain at a chunk boundary).
    bool pend[2] = {false, false};
    auto issue_chunk = [&](int g) -> int {
      LzEngine<T>& e = engs[g];
      const int steps = e.plan_steps();
      for (int s2 = 0; s2 < steps; ++s2) e.issue_step();
      TRY(e.finish_chunk_async());
      pend[g] = true;
      return SSA_OK;
    };
    for (int g = 0; g < ng; ++g)
      if (!engs[g].live.empty() && engs[g].any_active()) TRY(issue_chunk(g));
    for (;;) {
      bool any = false;
      for (int g = 0; g < ng; ++g) {
        if (!pend[g]) continue;
        pend[g] = false;
        TRY(engs[g].finish_chunk_sync());
        if (engs[g].any_active()) TRY(issue_chunk(g));
        any |= pend[g];
      }
      if (!any) break;
    }
    for (int g = 0; g < ng; ++g) {
      LzEngine<T>& eng = engs[g];
      if (eng.live.empty()) continue;
      std::vector<int> all(eng.live.size());
      for (size_t i = 0; i < all.size(); ++i) all[i] = (int)i;
      TRY(eng.retire(all));
      CU(cudaStreamSynchronize(eng.st));
      if (std::is_same<T, float>::value && ritz_tc_timeouts(eng.st) != 0)
        return fail(SSA_ETIMEOUT, "a tensor-core Ritz update did not complete");
      for (size_t i = 0; i < eng.live.size(); ++i) {
        const LzState& h = eng.hst[i];
        if (!h.converged) {
          const int idx = (int)(std::find(cs, cs + n, eng.live[i]) - cs);
          if (status) status[idx] = SSA_ENOTCONV;
          if (rc_all == SSA_OK) rc_all = fail(SSA_ENOTCONV, "restarts exhausted (max residual %.3g)", h.maxres);
        }
      }
    }
    return SSA_OK;
  };
  rc_run = run();
  if (ng == 2) {
    // later work on the batch stream (reconstruction) follows both halves;
    // the engines free their item arrays on their streams before those go
    for (int g = 0; g < 2; ++g) {
      engs[g].release_items();
      cudaStreamSynchronize(gst[g]);
      cudaStreamDestroy(gst[g]);
      engs[g].st = st;
    }
    cudaEventDestroy(ready);
  }
  if (rc_run != SSA_OK) return rc_run;
  for (auto e : evs) cudaEventDestroy(e);
  for (int i = 0; i < n; ++i)
    if (rc[i] != SSA_OK && rc_all == SSA_OK) rc_all = rc[i];
  return rc_all;
}

// Continued decomposition to a larger rank: the previous run's r1 Ritz
// vectors, their values and couplings and the residual direction seed the
// new workspace as a thick restart keeping r1 vectors (the Krylov state is
// reused; only the new part of the space is built).  A previous run that
// spanned the whole space, broke down or did not converge starts afresh.
template <typename T>
static int continue_T(ssa_ctx* c, const ssa_params& p) {
  const Workspace w1 = c->ws;                 // pointers into the old arena (freed by alloc_ws)
  const LzState h1 = w1.host_st;
  // the rank rule holds whichever way the continuation is carried out
  if (p.rank <= w1.r || p.rank > std::min(c->L, c->K))
    return fail(SSA_ERANK, "continuation needs a rank in (%d, %lld]", w1.r, (long long)std::min(c->L, c->K));
  if (h1.full || h1.breakdown || !h1.converged || w1.prec != p.prec) {
    int32_t stv = 0;
    return decompose_batch_T<T>(&c, 1, &p, &stv);
  }
  const int r1 = w1.r, k1 = w1.k;
  const int64_t Ls = w1.Ls, Kl = w1.Kl;
  cudaStream_t st = c->stream;
  double *tU = nullptr, *tP = nullptr, *tsig = nullptr, *tcs = nullptr;
  T *tV = nullptr, *tv = nullptr;
  LzState* tst = nullptr;
  auto cleanup = [&]() {
    for (void* q : {(void*)tU, (void*)tP, (void*)tsig, (void*)tcs, (void*)tV, (void*)tv, (void*)tst})
      if (q) c->release(q);
  };
  int rc = c->allocT(&tU, (size_t)Ls * r1);
  if (rc == SSA_OK) rc = c->allocT(&tV, (size_t)Kl * r1);
  if (rc == SSA_OK) rc = c->allocT(&tv, (size_t)Kl);
  if (rc == SSA_OK) rc = c->allocT(&tP, (size_t)k1 * k1);
  if (rc == SSA_OK) rc = c->allocT(&tsig, (size_t)r1);
  if (rc == SSA_OK) rc = c->allocT(&tcs, 1);
  if (rc == SSA_OK) rc = c->allocT(&tst, 1);
  struct { void* d; const void* s; size_t n; } cp[] = {
      {tU, w1.U, sizeof(double) * Ls * r1}, {tV, w1.V, sizeof(T) * Kl * r1},
      {tv, (const T*)w1.V + Kl * k1, sizeof(T) * Kl}, {tP, w1.P, sizeof(double) * k1 * k1},
      {tsig, w1.sig, sizeof(double) * r1}, {tcs, w1.colscale + k1, sizeof(double)}, {tst, w1.st, sizeof(LzState)}};
  for (auto& q : cp)
    if (rc == SSA_OK && cudaMemcpyAsync(q.d, q.s, q.n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      rc = fail(SSA_ECUDA, "saving the previous Krylov state failed");
  ssa_ctx* cc = c;
  if (rc == SSA_OK) rc = ensure_spectra<T>(&cc, 1, st);
  if (rc == SSA_OK) rc = alloc_ws<T>(c, p, c->ws);
  Workspace& w2 = c->ws;
  if (rc == SSA_OK && w2.k <= r1) rc = fail(SSA_ERANK, "Krylov dimension %d leaves no room past %d kept vectors", w2.k, r1);
  struct { void* d; const void* s; size_t n; } cp2[] = {
      {w2.U, tU, sizeof(double) * Ls * r1}, {w2.V, tV, sizeof(T) * Kl * r1},
      {(T*)w2.V + Kl * r1, tv, sizeof(T) * Kl}};
  for (auto& q : cp2)
    if (rc == SSA_OK && cudaMemcpyAsync(q.d, q.s, q.n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      rc = fail(SSA_ECUDA, "seeding the new Krylov state failed");
  if (rc == SSA_OK) {
    k_state_resume<<<1, 256, 0, st>>>(w2.st, w2.B, w2.k, w2.colscale, tsig, tP, k1, tst, tcs, r1); count_launch();
    if (cudaGetLastError() != cudaSuccess) rc = fail(SSA_ECUDA, "resume launch failed");
  }
  cleanup();
  if (rc != SSA_OK) {
    c->ws.done = false;
    return rc;
  }
  LzEngine<T> e;
  e.st = st;
  e.device = c->device;
  e.add_resumed(c, r1);
  TRY(e.build());
  while (e.any_active()) {
    TRY(e.run_chunk());
  }
  std::vector<int> all{0};
  TRY(e.retire(all));
  CU(cudaStreamSynchronize(st));
  const LzState& h = e.hst[0];
  if (!h.converged) return fail(SSA_ENOTCONV, "restarts exhausted (max residual %.3g)", h.maxres);
  return SSA_OK;
}

// ============================================================== reconstruction
// Reconstruction arithmetic runs in TC (FP64 unless the grid is too long for
// an FP64 single-CTA pass); the decomposition's vectors are read as TV.
// One problem's reconstruction request: its grouping and output buffer.
struct RecReq {
  const int32_t* group_of;   // r entries (host)
  int ng;
  int residual;
  double* out;               // (ng + residual) x total, host or device
};

template <typename TC, typename TV>
static int reconstruct_T(ssa_ctx* const* cs, int n, const RecReq* req, int on_device, bool border = false) {
  typedef TC T;
  ssa_ctx* c0 = cs[0];
  cudaStream_t st = c0->stream;
  PhaseScope ps_(PH_RECON, st);
  // component lists of every (problem, group), flattened for one upload
  std::vector<int32_t> flat;
  std::vector<std::vector<int32_t>> start(n);
  for (int p = 0; p < n; ++p) {
    const int r = cs[p]->ws.r, ng = req[p].ng;
    std::vector<std::vector<int32_t>> comps(ng);
    for (int i = 0; i < r; ++i) {
      const int g = req[p].group_of[i];
      if (g < -1 || g >= ng) return fail(SSA_EINVAL, "group_of[%d] = %d out of range", i, g);
      if (g >= 0) comps[g].push_back(i);
    }
    start[p].assign(ng + 1, 0);
    for (int g = 0; g < ng; ++g) {
      start[p][g] = (int32_t)flat.size();
      flat.insert(flat.end(), comps[g].begin(), comps[g].end());
    }
    start[p][ng] = (int32_t)flat.size();
  }
  int32_t* d_flat = nullptr;
  TRY(upload(c0, flat, &d_flat));
  std::vector<void*> tmp;
  std::vector<double*> dout(n, nullptr);
  const Cx<T>* tw = twiddles<T>(c0->device);
  for (int p = 0; p < n; ++p) {
    const int nout = req[p].ng + (req[p].residual ? 1 : 0);
    if (on_device) dout[p] = req[p].out;
    else {
      TRY(c0->alloc((void**)&dout[p], sizeof(double) * (size_t)cs[p]->total * nout));
      tmp.push_back(dout[p]);
    }
  }
  // ---- series on one grid: F(U_i) once per problem and grid size (each
  // channel keeps its own M_q >= N_q: the group's convolution of U with the
  // channel's V slice has linear length N_q), then one CTA per (problem,
  // group, channel)
  {
    std::vector<RecColItem<T, TV>> ui;
    std::vector<Rec1Item<T, TV>> ri;
    int max_log2Mx = 1;
    for (int p = 0; p < n; ++p) {
      ssa_ctx* c = cs[p];
      if (c->log2My != 0) continue;
      Workspace& w = c->ws;
      const int r = w.r, ng = req[p].ng;
      double* o = dout[p];
      Cx<T>* gu_of[32] = {};
      for (const Channel& h : c->ch) {
        if (gu_of[h.log2M]) continue;
        const int H = 1 << (h.log2M - 1);
        Cx<T>* gu = nullptr;
        TRY(c0->alloc((void**)&gu, sizeof(Cx<T>) * (size_t)(H + 1) * r));
        tmp.push_back(gu);
        gu_of[h.log2M] = gu;
        for (int i = 0; i < r; ++i) {
          if (req[p].group_of[i] < 0) continue;      // component in no group
          RecColItem<T, TV> u;
          u.vec = (const TV*)w.Uo + (size_t)c->L * i; u.map = c->Lset.dev(); u.dst = gu + (size_t)(H + 1) * i;
          u.log2Mx = h.log2M; u.ncols = 1;
          ui.push_back(u);
        }
        max_log2Mx = std::max(max_log2Mx, h.log2M);
      }
      for (int g = 0; g < ng; ++g)
        for (size_t q = 0; q < c->ch.size(); ++q) {
          const Channel& h = c->ch[q];
          const int H = 1 << (h.log2M - 1);
          Rec1Item<T, TV> it;
          it.V = (const TV*)w.Vo + h.koff; it.ldv = c->K; it.map = h.K.dev();
          it.gu = gu_of[h.log2M]; it.ldgu = H + 1; it.sigma = w.sigma;
          it.comps = d_flat + start[p][g]; it.ncomp = start[p][g + 1] - start[p][g];
          it.log2Mx = h.log2M; it.w = h.w; it.n = (int32_t)h.nx;
          it.out = o + (size_t)g * c->total + h.data_off;
          it.inv_norm = 1.0 / (double)(2 * H);
          ri.push_back(it);
        }
    }
    if (!ui.empty()) {
      RecColItem<T, TV>* d_ui = nullptr; Rec1Item<T, TV>* d_ri = nullptr;
      TRY(upload(c0, ui, &d_ui));
      tmp.push_back(d_ui);
      launch_rec_col_fft<T, TV>(d_ui, (int)ui.size(), max_log2Mx, 1, tw, st);
      if (!ri.empty()) {
        TRY(upload(c0, ri, &d_ri));
        tmp.push_back(d_ri);
        launch_rec1d<T, TV>(d_ri, (int)ri.size(), max_log2Mx, tw, st);
      }
      if constexpr (std::is_same<TC, float>::value && std::is_same<TV, float>::value) {
        if (border) {
          // low-weight elements by direct FP64 sums (complete series only)
          std::vector<RecBorderItem> bi;
          for (int p = 0; p < n; ++p) {
            ssa_ctx* c = cs[p];
            if (c->log2My != 0) continue;
            Workspace& w = c->ws;
            for (int g = 0; g < req[p].ng; ++g)
              for (const Channel& h : c->ch) {
                RecBorderItem b;
                b.U = (const float*)w.Uo; b.V = (const float*)w.Vo + h.koff; b.ldv = c->K; b.sigma = w.sigma;
                b.comps = d_flat + start[p][g]; b.ncomp = start[p][g + 1] - start[p][g];
                b.L = (int32_t)c->L; b.K = (int32_t)h.K.count; b.pad_ = 0;
                b.out = dout[p] + (size_t)g * c->total + h.data_off;
                bi.push_back(b);
              }
          }
          if (!bi.empty()) {
            RecBorderItem* d_bi = nullptr;
            TRY(upload(c0, bi, &d_bi));
            tmp.push_back(d_bi);
            launch_rec_border(d_bi, (int)bi.size(), st);
          }
        }
      }
      CU(cudaGetLastError());
    }
  }
  // ---- grids with a y extent, one problem at a time: per component 2D
  // transforms accumulated per group in frequency space (Lemma hbh_tbt_elmat)
  for (int p = 0; p < n; ++p) {
    ssa_ctx* c = cs[p];
    if (c->log2My == 0) continue;
    Workspace& w = c->ws;
    const int r = w.r, ng = req[p].ng;
    if (ng == 0) continue;
    const int32_t* group_of = req[p].group_of;
    const int H = 1 << (c->log2Mx - 1), My = 1 << c->log2My;
    const size_t hs = (size_t)(H + 1) * My;
    double* o = dout[p];
    const bool fold = c->fold_B != 0;
    int fymax = 1;
    for (auto& h : c->ch) fymax = std::max(fymax, h.fy);
    Cx<T> *gx = nullptr, *gu = nullptr, *acc = nullptr, *g2 = nullptr;
    double* S = nullptr;
    TRY(c0->alloc((void**)&gx, sizeof(Cx<T>) * hs));
    TRY(c0->alloc((void**)&gu, sizeof(Cx<T>) * hs));
    TRY(c0->alloc((void**)&acc, sizeof(Cx<T>) * hs * ng));
    TRY(c0->alloc((void**)&g2, sizeof(Cx<T>) * hs));
    tmp.push_back(gx); tmp.push_back(gu); tmp.push_back(acc); tmp.push_back(g2);
    if (fold) {
      TRY(c0->alloc((void**)&S, sizeof(double) * (size_t)(2 * H) * fymax));
      tmp.push_back(S);
    }
    std::vector<double> sig(r);
    CU(cudaMemcpyAsync(sig.data(), w.sigma, sizeof(double) * r, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    // items: per (channel, component) two column transforms and two y-passes;
    // per (channel, group) the inverse y-pass, inverse x-pass and (segment
    // form) the overlap-add
    std::vector<RecColItem<T, TV>> allc;
    std::vector<YItem<T>> ally, yi;
    std::vector<Rec2Item<T>> xi;
    std::vector<RecFoldItem> fi;
    for (size_t q = 0; q < c->ch.size(); ++q) {
      const Channel& h = c->ch[q];
      const MapDev wl = fold ? fold_map(c->fold_B, c->lb, c->L) : c->Lset.dev();
      const MapDev ko = fold ? fold_map(c->fold_B, h.kb, h.K.count) : h.K.dev();
      const int wcols = fold ? c->lb : c->ey, kcols = fold ? h.kb : h.cy;
      for (int i = 0; i < r; ++i) {
        const int g = group_of[i];
        RecColItem<T, TV> a;
        a.vec = (const TV*)w.Uo + (size_t)c->L * i; a.map = wl; a.dst = gx; a.log2Mx = c->log2Mx;
        a.ncols = wcols;
        RecColItem<T, TV> b;
        b.vec = (const TV*)w.Vo + (size_t)c->K * i + h.koff; b.map = ko; b.dst = gx; b.log2Mx = c->log2Mx;
        b.ncols = kcols;
        YItem<T> ya;
        ya.src = gx; ya.dst = gu; ya.mul = nullptr; ya.st = nullptr; ya.log2Mx = c->log2Mx; ya.log2My = c->log2My;
        ya.in_hi = wcols; ya.out_hi = My; ya.scale = T(0);
        ya.tk = tuned_ytk<T>(c->log2Mx, c->log2My);
        YItem<T> yb = ya;
        yb.dst = acc + (size_t)std::max(g, 0) * hs; yb.mul = gu; yb.in_hi = kcols;
        yb.scale = (T)(sig[i] / ((double)(2 * H) * (double)My));
        allc.push_back(a); allc.push_back(b);
        ally.push_back(ya); ally.push_back(yb);
      }
      const int oy = fold ? h.fy : (int)h.ny;
      for (int g = 0; g < ng; ++g) {
        YItem<T> y;
        y.src = acc + (size_t)g * hs; y.dst = g2; y.mul = nullptr; y.st = nullptr;
        y.log2Mx = c->log2Mx; y.log2My = c->log2My; y.in_hi = My; y.out_hi = oy; y.scale = T(0);
        y.tk = tuned_ytk<T>(c->log2Mx, c->log2My);
        yi.push_back(y);
        Rec2Item<T> x;
        x.g2 = g2; x.log2Mx = c->log2Mx; x.pad_ = 0; x.inv_norm = 1.0;
        if (fold) {
          x.w = nullptr; x.out = S; x.nx = 2 * H; x.ny = h.fy;
          fi.push_back({S, h.w, o + (size_t)g * c->total + h.data_off, (int64_t)c->fold_B, h.nx, (int64_t)h.fy});
        } else {
          x.w = h.w; x.out = o + (size_t)g * c->total + h.data_off; x.nx = (int)h.nx; x.ny = (int)h.ny;
        }
        xi.push_back(x);
      }
    }
    RecColItem<T, TV>* d_cu = nullptr; YItem<T>* d_yu = nullptr; YItem<T>* d_yi = nullptr;
    Rec2Item<T>* d_xi = nullptr; RecFoldItem* d_fi = nullptr;
    TRY(upload(c0, allc, &d_cu)); tmp.push_back(d_cu);
    TRY(upload(c0, ally, &d_yu)); tmp.push_back(d_yu);
    TRY(upload(c0, yi, &d_yi)); tmp.push_back(d_yi);
    TRY(upload(c0, xi, &d_xi)); tmp.push_back(d_xi);
    if (fold) { TRY(upload(c0, fi, &d_fi)); tmp.push_back(d_fi); }
    const int rtk = tuned_ytk<T>(c->log2Mx, c->log2My);
    const int rbuf = rtk * padded_len(1 << c->log2My);   // staging elements of that tile width
    const Tiles y1{nullptr, 1, ypass_blocks(c->log2Mx, rtk)};
    for (size_t q = 0; q < c->ch.size(); ++q) {
      const Channel& h = c->ch[q];
      const int wcols = fold ? c->lb : c->ey, kcols = fold ? h.kb : h.cy;
      CU(cudaMemsetAsync(acc, 0, sizeof(Cx<T>) * hs * ng, st));
      for (int i = 0; i < r; ++i) {
        if (group_of[i] < 0) continue;
        const size_t e = 2 * ((size_t)q * r + i);
        launch_rec_col_fft<T, TV>(d_cu + e, 1, c->log2Mx, wcols, tw, st);
        launch_ypass<T>(d_yu + e, y1, Y_FWD, c->log2My, -1, tw, st, rbuf);
        launch_rec_col_fft<T, TV>(d_cu + e + 1, 1, c->log2Mx, kcols, tw, st);
        launch_ypass<T>(d_yu + e + 1, y1, Y_CONVACC, c->log2My, -1, tw, st, rbuf);
      }
      for (int g = 0; g < ng; ++g) {
        const size_t e = (size_t)q * ng + g;
        launch_ypass<T>(d_yi + e, y1, Y_INV, c->log2My, -1, tw, st, rbuf);
        launch_rec_xinv<T>(d_xi + e, 1, c->log2Mx, xi[e].ny, tw, st);
        if (fold) launch_rec_fold(d_fi + e, 1, h.nx, st);
      }
      CU(cudaGetLastError());
    }
  }
  // residual (one launch for every channel of every problem) and copy-out
  {
    std::vector<ResItem> ri;
    int64_t max_n = 1;
    for (int p = 0; p < n; ++p) {
      ssa_ctx* c = cs[p];
      if (!req[p].residual) continue;
      const int ng = req[p].ng;
      const size_t esz = c->dtype == SSA_F64 ? 8 : 4;
      for (size_t q = 0; q < c->ch.size(); ++q) {
        const Channel& h = c->ch[q];
        ri.push_back({(const char*)c->data + h.data_off * esz, c->dtype == SSA_F64, ng, h.w,
                      dout[p] + h.data_off, c->total, h.nx * h.ny, dout[p] + (size_t)ng * c->total + h.data_off});
        max_n = std::max<int64_t>(max_n, h.nx * h.ny);
      }
    }
    if (!ri.empty()) {
      ResItem* d_ri = nullptr;
      TRY(upload(c0, ri, &d_ri));
      tmp.push_back(d_ri);
      launch_residual_batch(d_ri, (int)ri.size(), max_n, st);
      CU(cudaGetLastError());
    }
  }
  for (int p = 0; p < n; ++p) {
    ssa_ctx* c = cs[p];
    const int nout = req[p].ng + (req[p].residual ? 1 : 0);
    if (!on_device)
      CU(cudaMemcpyAsync(req[p].out, dout[p], sizeof(double) * (size_t)c->total * nout, cudaMemcpyDeviceToHost, st));
  }
  CU(cudaStreamSynchronize(st));
  for (void* t : tmp) c0->release(t);
  c0->release(d_flat);
  if (ypass_bad_tiles(st) != 0) return fail(SSA_ECUDA, "a y-pass tile did not fit its launch's buffers");
  return SSA_OK;
}

template <typename T>
static int matvec_T(ssa_ctx* c, int transpose, const double* in, double* out, int on_device) {
  TRY(ensure_spectrum<T>(c));
  const int64_t nin = transpose ? c->L : c->K, nout = transpose ? c->K : c->L;
  const int nch = (int)c->ch.size();
  T *din = nullptr, *dparts = nullptr;
  double *dd = nullptr, *dres = nullptr;
  TRY(c->alloc((void**)&din, sizeof(T) * nin));
  const int nparts = transpose ? 1 : nch;
  TRY(c->alloc((void**)&dparts, sizeof(T) * (size_t)nout * nparts));
  if (on_device) { dd = const_cast<double*>(in); dres = out; }
  else {
    TRY(c->allocT(&dd, (size_t)nin));
    TRY(c->allocT(&dres, (size_t)nout));
    CU(cudaMemcpyAsync(dd, in, sizeof(double) * nin, cudaMemcpyHostToDevice, c->stream));
  }
  k_convert<T, double><<<grid1(nin), 256, 0, c->stream>>>(dd, din, nin); count_launch();
  CU(cudaGetLastError());
  void *g1 = nullptr, *g2 = nullptr;
  const size_t hs = c->log2My > 0 ? ((size_t)((1 << (c->log2Mx - 1)) + 1) << c->log2My) : 0;
  if (hs) { TRY(c->alloc(&g1, sizeof(Cx<T>) * hs * nch)); TRY(c->alloc(&g2, sizeof(Cx<T>) * hs * nch)); }
  MvSet<T> s;
  for (int q = 0; q < nch; ++q) {
    const Channel& h = c->ch[q];
    VecRef vi{}, vo{};
    vi.base = din; vi.off = transpose ? 0 : h.koff; vi.ld = 0; vi.st = nullptr;
    vo.base = dparts; vo.off = transpose ? h.koff : (int64_t)q * nout; vo.ld = 0; vo.st = nullptr;
    s.add(make_mv<T>(c, h, transpose != 0, vi, 0, vo, hs ? (Cx<T>*)g1 + q * hs : nullptr,
                     hs ? (Cx<T>*)g2 + q * hs : nullptr, nullptr));
  }
  TRY(finish_set(s, [&](auto& v, auto** d) { return upload(c, v, d); }));
  run_mv<T>(c->device, s, 0, c->stream);
  k_sum_parts_to_double<T><<<grid1(nout), 256, 0, c->stream>>>(dparts, nparts, nout, nout, dres); count_launch();
  CU(cudaGetLastError());
  if (!on_device) CU(cudaMemcpyAsync(out, dres, sizeof(double) * nout, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  if (s.n1() && mv_async_timeouts(c->stream) != 0)
    return fail(SSA_ETIMEOUT, "a bulk copy of a data spectrum did not complete");
  c->release(din); c->release(dparts);
  if (!on_device) { c->release(dd); c->release(dres); }
  if (g1) { c->release(g1); c->release(g2); }
  for (auto* d : s.d1)
    if (d) c->release(d);
  if (s.d2) {
    c->release(s.d2); c->release(s.dy2);
    c->release(s.t_xf); c->release(s.t_yp); c->release(s.t_xi);
  }
  return SSA_OK;
}

static int embed_prepare(const ssa_input* in, const ssa_window* win, void* cuda_stream, ssa_ctx** out) {
  if (!in || !win || !out || !in->data) return fail(SSA_EINVAL, "null argument");
  *out = nullptr;
  if (in->dtype != SSA_F32 && in->dtype != SSA_F64) return fail(SSA_EINVAL, "dtype must be SSA_F32 or SSA_F64");
  ssa_ctx* c = new ssa_ctx();
  auto bail = [&](int rc) { ssa_destroy(c); return rc; };
  CU(cudaGetDevice(&c->device));
  if (ensure_tables(c->device) != SSA_OK) return bail(SSA_ECUDA);
  c->kind = in->kind;
  c->dtype = in->dtype;
  if (cuda_stream) c->stream = (cudaStream_t)cuda_stream;
  else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
      return bail(fail(SSA_ECUDA, "stream creation failed"));
    c->own_stream = true;
  }
  // channel geometry
  if (in->kind == SSA_1D) {
    if (in->n < 2) return bail(fail(SSA_EINVAL, "series length %lld < 2", (long long)in->n));
    if (win->L < 2 || win->L >= in->n) return bail(fail(SSA_EINVAL, "window L=%lld must satisfy 1 < L < N=%lld", (long long)win->L, (long long)in->n));
    Channel h; h.nx = in->n; h.ny = 1; h.data_off = 0;
    c->ch.push_back(h);
    c->total = in->n;
  } else if (in->kind == SSA_MSSA) {
    if (in->n_series < 1 || !in->lengths) return bail(fail(SSA_EINVAL, "MSSA needs n_series >= 1 and lengths"));
    int64_t off = 0, mn = INT64_MAX;
    for (int q = 0; q < in->n_series; ++q) {
      Channel h; h.nx = in->lengths[q]; h.ny = 1; h.data_off = off;
      if (h.nx < 2) return bail(fail(SSA_EINVAL, "series %d has length %lld", q, (long long)h.nx));
      off += h.nx; mn = std::min(mn, h.nx);
      c->ch.push_back(h);
    }
    if (win->L < 2 || win->L >= mn) return bail(fail(SSA_EINVAL, "window L=%lld must satisfy 1 < L < min N_p=%lld", (long long)win->L, (long long)mn));
    c->total = off;
  } else if (in->kind == SSA_2D) {
    if (in->nx < 1 || in->ny < 1) return bail(fail(SSA_EINVAL, "image size"));
    if (win->lx < 1 || win->ly < 1 || win->lx > in->nx || win->ly > in->ny || win->lx * win->ly <= 1 ||
        win->lx * win->ly >= in->nx * in->ny)
      return bail(fail(SSA_EINVAL, "window %lldx%lld must satisfy 1<=lx<=nx, 1<=ly<=ny, 1<lx*ly<nx*ny",
                       (long long)win->lx, (long long)win->ly));
    Channel h; h.nx = in->nx; h.ny = in->ny; h.data_off = 0;
    c->ch.push_back(h);
    c->total = in->nx * in->ny;
  } else {
    return bail(fail(SSA_EINVAL, "unknown kind %d", in->kind));
  }
  int64_t mx = 0, my = 0;
  for (auto& h : c->ch) { mx = std::max(mx, h.nx); my = std::max(my, h.ny); }
  c->log2Mx = std::max(ilog2_ceil(mx), 4);
  c->log2My = (in->kind == SSA_2D) ? ilog2_ceil(my) : 0;
  if (in->kind != SSA_2D && c->log2Mx >= FOLD_MIN_LOG2) {
    // long series: segment form on a 2B x My grid (every channel of the system)
    std::vector<int64_t> ns;
    for (auto& h : c->ch) ns.push_back(h.nx);
    const FoldGeom g = fold_geometry(ns, win->L);
    c->fold_B = g.B;
    c->lb = g.lb;
    c->log2Mx = ilog2_ceil(2 * (int64_t)g.B);
    c->log2My = g.log2My;
    for (size_t q = 0; q < c->ch.size(); ++q) {
      c->ch[q].kb = g.kb[q];
      c->ch[q].fy = g.fy[q];
      c->ch[q].log2M = c->log2Mx;
    }
  } else {
    if (c->log2Mx > 14) return bail(fail(SSA_EUNSUPPORTED, "FFT length %lld along x exceeds 16384", (long long)(1ll << c->log2Mx)));
    // series of a system each get the shortest grid that holds them (any
    // M >= N_p gives the same product); images keep the common grid
    for (auto& h : c->ch) h.log2M = (in->kind == SSA_2D) ? c->log2Mx : std::max(ilog2_ceil(h.nx), 4);
  }
  if (c->log2My > 12) return bail(fail(SSA_EUNSUPPORTED, "FFT length %lld along y exceeds 4096", (long long)(1ll << c->log2My)));
  // data (and mask) to the device; masked samples become NaN in the device copy
  const size_t esz = in->dtype == SSA_F64 ? 8 : 4;
  {
    // one arena for everything the embedding keeps (sizes from the geometry)
    const size_t lx = in->kind == SSA_2D ? (size_t)win->lx : (size_t)win->L;
    const size_t ly = in->kind == SSA_2D ? (size_t)win->ly : 1;
    const size_t ww = (lx + 31) / 32;
    size_t need = rnd256(esz * c->total) + (in->mask ? rnd256(c->total) : 0) + 2 * rnd256(ly * ww * 4) +
                  2 * rnd256((ly + 1) * 4) + rnd256(4) + rnd256(2 * ly * 4);
    size_t nsq = 0;
    for (auto& h : c->ch) {
      const size_t nw = (h.nx + 31) / 32;
      const size_t cy = h.ny, kw = nw;
      need += rnd256(h.ny * nw * 4) * 2 + rnd256(cy * kw * 4) + 2 * rnd256((cy + 1) * 4) + rnd256(h.nx * h.ny * 4) +
              rnd256(h.ny * (nw + 1) * 4) + rnd256(cy * (kw + 1) * 4);
      nsq += (size_t)((h.nx + 255) >> 8) * h.ny;
    }
    need += rnd256(8 * nsq) + rnd256(8);
    int rc0 = c->make_arena(c->embed_arena, need);
    if (rc0) return bail(rc0);
    c->cur = &c->embed_arena;
  }
  int rc = c->alloc(&c->data, esz * (size_t)c->total);
  if (rc) return bail(rc);
  if (cudaMemcpyAsync(c->data, in->data, esz * c->total, in->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                      c->stream) != cudaSuccess)
    return bail(fail(SSA_ECUDA, "input copy failed"));
  if (in->mask) {
    uint8_t* dm = nullptr;
    rc = c->allocT(&dm, (size_t)c->total);
    if (rc) return bail(rc);
    if (cudaMemcpyAsync(dm, in->mask, (size_t)c->total, in->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        c->stream) != cudaSuccess)
      return bail(fail(SSA_ECUDA, "mask copy failed"));
    // fold the mask into the data as NaN so the observed set is one test
    extern void launch_apply_mask(void*, int, const uint8_t*, int64_t, cudaStream_t);
    launch_apply_mask(c->data, in->dtype == SSA_F64, dm, c->total, c->stream);
    c->release(dm);
  }
  *out = c;
  return SSA_OK;
}


// precision of the reconstruction sums: FP64 unless one FP64 pass would not
// fit a CTA (x grids above 8192)
static int reconstruct_dispatch(ssa_ctx* const* ctxs, int n, const RecReq* req, int on_device) {
  const int prec = ctxs[0]->ws.prec;
  if (prec == SSA_PREC_FP64) return reconstruct_T<double, double>(ctxs, n, req, on_device);
  // FP32 form: complete series (dense origins, L and every K_q at least
  // REC_BORDER_W) take FP32 FFT sums plus direct FP64 sums where the weight
  // is small; the rest FP64 FFT sums where the grid allows it.
  std::vector<ssa_ctx*> fc, sc;
  std::vector<RecReq> fr, sr;
  int max_log2Mx = 0;
  for (int i = 0; i < n; ++i) {
    ssa_ctx* c = ctxs[i];
    bool fast = c->log2My == 0 && c->log2Mx <= 14 && c->L >= REC_BORDER_W;
    for (const Channel& h : c->ch) fast = fast && h.K.dense && h.K.count >= REC_BORDER_W;
    if (fast) { fc.push_back(c); fr.push_back(req[i]); }
    else { sc.push_back(c); sr.push_back(req[i]); max_log2Mx = std::max(max_log2Mx, c->log2Mx); }
  }
  if (!fc.empty()) {
    const int rc = reconstruct_T<float, float>(fc.data(), (int)fc.size(), fr.data(), on_device, true);
    if (rc != SSA_OK) return rc;
  }
  if (sc.empty()) return SSA_OK;
  if (max_log2Mx <= 13) return reconstruct_T<double, float>(sc.data(), (int)sc.size(), sr.data(), on_device);
  return reconstruct_T<float, float>(sc.data(), (int)sc.size(), sr.data(), on_device);
}

// ============================================================== C ABI
extern "C" {

const char* ssa_version(void) { return "ssa-gb300 0.1 (sm_103a)"; }

const char* ssa_strerror(int code) {
  switch (code) {
    case SSA_OK: return "ok";
    case SSA_EINVAL: return "invalid argument";
    case SSA_EEMPTY: return "empty origin set";
    case SSA_ERANK: return "rank out of range";
    case SSA_ENOMEM: return "out of device memory";
    case SSA_ENOTCONV: return "not converged";
    case SSA_ETIMEOUT: return "timeout";
    case SSA_ECUDA: return "CUDA error";
    case SSA_ESTATE: return "call out of order";
    case SSA_EUNSUPPORTED: return "unsupported size";
  }
  return "unknown error";
}

const char* ssa_last_error(void) { return g_err; }

int ssa_profile_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  g_prof.on = on != 0;
  return SSA_OK;
}

int ssa_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  g_prof.resolve();
  for (int i = 0; i < PH_COUNT; ++i) { g_prof.ms[i] = 0.0; g_prof.launches[i] = 0; g_prof.calls[i] = 0; }
  return SSA_OK;
}

int ssa_profile_read(int32_t phase, double* ms, int64_t* launches, int64_t* calls) {
  if (phase < 0 || phase >= PH_COUNT) return fail(SSA_EINVAL, "phase %d", phase);
  std::lock_guard<std::mutex> lk(g_prof.mu);
  g_prof.resolve();
  if (ms) *ms = g_prof.ms[phase];
  if (launches) *launches = g_prof.launches[phase];
  if (calls) *calls = g_prof.calls[phase];
  return SSA_OK;
}

int64_t ssa_kernel_launches(void) { return (int64_t)g_launches.load(); }

int ssa_embed_batch(const ssa_input* ins, const ssa_window* wins, int32_t n, void* cuda_stream, ssa_ctx** outs,
                    int32_t* status) {
  if (!ins || !wins || !outs || n < 1) return fail(SSA_EINVAL, "null argument");
  // one stream for the whole batch: the caller's, or one shared per host thread
  static thread_local cudaStream_t own = nullptr;
  void* bs = cuda_stream;
  if (!bs && n > 1) {
    if (!own && cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking) != cudaSuccess)
      return fail(SSA_ECUDA, "stream creation failed");
    bs = (void*)own;
  }
  std::vector<int> rc(n, SSA_OK);
  for (int i = 0; i < n; ++i) {
    outs[i] = nullptr;
    rc[i] = embed_prepare(&ins[i], &wins[i], bs, &outs[i]);
  }
  cudaStream_t st = nullptr;
  for (int i = 0; i < n; ++i)
    if (outs[i]) { st = outs[i]->stream; break; }
  int first = SSA_OK;
  auto finish = [&]() {
    for (int i = 0; i < n; ++i) {
      if (rc[i] != SSA_OK) {
        if (outs[i]) ssa_destroy(outs[i]);
        outs[i] = nullptr;
        if (first == SSA_OK) first = rc[i];
      }
      if (status) status[i] = rc[i];
    }
    return first;
  };
  if (!st) return finish();
  // batch scratch: totals and error flags (device) + pinned mirrors
  size_t ncount = 0;
  for (int i = 0; i < n; ++i)
    if (outs[i]) ncount += outs[i]->ch.size() + 1;
  int32_t* d_tot = nullptr;
  int* d_err = nullptr;
  if (cudaMallocAsync((void**)&d_tot, sizeof(int32_t) * (ncount + 1), st) != cudaSuccess ||
      cudaMallocAsync((void**)&d_err, sizeof(int) * n, st) != cudaSuccess)
    return fail(SSA_ENOMEM, "embed scratch");
  cudaMemsetAsync(d_err, 0, sizeof(int) * n, st);
  int32_t* pin = pinned_slots(ncount + n + 1);
  if (!pin) return fail(SSA_ENOMEM, "pinned staging allocation failed");
  EmbedBatch eb;
  eb.cnt_slot_L.assign(n, -1);
  eb.cnt_slot_K.resize(n);
  PhaseScope ps_(PH_SHAPES, st);
  for (int i = 0; i < n; ++i)
    if (rc[i] == SSA_OK) rc[i] = embed_stage1(outs[i], &wins[i], eb, i, d_tot, d_err);
  ObsItem* d_obs = nullptr; OriginItem* d_org = nullptr; CountItem* d_cnt = nullptr; WeightItem* d_wts = nullptr;
  NormItem* d_nrm = nullptr;
  auto upload_raw = [&](auto& vec, auto** dptr) -> int {
    typedef typename std::remove_reference<decltype(vec[0])>::type X;
    if (cudaMallocAsync((void**)dptr, sizeof(X) * std::max<size_t>(vec.size(), 1), st) != cudaSuccess) return SSA_ENOMEM;
    if (!vec.empty() && g_ring.copy(*dptr, vec.data(), sizeof(X) * vec.size(), st) != SSA_OK) return SSA_ECUDA;
    return SSA_OK;
  };
  PrefixItem *d_opre = nullptr, *d_kpre = nullptr;
  // block ranges of every item in each batched launch
  std::vector<int32_t> t_obs{0}, t_org{0}, t_cnt{0}, t_opre{0}, t_kpre{0}, t_wts{0};
  for (auto& o : eb.obs) t_obs.push_back(t_obs.back() + ((o.nx + 255) >> 8) * o.ny);
  for (auto& o : eb.org) t_org.push_back(t_org.back() + ((o.cx + 255) >> 8) * o.cy);
  for (auto& o : eb.cnt) t_cnt.push_back(t_cnt.back() + o.ncols);
  for (auto& o : eb.opre) t_opre.push_back(t_opre.back() + o.ncols);
  for (auto& o : eb.kpre) t_kpre.push_back(t_kpre.back() + o.ncols);
  int32_t *p_obs = nullptr, *p_org = nullptr, *p_cnt = nullptr, *p_opre = nullptr, *p_kpre = nullptr, *p_wts = nullptr;
  int urc = upload_raw(eb.obs, &d_obs);
  if (urc == SSA_OK) urc = upload_raw(eb.org, &d_org);
  if (urc == SSA_OK) urc = upload_raw(eb.cnt, &d_cnt);
  if (urc == SSA_OK) urc = upload_raw(eb.opre, &d_opre);
  if (urc == SSA_OK) urc = upload_raw(eb.kpre, &d_kpre);
  if (urc == SSA_OK) urc = upload_raw(t_obs, &p_obs);
  if (urc == SSA_OK) urc = upload_raw(t_org, &p_org);
  if (urc == SSA_OK) urc = upload_raw(t_cnt, &p_cnt);
  if (urc == SSA_OK) urc = upload_raw(t_opre, &p_opre);
  if (urc == SSA_OK) urc = upload_raw(t_kpre, &p_kpre);
  if (urc == SSA_OK) urc = upload_raw(eb.norms, &d_nrm);
  if (urc != SSA_OK) return fail(urc, "embed item upload");
  launch_obs_batch(d_obs, p_obs, (int)eb.obs.size(), t_obs.back(), st);
  launch_norm_batch(d_nrm, (int)eb.norms.size(), st);
  launch_prefix_batch(d_opre, p_opre, (int)eb.opre.size(), t_opre.back(), st);
  launch_origins_batch(d_org, p_org, (int)eb.org.size(), t_org.back(), st);
  launch_prefix_batch(d_kpre, p_kpre, (int)eb.kpre.size(), t_kpre.back(), st);
  launch_counts_batch(d_cnt, p_cnt, (int)eb.cnt.size(), t_cnt.back(), st);
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(pin, d_tot, sizeof(int32_t) * std::max<size_t>(ncount, 1), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  std::vector<int32_t> totals(pin, pin + ncount);
  for (int i = 0; i < n; ++i)
    if (rc[i] == SSA_OK) rc[i] = embed_stage2(outs[i], eb, i, totals.data());
  for (auto& o : eb.wts) t_wts.push_back(t_wts.back() + ((o.nx + 255) >> 8) * o.ny);
  urc = upload_raw(eb.wts, &d_wts);
  if (urc == SSA_OK) urc = upload_raw(t_wts, &p_wts);
  if (urc != SSA_OK) return fail(urc, "embed item upload");
  launch_weights_batch(d_wts, p_wts, (int)eb.wts.size(), t_wts.back(), st);
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(pin, d_err, sizeof(int) * n, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  for (int i = 0; i < n; ++i)
    if (rc[i] == SSA_OK) rc[i] = embed_stage3(outs[i], pin[i]);
  cudaFreeAsync(d_tot, st); cudaFreeAsync(d_err, st);
  cudaFreeAsync(d_obs, st); cudaFreeAsync(d_org, st); cudaFreeAsync(d_cnt, st); cudaFreeAsync(d_wts, st);
  cudaFreeAsync(d_opre, st); cudaFreeAsync(d_kpre, st); cudaFreeAsync(d_nrm, st);
  for (int32_t* q : {p_obs, p_org, p_cnt, p_opre, p_kpre, p_wts}) cudaFreeAsync(q, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(SSA_ECUDA, "embed: %s", cudaGetErrorString(e));
  return finish();
}

int ssa_embed(const ssa_input* in, const ssa_window* win, void* cuda_stream, ssa_ctx** out) {
  if (!out) return fail(SSA_EINVAL, "null argument");
  int32_t st = 0;
  return ssa_embed_batch(in, win, 1, cuda_stream, out, &st);
}

int ssa_decompose_batch(ssa_ctx* const* ctxs, int32_t n, const ssa_params* params, int32_t* status) {
  if (!ctxs || n < 1 || !params) return fail(SSA_EINVAL, "null argument");
  const int prec = params[0].prec;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return fail(SSA_EINVAL, "null context %d", i);
    if (params[i].prec != prec) return fail(SSA_EINVAL, "one precision form per batch");
    if (params[i].prec == SSA_PREC_FP64 && ctxs[i]->log2Mx > 13)
      return fail(SSA_EUNSUPPORTED, "FP64 form supports FFT length <= 8192 along x");
  }
  if (prec == SSA_PREC_FP64) return decompose_batch_T<double>(ctxs, n, params, status);
  if (prec == SSA_PREC_FP32FFT_FP64REORTH) return decompose_batch_T<float>(ctxs, n, params, status);
  return fail(SSA_EINVAL, "unknown precision %d", prec);
}

int ssa_decompose(ssa_ctx* ctx, const ssa_params* params) {
  int32_t st = 0;
  return ssa_decompose_batch(&ctx, 1, params, &st);
}

int ssa_continue(ssa_ctx* ctx, const ssa_params* params) {
  if (!ctx || !params) return fail(SSA_EINVAL, "null argument");
  if (!ctx->ws.done) return fail(SSA_ESTATE, "context has no decomposition to continue");
  if (params->prec == SSA_PREC_FP64 && ctx->log2Mx > 13)
    return fail(SSA_EUNSUPPORTED, "FP64 form supports FFT length <= 8192 along x");
  if (params->prec == SSA_PREC_FP64) return continue_T<double>(ctx, *params);
  if (params->prec == SSA_PREC_FP32FFT_FP64REORTH) return continue_T<float>(ctx, *params);
  return fail(SSA_EINVAL, "unknown precision %d", params->prec);
}

int ssa_get_info(const ssa_ctx* c, ssa_info* info) {
  if (!c || !info) return fail(SSA_EINVAL, "null argument");
  std::memset(info, 0, sizeof(*info));
  info->L = c->L; info->K = c->K;
  info->nx = c->ch[0].nx; info->ny = c->ch[0].ny;
  info->n_channels = (int32_t)c->ch.size();
  info->fft_mx = 1ll << c->log2Mx; info->fft_my = 1ll << c->log2My;
  info->device_bytes = c->bytes;
  if (c->ws.done) {
    info->rank = c->ws.r; info->krylov_dim = c->ws.k; info->restarts = c->ws.host_st.restarts;
    info->converged = c->ws.host_st.converged; info->prec = c->ws.prec;
    info->breakdowns = c->ws.host_st.breakdown;
    info->max_residual = c->ws.host_st.maxres;
    info->jacobi_sweeps = c->ws.host_st.sweeps;
    info->jacobi_sweeps_fp32 = c->ws.host_st.sweeps32;
  }
  return SSA_OK;
}

int ssa_get_sigma(const ssa_ctx* c, double* sigma, int32_t r) {
  if (!c || !sigma) return fail(SSA_EINVAL, "null argument");
  if (!c->ws.done) return fail(SSA_ESTATE, "no decomposition yet");
  if (r < 0 || r > c->ws.r) return fail(SSA_EINVAL, "r=%d exceeds the decomposed rank %d", r, c->ws.r);
  CU(cudaMemcpyAsync(sigma, c->ws.sigma, sizeof(double) * r, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return SSA_OK;
}

int ssa_get_vectors(const ssa_ctx* cc, double* U, double* V, int32_t on_device) {
  ssa_ctx* c = const_cast<ssa_ctx*>(cc);
  if (!c) return fail(SSA_EINVAL, "null argument");
  if (!c->ws.done) return fail(SSA_ESTATE, "no decomposition yet");
  const Workspace& w = c->ws;
  struct { double* dst; const void* src; int64_t n; } jobs[2] = {{U, w.Uo, c->L * w.r}, {V, w.Vo, c->K * w.r}};
  for (auto& j : jobs) {
    if (!j.dst) continue;
    double* d = j.dst;
    if (!on_device) TRY(c->allocT(&d, (size_t)j.n));
    if (w.prec == SSA_PREC_FP64)
      CU(cudaMemcpyAsync(d, j.src, sizeof(double) * j.n, cudaMemcpyDeviceToDevice, c->stream));
    else
      k_convert<double, float><<<grid1(j.n), 256, 0, c->stream>>>((const float*)j.src, d, j.n); count_launch();
    CU(cudaGetLastError());
    if (!on_device) {
      CU(cudaMemcpyAsync(j.dst, d, sizeof(double) * j.n, cudaMemcpyDeviceToHost, c->stream));
      CU(cudaStreamSynchronize(c->stream));
      c->release(d);
    }
  }
  CU(cudaStreamSynchronize(c->stream));
  return SSA_OK;
}

int ssa_reconstruct_batch(ssa_ctx* const* ctxs, int32_t n, const int32_t* group_of, int32_t n_groups,
                          int32_t residual, double* const* outs, int32_t on_device) {
  if (!ctxs || n < 1 || !group_of || !outs || n_groups < 0) return fail(SSA_EINVAL, "null argument");
  const int prec = ctxs[0]->ws.prec;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i] || !ctxs[i]->ws.done) return fail(SSA_ESTATE, "context %d has no decomposition", i);
    if (ctxs[i]->ws.prec != prec || ctxs[i]->ws.r != ctxs[0]->ws.r) return fail(SSA_EINVAL, "batch mixes precision or rank");
    if (!outs[i]) return fail(SSA_EINVAL, "null output %d", i);
  }
  if (n_groups + (residual ? 1 : 0) == 0) return SSA_OK;
  std::vector<RecReq> req(n);
  for (int i = 0; i < n; ++i) req[i] = {group_of, n_groups, residual, outs[i]};
  return reconstruct_dispatch(ctxs, n, req.data(), on_device);
}

int ssa_reconstruct(ssa_ctx* ctx, const int32_t* group_of, int32_t n_groups, int32_t residual, double* out,
                    int32_t on_device) {
  return ssa_reconstruct_batch(&ctx, 1, group_of, n_groups, residual, &out, on_device);
}

int ssa_wcor(ssa_ctx* ctx, const int32_t* group_of, int32_t n_groups, double* wcor, double* contrib) {
  if (!ctx || !group_of || !wcor) return fail(SSA_EINVAL, "null argument");
  if (!ctx->ws.done) return fail(SSA_ESTATE, "context has no decomposition");
  if (n_groups < 1 || n_groups > WCOR_MAX) return fail(SSA_EINVAL, "n_groups %d outside [1, %d]", n_groups, WCOR_MAX);
  ssa_ctx* c = ctx;
  const int n = n_groups, m = n + 1;
  const int64_t total = c->total;
  double* Y = nullptr;
  int32_t* w = nullptr;
  int2* pairs = nullptr;
  double* partials = nullptr;
  double* G = nullptr;
  double* res = nullptr;
  auto cleanup = [&]() {
    for (void* q : {(void*)Y, (void*)w, (void*)pairs, (void*)partials, (void*)G, (void*)res})
      if (q) c->release(q);
  };
  int rc = c->allocT(&Y, (size_t)n * total);
  if (rc == SSA_OK) rc = ssa_reconstruct_batch(&c, 1, group_of, n_groups, 0, &Y, 1);
  if (rc == SSA_OK) rc = c->allocT(&w, (size_t)total);
  if (rc == SSA_OK)
    for (auto& h : c->ch)
      if (cudaMemcpyAsync(w + h.data_off, h.w, sizeof(int32_t) * h.nx * h.ny, cudaMemcpyDeviceToDevice, c->stream) !=
          cudaSuccess) {
        rc = fail(SSA_ECUDA, "weights copy failed");
        break;
      }
  std::vector<int2> hp;
  for (int i = 0; i < m; ++i)
    for (int j = i; j < m; ++j) hp.push_back(make_int2(i, j));
  const int npair = (int)hp.size();
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>((total + WGRAM_CH - 1) / WGRAM_CH, std::max(sms, 1)));
  if (rc == SSA_OK) rc = upload(c, hp, &pairs);
  if (rc == SSA_OK) rc = c->allocT(&partials, (size_t)nblk * npair);
  if (rc == SSA_OK) rc = c->allocT(&G, (size_t)m * m);
  if (rc == SSA_OK) rc = c->allocT(&res, (size_t)n * n + n);
  if (rc == SSA_OK) {
    launch_wgram(Y, total, n, c->data, c->dtype == SSA_F64 ? 1 : 0, w, total, pairs, npair, partials, nblk, c->stream);
    launch_wcor_final(partials, nblk, pairs, npair, n, G, res, res + (size_t)n * n, c->stream);
    if (cudaGetLastError() != cudaSuccess) rc = fail(SSA_ECUDA, "w-correlation launch failed");
  }
  if (rc == SSA_OK && cudaMemcpyAsync(wcor, res, sizeof(double) * n * n, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    rc = fail(SSA_ECUDA, "copy of the w-correlations failed");
  if (rc == SSA_OK && contrib &&
      cudaMemcpyAsync(contrib, res + (size_t)n * n, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    rc = fail(SSA_ECUDA, "copy of the contributions failed");
  if (rc == SSA_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = fail(SSA_ECUDA, "w-correlation failed");
  cleanup();
  return rc;
}

int ssa_forecast(ssa_ctx* ctx, const int32_t* idx, int32_t n_idx, int32_t M, double* out) {
  if (!ctx || !idx || !out) return fail(SSA_EINVAL, "null argument");
  ssa_ctx* c = ctx;
  if (c->kind != SSA_1D && c->kind != SSA_MSSA) return fail(SSA_EINVAL, "forecasting needs a series or a system of series");
  if (!c->ws.done) return fail(SSA_ESTATE, "context has no decomposition");
  if (M < 1 || n_idx < 1) return fail(SSA_EINVAL, "M and n_idx must be positive");
  const int r = c->ws.r;
  std::vector<int32_t> gof(std::max(r, 1), -1);
  std::vector<int32_t> hidx(idx, idx + n_idx);
  for (int32_t i : hidx) {
    if (i < 0 || i >= r) return fail(SSA_EINVAL, "component %d outside [0, %d)", i, r);
    gof[i] = 0;
  }
  const int64_t L = c->L, total = c->total;
  const int s = (int)c->ch.size();
  std::vector<int64_t> hoff, hlen;
  for (auto& h : c->ch) { hoff.push_back(h.data_off); hlen.push_back(h.nx * h.ny); }
  const int64_t ldw = L - 1 + M;
  double *Y = nullptr, *R = nullptr, *nu2 = nullptr, *work = nullptr, *dout = nullptr;
  int32_t* didx = nullptr;
  int64_t *doff = nullptr, *dlen = nullptr;
  auto cleanup = [&]() {
    for (void* q : {(void*)Y, (void*)R, (void*)nu2, (void*)work, (void*)dout, (void*)didx, (void*)doff, (void*)dlen})
      if (q) c->release(q);
  };
  int rc = c->allocT(&Y, (size_t)total);
  if (rc == SSA_OK) rc = ssa_reconstruct_batch(&c, 1, gof.data(), 1, 0, &Y, 1);
  if (rc == SSA_OK) rc = upload(c, hidx, &didx);
  if (rc == SSA_OK) rc = upload(c, hoff, &doff);
  if (rc == SSA_OK) rc = upload(c, hlen, &dlen);
  if (rc == SSA_OK) rc = c->allocT(&R, (size_t)std::max<int64_t>(L - 1, 1));
  if (rc == SSA_OK) rc = c->allocT(&nu2, 1);
  if (rc == SSA_OK) rc = c->allocT(&work, (size_t)s * ldw);
  if (rc == SSA_OK) rc = c->allocT(&dout, (size_t)s * M);
  if (rc == SSA_OK) {
    if (c->ws.prec == SSA_PREC_FP64) launch_lrr<double>((const double*)c->ws.Uo, L, didx, n_idx, R, nu2, c->stream);
    else launch_lrr<float>((const float*)c->ws.Uo, L, didx, n_idx, R, nu2, c->stream);
    launch_forecast_rec(Y, doff, dlen, s, L, R, M, work, ldw, dout, c->stream);
    if (cudaGetLastError() != cudaSuccess) rc = fail(SSA_ECUDA, "forecast launch failed");
  }
  double hnu2 = 0.0;
  if (rc == SSA_OK && cudaMemcpyAsync(out, dout, sizeof(double) * s * M, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    rc = fail(SSA_ECUDA, "copy of the forecast failed");
  if (rc == SSA_OK && cudaMemcpyAsync(&hnu2, nu2, sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    rc = fail(SSA_ECUDA, "copy of nu^2 failed");
  if (rc == SSA_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = fail(SSA_ECUDA, "forecast failed");
  cleanup();
  if (rc == SSA_OK && !(hnu2 < 1.0))
    rc = fail(SSA_EINVAL, "nu^2 = %g >= 1: the group's window space holds the last unit vector, no recurrence", hnu2);
  return rc;
}

int ssa_forecast_vector(ssa_ctx* ctx, const int32_t* idx, int32_t n_idx, int32_t M, double* out) {
  if (!ctx || !idx || !out) return fail(SSA_EINVAL, "null argument");
  ssa_ctx* c = ctx;
  if (c->kind != SSA_1D && c->kind != SSA_MSSA) return fail(SSA_EINVAL, "forecasting needs a series or a system of series");
  if (!c->ws.done) return fail(SSA_ESTATE, "context has no decomposition");
  if (M < 1 || n_idx < 1) return fail(SSA_EINVAL, "M and n_idx must be positive");
  if (M > 65535) return fail(SSA_EINVAL, "M = %d above 65535", M);
  const int r = c->ws.r;
  std::vector<int32_t> hidx(idx, idx + n_idx);
  for (int32_t i : hidx)
    if (i < 0 || i >= r) return fail(SSA_EINVAL, "component %d outside [0, %d)", i, r);
  const int64_t L = c->L;
  const int s = (int)c->ch.size();
  std::vector<int64_t> hoff, hlen;
  for (auto& h : c->ch) { hoff.push_back(h.data_off); hlen.push_back(h.nx * h.ny); }
  double *G = nullptr, *D = nullptr, *nu2 = nullptr, *cs = nullptr, *dout = nullptr;
  int32_t* didx = nullptr;
  int64_t *doff = nullptr, *dlen = nullptr;
  auto cleanup = [&]() {
    for (void* q : {(void*)G, (void*)D, (void*)nu2, (void*)cs, (void*)dout, (void*)didx, (void*)doff, (void*)dlen})
      if (q) c->release(q);
  };
  int rc = upload(c, hidx, &didx);
  if (rc == SSA_OK) rc = upload(c, hoff, &doff);
  if (rc == SSA_OK) rc = upload(c, hlen, &dlen);
  if (rc == SSA_OK) rc = c->allocT(&G, (size_t)n_idx * n_idx);
  if (rc == SSA_OK) rc = c->allocT(&D, (size_t)n_idx * n_idx);
  if (rc == SSA_OK) rc = c->allocT(&nu2, 1);
  if (rc == SSA_OK) rc = c->allocT(&cs, (size_t)s * (M + L) * n_idx);
  if (rc == SSA_OK) rc = c->allocT(&dout, (size_t)s * M);
  if (rc == SSA_OK) {
    const int x_f64 = c->dtype == SSA_F64 ? 1 : 0;
    if (c->ws.prec == SSA_PREC_FP64)
      launch_vector_forecast<double>((const double*)c->ws.Uo, L, didx, n_idx, c->data, x_f64, doff, dlen, s, M, G, D,
                                     nu2, cs, dout, c->stream);
    else
      launch_vector_forecast<float>((const float*)c->ws.Uo, L, didx, n_idx, c->data, x_f64, doff, dlen, s, M, G, D,
                                    nu2, cs, dout, c->stream);
    if (cudaGetLastError() != cudaSuccess) rc = fail(SSA_ECUDA, "vector forecast launch failed");
  }
  double hnu2 = 0.0;
  if (rc == SSA_OK && cudaMemcpyAsync(out, dout, sizeof(double) * s * M, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    rc = fail(SSA_ECUDA, "copy of the forecast failed");
  if (rc == SSA_OK && cudaMemcpyAsync(&hnu2, nu2, sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    rc = fail(SSA_ECUDA, "copy of nu^2 failed");
  if (rc == SSA_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = fail(SSA_ECUDA, "vector forecast failed");
  cleanup();
  if (rc == SSA_OK && !(hnu2 < 1.0))
    rc = fail(SSA_EINVAL, "nu^2 = %g >= 1: the group's window space holds the last unit vector, no recurrence", hnu2);
  return rc;
}

int ssa_forecast_row(ssa_ctx* ctx, const int32_t* idx, int32_t n_idx, int32_t M, int32_t vector, double* out) {
  if (!ctx || !idx || !out) return fail(SSA_EINVAL, "null argument");
  ssa_ctx* c = ctx;
  if (c->kind != SSA_1D && c->kind != SSA_MSSA) return fail(SSA_EINVAL, "forecasting needs a series or a system of series");
  if (!c->ws.done) return fail(SSA_ESTATE, "context has no decomposition");
  if (M < 1 || n_idx < 1) return fail(SSA_EINVAL, "M and n_idx must be positive");
  if (M > 65535 || n_idx > RF_MAXR) return fail(SSA_EINVAL, "M <= 65535 and n_idx <= %d", RF_MAXR);
  const int s = (int)c->ch.size();
  if (s > RF_MAXS) return fail(SSA_EINVAL, "row forecasts take at most %d series", RF_MAXS);
  const int r = c->ws.r;
  std::vector<int32_t> hidx(idx, idx + n_idx);
  std::vector<int32_t> gof(std::max(r, 1), -1);
  for (int32_t i : hidx) {
    if (i < 0 || i >= r) return fail(SSA_EINVAL, "component %d outside [0, %d)", i, r);
    gof[i] = 0;
  }
  const int64_t L = c->L, K = c->K, total = c->total;
  std::vector<int64_t> hkoff, hkc, hoff, hlen, hwo;
  int64_t kstar = 0, wtot = 0;
  for (auto& h : c->ch) {
    if (h.K.count < 2) return fail(SSA_EINVAL, "a series with fewer than two window origins");
    hkoff.push_back(h.koff); hkc.push_back(h.K.count); hoff.push_back(h.data_off); hlen.push_back(h.nx * h.ny);
    hwo.push_back(wtot);
    wtot += h.K.count - 1 + M;
    kstar = std::max<int64_t>(kstar, h.K.count);
  }
  const int na = std::max(s, n_idx);
  double *Y = nullptr, *A = nullptr, *Bm = nullptr, *work = nullptr, *cs = nullptr, *dout = nullptr;
  int32_t* didx = nullptr;
  int* dfail = nullptr;
  int64_t *dkoff = nullptr, *dkc = nullptr, *doff = nullptr, *dlen = nullptr, *dwo = nullptr;
  auto cleanup = [&]() {
    for (void* q : {(void*)Y, (void*)A, (void*)Bm, (void*)work, (void*)cs, (void*)dout, (void*)didx, (void*)dfail,
                    (void*)dkoff, (void*)dkc, (void*)doff, (void*)dlen, (void*)dwo})
      if (q) c->release(q);
  };
  int rc = SSA_OK;
  if (!vector) {
    rc = c->allocT(&Y, (size_t)total);
    if (rc == SSA_OK) rc = ssa_reconstruct_batch(&c, 1, gof.data(), 1, 0, &Y, 1);
    if (rc == SSA_OK) rc = c->allocT(&work, (size_t)wtot);
  } else {
    rc = c->allocT(&cs, (size_t)(M + kstar) * n_idx);
  }
  if (rc == SSA_OK) rc = upload(c, hidx, &didx);
  if (rc == SSA_OK) rc = upload(c, hkoff, &dkoff);
  if (rc == SSA_OK) rc = upload(c, hkc, &dkc);
  if (rc == SSA_OK) rc = upload(c, hoff, &doff);
  if (rc == SSA_OK) rc = upload(c, hlen, &dlen);
  if (rc == SSA_OK) rc = upload(c, hwo, &dwo);
  if (rc == SSA_OK) rc = c->allocT(&A, (size_t)na * na);
  if (rc == SSA_OK) rc = c->allocT(&Bm, (size_t)na * n_idx);
  if (rc == SSA_OK) rc = c->allocT(&dout, (size_t)s * M);
  if (rc == SSA_OK) rc = c->allocT(&dfail, 1);
  if (rc == SSA_OK && cudaMemsetAsync(dfail, 0, sizeof(int), c->stream) != cudaSuccess) rc = fail(SSA_ECUDA, "memset failed");
  if (rc == SSA_OK) {
    const int x_f64 = c->dtype == SSA_F64 ? 1 : 0;
    if (c->ws.prec == SSA_PREC_FP64)
      launch_row_forecast<double>(vector ? 1 : 0, (const double*)c->ws.Vo, K, didx, n_idx, dkoff, dkc, doff, dlen, s, L,
                                  M, kstar, Y, c->data, x_f64, A, Bm, work, dwo, cs, dout, dfail, c->stream);
    else
      launch_row_forecast<float>(vector ? 1 : 0, (const float*)c->ws.Vo, K, didx, n_idx, dkoff, dkc, doff, dlen, s, L,
                                 M, kstar, Y, c->data, x_f64, A, Bm, work, dwo, cs, dout, dfail, c->stream);
    if (cudaGetLastError() != cudaSuccess) rc = fail(SSA_ECUDA, "row forecast launch failed");
  }
  int hfail = 0;
  if (rc == SSA_OK && cudaMemcpyAsync(out, dout, sizeof(double) * s * M, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    rc = fail(SSA_ECUDA, "copy of the forecast failed");
  if (rc == SSA_OK && cudaMemcpyAsync(&hfail, dfail, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    rc = fail(SSA_ECUDA, "copy of the solve status failed");
  if (rc == SSA_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = fail(SSA_ECUDA, "row forecast failed");
  cleanup();
  if (rc == SSA_OK && hfail)
    rc = fail(SSA_EINVAL, "the row forecast's system is singular (the last rows of the group's origin vectors span too much)");
  return rc;
}

int ssa_get_shape(const ssa_ctx* cc, int64_t* L, int64_t* K, uint8_t* origin_mask, int32_t* weights) {
  ssa_ctx* c = const_cast<ssa_ctx*>(cc);
  if (!c) return fail(SSA_EINVAL, "null argument");
  if (L) *L = c->L;
  if (K) *K = c->K;
  if (origin_mask) {
    uint8_t* d = nullptr;
    TRY(c->allocT(&d, (size_t)c->total));
    for (auto& h : c->ch) {
      dim3 g(grid1(h.nx), (unsigned)h.ny);
      if (h.K.count > 0 || h.K.bits) {
        k_kmask<<<g, 256, 0, c->stream>>>(h.K.bits, h.K.words, h.cx, h.cy, (int)h.nx, (int)h.ny, d + h.data_off); count_launch();
      } else {
        CU(cudaMemsetAsync(d + h.data_off, 0, (size_t)(h.nx * h.ny), c->stream));
      }
    }
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(origin_mask, d, (size_t)c->total, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    c->release(d);
  }
  if (weights) {
    for (auto& h : c->ch)
      CU(cudaMemcpyAsync(weights + h.data_off, h.w, sizeof(int32_t) * h.nx * h.ny, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
  }
  return SSA_OK;
}

int ssa_matvec(ssa_ctx* ctx, int32_t transpose, int32_t prec, const double* in, double* out, int32_t on_device) {
  if (!ctx || !in || !out) return fail(SSA_EINVAL, "null argument");
  if (prec == SSA_PREC_FP64) {
    if (ctx->log2Mx > 13) return fail(SSA_EUNSUPPORTED, "FP64 form supports FFT length <= 8192 along x");
    return matvec_T<double>(ctx, transpose, in, out, on_device);
  }
  return matvec_T<float>(ctx, transpose, in, out, on_device);
}

// ---------------------------------------------------------------- autotuner
// Times decompositions of ctx (with its own Krylov dimension kd) on the
// context's stream: the span between two events, host round trips included;
// the faster of `reps` runs.
static int tune_run(ssa_ctx* ctx, const ssa_params& p0, int kd, double* ms, int reps = 2) {
  ssa_params p = p0;
  p.krylov_dim = kd;
  cudaEvent_t a = nullptr, b = nullptr;
  CU(cudaEventCreate(&a));
  CU(cudaEventCreate(&b));
  int rc = SSA_OK;
  double best = 1e300;
  for (int i = 0; i < reps && rc == SSA_OK; ++i) {
    cudaEventRecord(a, ctx->stream);
    rc = ssa_decompose(ctx, &p);
    cudaEventRecord(b, ctx->stream);
    cudaEventSynchronize(b);
    float f = 0.0f;
    cudaEventElapsedTime(&f, a, b);
    best = std::min(best, (double)f);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms = best;
  return rc;
}

int ssa_autotune(ssa_ctx* ctx, const ssa_params* params, ssa_tune_result* out) {
  if (!ctx || !params) return fail(SSA_EINVAL, "null argument");
  if (params->rank < 1 || params->rank > std::min(ctx->L, ctx->K))
    return fail(SSA_ERANK, "rank %d outside [1, min(L, K)]", params->rank);
  const bool f64 = params->prec == SSA_PREC_FP64;
  const int esz = f64 ? 16 : 8;                     // complex element of the form
  const int r = params->rank;
  const std::string kkey = kdim_key(params->prec, ctx->kind, ctx->L, ctx->K, r);
  const std::string tkey = ytk_key(esz, ctx->log2Mx, ctx->log2My);
  {
    std::lock_guard<std::mutex> lk(g_plans.mu);     // candidates are timed without earlier plans
    g_plans.kdim.erase(kkey);
    g_plans.ytk.erase(tkey);
  }
  // Krylov dimensions around the default 2r + 16
  const int d = default_k(r, ctx->L, ctx->K, 0);
  const int kmax = (int)std::min<int64_t>(KMAX, std::min(ctx->L, ctx->K));
  std::vector<int> ks;
  for (int c : {std::max(r + 2, (2 * d) / 3), d, (3 * d) / 2, 2 * d}) {
    const int kc = std::max(r, std::min(c, kmax));
    if (std::find(ks.begin(), ks.end(), kc) == ks.end()) ks.push_back(kc);
  }
  // A candidate replaces the default only when it is faster by more than
  // TUNE_MIN_GAIN: one decomposition's time moves by about a percent from run
  // to run, and a choice inside that band is noise (it can be slower for the
  // batches the plan is then used for).
  constexpr double TUNE_MIN_GAIN = 0.02;
  double ms = 0.0, ms_default = 0.0;
  int tried = 0;
  TRY(tune_run(ctx, *params, d, &ms, 1));           // warm-up: spectra, workspaces
  std::vector<std::pair<int, double>> timed;        // converged candidates
  bool def_ok = false;
  for (int kc : ks) {
    const int rc = tune_run(ctx, *params, kc, &ms);
    ++tried;
    if (kc == d) { ms_default = ms; def_ok = rc == SSA_OK; }
    if (rc == SSA_OK) timed.push_back({kc, ms});
  }
  int best_k = d;
  double best_ms = def_ok ? ms_default : 1e300;
  for (auto& c : timed)
    if (c.first != d && c.second < best_ms && (!def_ok || c.second < ms_default * (1.0 - TUNE_MIN_GAIN))) {
      best_ms = c.second;
      best_k = c.first;
    }
  // y-pass tile of 2D grids: powers of two around the default that fit the
  // shared memory of a block
  const int dtk = f64 ? ypass_tk<double>(ctx->log2My) : ypass_tk<float>(ctx->log2My);
  int best_tk = dtk;
  if (ctx->log2My > 0) {
    const int pl = padded_len(1 << ctx->log2My);
    const int nb = YPASS_BUF_BYTES / esz;
    for (int tk : {dtk / 2, dtk * 2, dtk * 4}) {
      if (tk < 1 || tk > 64) continue;
      // (a launch shared with taller grids carries their twiddle table: the
      // largest y-grid, 2^12, is assumed)
      const size_t bytes = (size_t)esz * (2 * (size_t)std::max(nb, tk * pl) + (1 << 12) / 8 + 1);
      if (bytes > (size_t)device_max_smem()) continue;
      {
        std::lock_guard<std::mutex> lk(g_plans.mu);
        g_plans.ytk[tkey] = tk;
      }
      const int rc = tune_run(ctx, *params, best_k, &ms);
      ++tried;
      if (rc == SSA_OK && ms < best_ms * (1.0 - TUNE_MIN_GAIN)) { best_ms = ms; best_tk = tk; }
    }
  }
  {
    std::lock_guard<std::mutex> lk(g_plans.mu);
    g_plans.kdim[kkey] = best_k;
    if (ctx->log2My > 0) g_plans.ytk[tkey] = best_tk;
  }
  // leave the context decomposed with the chosen plan
  TRY(tune_run(ctx, *params, 0, &ms, 1));
  if (out) {
    out->krylov_dim = best_k;
    out->ytk = ctx->log2My > 0 ? best_tk : 0;
    out->n_tried = tried;
    out->pad_ = 0;
    out->ms_default = ms_default;
    out->ms_best = best_ms;
  }
  return SSA_OK;
}

int ssa_plans_export(char* buf, int64_t cap, int64_t* len) {
  std::string t;
  {
    std::lock_guard<std::mutex> lk(g_plans.mu);
    for (auto& kv : g_plans.kdim) t += "kdim " + kv.first + " " + std::to_string(kv.second) + "\n";
    for (auto& kv : g_plans.ytk) t += "ytk " + kv.first + " " + std::to_string(kv.second) + "\n";
  }
  if (len) *len = (int64_t)t.size();
  if (buf && cap > 0) {
    const size_t n = std::min<size_t>(t.size(), (size_t)cap - 1);
    std::memcpy(buf, t.data(), n);
    buf[n] = 0;
    if (n < t.size()) return fail(SSA_EINVAL, "buffer of %lld bytes holds %zu of %zu", (long long)cap, n, t.size());
  }
  return SSA_OK;
}

int ssa_plans_import(const char* text) {
  if (!text) return fail(SSA_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(g_plans.mu);
  const char* p = text;
  while (*p) {
    const char* e = std::strchr(p, '\n');
    const std::string line(p, e ? (size_t)(e - p) : std::strlen(p));
    p = e ? e + 1 : p + line.size();
    if (line.empty()) continue;
    char kind[16] = {}, key[96] = {};
    int v = 0;
    if (std::sscanf(line.c_str(), "%15s %95s %d", kind, key, &v) != 3 || v < 1)
      return fail(SSA_EINVAL, "bad plan line: %s", line.c_str());
    if (!std::strcmp(kind, "kdim") && v <= KMAX) g_plans.kdim[key] = v;
    else if (!std::strcmp(kind, "ytk") && v <= 64) g_plans.ytk[key] = v;
    else return fail(SSA_EINVAL, "bad plan line: %s", line.c_str());
  }
  return SSA_OK;
}

int ssa_synchronize(ssa_ctx* c) {
  if (!c) return fail(SSA_EINVAL, "null argument");
  CU(cudaStreamSynchronize(c->stream));
  return SSA_OK;
}

void ssa_destroy(ssa_ctx* c) {
  if (!c) return;
  if (c->stream) {
    for (auto& a : c->allocs) cudaFreeAsync(a.first, c->stream);
    cudaStreamSynchronize(c->stream);
    if (c->own_stream) cudaStreamDestroy(c->stream);
  }
  delete c;
}

}  // extern "C"

// NaN at masked-out samples (the observed set is then "not NaN")
__global__ void k_apply_mask(void* data, int dbl, const uint8_t* m, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!m[i]) {
      if (dbl) ((double*)data)[i] = __longlong_as_double(0x7ff8000000000000ll);
      else ((float*)data)[i] = __int_as_float(0x7fc00000);
    }
}

void launch_apply_mask(void* data, int dbl, const uint8_t* m, int64_t n, cudaStream_t st) {
  k_apply_mask<<<grid1(n), 256, 0, st>>>(data, dbl, m, n); count_launch();
}

// ============================================================== serving
// Continuous batching: requests are admitted (in arrival order) while the
// device-memory budget allows, join the Lanczos engine at a restart-cycle
// boundary, advance in the same launches as every other live request (each at
// its own cycle), and retire -- final Ritz vectors, reconstruction, results
// copied out, memory freed -- as soon as they converge.  Series (1D / MSSA)
// and images run in two engines on the same stream.
namespace {

struct SrvReq {
  int64_t ticket = 0;
  ssa_input in{};
  std::vector<char> data;
  std::vector<int64_t> lengths;
  std::vector<uint8_t> mask, wmask;
  ssa_window win{};
  ssa_params p{};
  std::vector<int32_t> group_of;
  int ng = 0, residual = 0;
  int64_t total = 0, est = 0, bytes = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  ssa_ctx* ctx = nullptr;
  int status = SSA_OK;
  std::vector<double> sigma, out;
  int32_t restarts = 0;
  double maxres = 0;
};

double now_s(const std::chrono::steady_clock::time_point& t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// Device bytes a request will hold at most (embedding, spectra, Lanczos
// workspace, reconstruction scratch), from its sizes alone.
int64_t estimate_bytes(const SrvReq& q, int prec) {
  const size_t cz = prec == SSA_PREC_FP64 ? 8 : 4;
  const size_t esz = q.in.dtype == SSA_F64 ? 8 : 4;
  std::vector<int64_t> ns;
  int64_t L = 0, Kmax = 0;
  if (q.in.kind == SSA_1D) ns.push_back(q.in.n);
  else if (q.in.kind == SSA_MSSA) ns = q.lengths;
  if (q.in.kind == SSA_2D) {
    L = q.win.lx * q.win.ly;
    Kmax = (q.in.nx - q.win.lx + 1) * (q.in.ny - q.win.ly + 1);
  } else {
    L = q.win.L;
    for (auto n : ns) Kmax += std::max<int64_t>(0, n - L + 1);
  }
  const int64_t nch = q.in.kind == SSA_MSSA ? (int64_t)ns.size() : 1;
  // FFT grid, as ssa_embed chooses it
  int64_t Mx = 16, My = 1, fymax = 1;
  bool fold = false;
  if (q.in.kind == SSA_2D) {
    while (Mx < q.in.nx) Mx *= 2;
    while (My < q.in.ny) My *= 2;
  } else {
    int64_t mx = 1;
    for (auto n : ns) mx = std::max(mx, n);
    while (Mx < mx) Mx *= 2;
    if (ilog2_ceil(mx) >= FOLD_MIN_LOG2) {
      const FoldGeom g = fold_geometry(ns, L);
      fold = true;
      Mx = 2 * (int64_t)g.B;
      My = int64_t(1) << g.log2My;
      for (int f : g.fy) fymax = std::max<int64_t>(fymax, f);
    }
  }
  const int64_t H = Mx / 2, hs = (H + 1) * My;
  int64_t b = 0;
  // embedding: data, mask, observed bits, origins, weights
  b += (int64_t)(esz + 1 + 4) * q.total + q.total / 4 + 4096 * (nch + 2);
  b += nch * hs * 2 * (int64_t)cz;                                   // spectra
  if (My > 1) b += nch * hs * 2 * (int64_t)cz;                       // spectrum scratch
  const int64_t r = q.p.rank, k = std::min<int64_t>(std::min<int64_t>(2 * r + 16, KMAX), std::min(L, Kmax));
  const int64_t Ls = std::min(L, Kmax), Kl = std::max(L, Kmax);
  b += 8 * Ls * (k + 1) + (int64_t)cz * Kl * (k + 1) + 8 * Ls + (int64_t)cz * Kl;   // bases, work vectors
  b += (int64_t)cz * (Ls + Kl) * nch + 4 * 8 * (k + 2) * (k + 2);                    // partials, small matrices
  b += (int64_t)cz * (L + Kmax) * r;                                 // outputs U, V
  if (My > 1) b += 2 * nch * hs * 2 * (int64_t)cz;                   // matvec x / y scratch
  const int64_t nout = q.ng + (q.residual ? 1 : 0);
  b += 8 * q.total * nout;                                           // reconstruction output
  if (My > 1) b += (3 + q.ng) * 16 * hs + (fold ? 8 * Mx * fymax : 0);
  else b += 16 * (H + 1) * r;
  return b + (1 << 20);
}

}  // namespace

struct ssa_server {
  ssa_server_config cfg{};
  cudaStream_t st = nullptr;
  bool own_stream = false;
  int device = 0;
  std::chrono::steady_clock::time_point t0;
  int64_t next_ticket = 1;
  int64_t bytes_live = 0;
  std::deque<SrvReq*> queue;
  std::vector<SrvReq*> live_series, live_images;
  std::map<int64_t, SrvReq*> finished;
  LzEngine<float> e32s, e32i;
  LzEngine<double> e64s, e64i;
  ~ssa_server() {
    for (auto* q : queue) delete q;
    for (auto* q : live_series) { ssa_destroy(q->ctx); delete q; }
    for (auto* q : live_images) { ssa_destroy(q->ctx); delete q; }
    for (auto& f : finished) delete f.second;
  }
};

namespace {

template <typename T>
int server_round(ssa_server* s, LzEngine<T>& eng, std::vector<SrvReq*>& live, std::vector<SrvReq*>& admitted,
                 int32_t* n_done) {
  // admit: spectra and workspaces, join the engine
  if (!admitted.empty()) {
    std::vector<ssa_ctx*> cs;
    std::vector<ssa_params> ps;
    for (auto* q : admitted) { cs.push_back(q->ctx); ps.push_back(q->p); }
    std::vector<int> rc;
    TRY(prepare_members<T>(cs.data(), (int)cs.size(), ps.data(), s->st, rc));
    for (size_t i = 0; i < admitted.size(); ++i) {
      SrvReq* q = admitted[i];
      if (rc[i] != SSA_OK) {
        q->status = rc[i];
        q->t_done = now_s(s->t0);
        s->bytes_live -= q->est;
        ssa_destroy(q->ctx);
        q->ctx = nullptr;
        s->finished[q->ticket] = q;
        if (n_done) ++*n_done;
        continue;
      }
      eng.add(q->ctx, q->p.seed);
      live.push_back(q);
    }
  }
  if (live.empty()) return SSA_OK;
  TRY(eng.build());
  TRY(eng.start_fresh());
  TRY(eng.run_chunk());
  // retire what is done; restart the rest
  std::vector<int> done;
  for (size_t i = 0; i < eng.live.size(); ++i)
    if (!eng.hst[i].active) done.push_back((int)i);
  TRY(eng.retire(done));
  if (!done.empty()) {
    std::vector<ssa_ctx*> cs;
    std::vector<RecReq> req;
    std::vector<SrvReq*> reqs;
    for (int i : done) {
      ssa_ctx* c = eng.live[i];
      SrvReq* q = nullptr;
      for (auto* x : live) if (x->ctx == c) { q = x; break; }
      reqs.push_back(q);
      const int nout = q->ng + (q->residual ? 1 : 0);
      q->out.assign((size_t)q->total * std::max(nout, 0), 0.0);
      q->restarts = eng.hst[i].restarts;
      q->maxres = eng.hst[i].maxres;
      if (!eng.hst[i].converged) q->status = SSA_ENOTCONV;
      if (nout > 0) {
        cs.push_back(c);
        req.push_back({q->group_of.data(), q->ng, q->residual, q->out.data()});
      }
    }
    if (!cs.empty()) TRY(reconstruct_dispatch(cs.data(), (int)cs.size(), req.data(), 0));
    CU(cudaStreamSynchronize(s->st));
    const double t = now_s(s->t0);
    for (auto* q : reqs) {
      q->sigma.assign(q->p.rank, 0.0);
      CU(cudaMemcpy(q->sigma.data(), q->ctx->ws.sigma, sizeof(double) * q->p.rank, cudaMemcpyDeviceToHost));
      q->bytes = q->ctx->bytes;
      q->t_done = t;
      s->bytes_live -= q->est;
      ssa_destroy(q->ctx);
      q->ctx = nullptr;
      s->finished[q->ticket] = q;
      live.erase(std::find(live.begin(), live.end(), q));
      if (n_done) ++*n_done;
    }
    eng.remove(done);
  }
  return SSA_OK;
}

template <typename T>
int server_step_T(ssa_server* s, std::vector<SrvReq*>& adm_s, std::vector<SrvReq*>& adm_i, int32_t* n_done,
                  LzEngine<T>& es, LzEngine<T>& ei) {
  TRY(server_round<T>(s, es, s->live_series, adm_s, n_done));
  TRY(server_round<T>(s, ei, s->live_images, adm_i, n_done));
  return SSA_OK;
}

}  // namespace

extern "C" {

int ssa_server_create(const ssa_server_config* cfg, void* cuda_stream, ssa_server** out) {
  if (!cfg || !out) return fail(SSA_EINVAL, "null argument");
  if (cfg->prec != SSA_PREC_FP32FFT_FP64REORTH && cfg->prec != SSA_PREC_FP64) return fail(SSA_EINVAL, "precision");
  ssa_server* s = new ssa_server();
  s->cfg = *cfg;
  if (s->cfg.memory_budget <= 0) s->cfg.memory_budget = int64_t(40) << 30;
  if (s->cfg.max_live <= 0) s->cfg.max_live = 512;
  s->t0 = std::chrono::steady_clock::now();
  if (cudaGetDevice(&s->device) != cudaSuccess || ensure_tables(s->device) != SSA_OK) {
    delete s;
    return fail(SSA_ECUDA, "device set-up failed");
  }
  if (cuda_stream) s->st = (cudaStream_t)cuda_stream;
  else {
    if (cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess) { delete s; return fail(SSA_ECUDA, "stream"); }
    s->own_stream = true;
  }
  for (auto* e : {&s->e32s, &s->e32i}) { e->st = s->st; e->device = s->device; }
  for (auto* e : {&s->e64s, &s->e64i}) { e->st = s->st; e->device = s->device; }
  *out = s;
  return SSA_OK;
}

int ssa_server_submit(ssa_server* s, const ssa_input* in, const ssa_window* win, const ssa_params* p,
                      const int32_t* group_of, int32_t n_groups, int32_t residual, int64_t* ticket) {
  if (!s || !in || !win || !p || !ticket || !in->data || n_groups < 0 || (n_groups > 0 && !group_of))
    return fail(SSA_EINVAL, "null argument");
  if (in->on_device) return fail(SSA_EINVAL, "server requests take host data");
  SrvReq* q = new SrvReq();
  q->in = *in;
  int64_t total = 0;
  if (in->kind == SSA_1D) total = in->n;
  else if (in->kind == SSA_MSSA) {
    if (!in->lengths || in->n_series < 1) { delete q; return fail(SSA_EINVAL, "MSSA lengths"); }
    q->lengths.assign(in->lengths, in->lengths + in->n_series);
    for (auto n : q->lengths) total += n;
    q->in.lengths = q->lengths.data();
  } else total = in->nx * in->ny;
  if (total <= 0) { delete q; return fail(SSA_EINVAL, "empty input"); }
  q->total = total;
  const size_t esz = in->dtype == SSA_F64 ? 8 : 4;
  q->data.assign((const char*)in->data, (const char*)in->data + esz * total);
  q->in.data = q->data.data();
  if (in->mask) { q->mask.assign(in->mask, in->mask + total); q->in.mask = q->mask.data(); }
  q->win = *win;
  if (win->wmask && in->kind == SSA_2D) {
    q->wmask.assign(win->wmask, win->wmask + win->lx * win->ly);
    q->win.wmask = q->wmask.data();
  }
  q->p = *p;
  q->p.prec = s->cfg.prec;
  q->ng = n_groups;
  q->residual = residual ? 1 : 0;
  q->group_of.assign(p->rank > 0 ? p->rank : 0, -1);
  for (int i = 0; i < p->rank && group_of; ++i) q->group_of[i] = group_of[i];
  q->ticket = s->next_ticket++;
  q->t_submit = now_s(s->t0);
  q->est = estimate_bytes(*q, s->cfg.prec);
  s->queue.push_back(q);
  *ticket = q->ticket;
  return SSA_OK;
}

int ssa_server_step(ssa_server* s, int32_t* n_done) {
  if (!s) return fail(SSA_EINVAL, "null argument");
  if (n_done) *n_done = 0;
  // admission in arrival order while the budget and the live count allow
  std::vector<SrvReq*> adm;
  const int64_t nlive = (int64_t)(s->live_series.size() + s->live_images.size());
  while (!s->queue.empty() && nlive + (int64_t)adm.size() < s->cfg.max_live) {
    SrvReq* q = s->queue.front();
    if (q->est > s->cfg.memory_budget) {
      s->queue.pop_front();
      q->status = fail(SSA_ENOMEM, "request needs %lld bytes, budget %lld", (long long)q->est,
                       (long long)s->cfg.memory_budget);
      q->t_done = now_s(s->t0);
      s->finished[q->ticket] = q;
      if (n_done) ++*n_done;
      continue;
    }
    if (s->bytes_live + q->est > s->cfg.memory_budget) break;
    s->queue.pop_front();
    s->bytes_live += q->est;
    q->t_admit = now_s(s->t0);
    adm.push_back(q);
  }
  std::vector<SrvReq*> adm_s, adm_i;
  if (!adm.empty()) {
    std::vector<ssa_input> ins;
    std::vector<ssa_window> wins;
    for (auto* q : adm) { ins.push_back(q->in); wins.push_back(q->win); }
    std::vector<ssa_ctx*> cs(adm.size(), nullptr);
    const int32_t unset = INT32_MIN;   // status left unwritten: the batch failed as a whole
    std::vector<int32_t> st(adm.size(), unset);
    const int brc = ssa_embed_batch(ins.data(), wins.data(), (int32_t)adm.size(), (void*)s->st, cs.data(), st.data());
    for (size_t i = 0; i < adm.size(); ++i) {
      SrvReq* q = adm[i];
      if (st[i] == unset && cs[i]) { ssa_destroy(cs[i]); cs[i] = nullptr; }
      if (st[i] != SSA_OK || !cs[i]) {
        q->status = st[i] == unset ? (brc != SSA_OK ? brc : SSA_ECUDA) : (st[i] != SSA_OK ? st[i] : SSA_ECUDA);
        q->t_done = now_s(s->t0);
        s->bytes_live -= q->est;
        s->finished[q->ticket] = q;
        if (n_done) ++*n_done;
        continue;
      }
      q->ctx = cs[i];
      (q->in.kind == SSA_2D ? adm_i : adm_s).push_back(q);
    }
  }
  if (s->cfg.prec == SSA_PREC_FP64) TRY(server_step_T<double>(s, adm_s, adm_i, n_done, s->e64s, s->e64i));
  else TRY(server_step_T<float>(s, adm_s, adm_i, n_done, s->e32s, s->e32i));
  return SSA_OK;
}

int ssa_server_stats(const ssa_server* s, int64_t* queued, int64_t* live, int64_t* finished, int64_t* bytes_live) {
  if (!s) return fail(SSA_EINVAL, "null argument");
  if (queued) *queued = (int64_t)s->queue.size();
  if (live) *live = (int64_t)(s->live_series.size() + s->live_images.size());
  if (finished) *finished = (int64_t)s->finished.size();
  if (bytes_live) *bytes_live = s->bytes_live;
  return SSA_OK;
}

int ssa_server_finished(const ssa_server* s, int64_t* tickets, int32_t cap, int32_t* n) {
  if (!s || !n || (cap > 0 && !tickets)) return fail(SSA_EINVAL, "null argument");
  int32_t m = 0;
  for (auto& f : s->finished) {
    if (m >= cap) break;
    tickets[m++] = f.first;
  }
  *n = m;
  return SSA_OK;
}

int ssa_server_take(ssa_server* s, int64_t ticket, ssa_server_result* res, double* sigma, double* out) {
  if (!s) return fail(SSA_EINVAL, "null argument");
  auto it = s->finished.find(ticket);
  if (it == s->finished.end()) return fail(SSA_ESTATE, "request %lld not finished", (long long)ticket);
  SrvReq* q = it->second;
  if (res) {
    std::memset(res, 0, sizeof(*res));
    res->ticket = q->ticket;
    res->status = q->status;
    res->rank = q->p.rank;
    res->out_len = (int64_t)q->out.size();
    res->restarts = q->restarts;
    res->max_residual = q->maxres;
    res->t_submit = q->t_submit;
    res->t_admit = q->t_admit;
    res->t_done = q->t_done;
    res->device_bytes = q->bytes;
    res->estimated_bytes = q->est;
  }
  if (sigma && !q->sigma.empty()) std::memcpy(sigma, q->sigma.data(), sizeof(double) * q->sigma.size());
  if (out && !q->out.empty()) std::memcpy(out, q->out.data(), sizeof(double) * q->out.size());
  s->finished.erase(it);
  delete q;
  return SSA_OK;
}

double ssa_server_clock(const ssa_server* s) { return s ? now_s(s->t0) : 0.0; }

void ssa_server_destroy(ssa_server* s) {
  if (!s) return;
  cudaStream_t st = s->st;
  bool own = s->own_stream;
  if (st) cudaStreamSynchronize(st);
  delete s;
  if (own && st) cudaStreamDestroy(st);
}

}  // extern "C"
