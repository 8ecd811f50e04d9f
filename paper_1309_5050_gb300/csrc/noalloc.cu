// A trajectory-matrix product for one series that allocates nothing.
//
// Some callers cannot allocate device memory at call time: code running
// inside a captured CUDA graph region, real-time or embedded hosts whose
// memory budget is fixed when they start, or plug-in hosts that forbid the
// library from touching the allocator.  ssa_matvec_series_noalloc serves them:
// the caller passes device buffers for the series and both vectors, and the
// only intermediate data -- the twiddle table and the half spectrum of the
// series -- live in one file-scope device array of fixed size, reserved when
// the library is loaded and held by every GPU that loads it until the process
// exits.
//
// Host code must not use the array's name as a device address (on the host it
// is only a stand-in): the address is looked up once per device with
// cudaGetSymbolAddress while that device is current, on the first call made on
// that device, and handed to the kernels.  That first call also fills the
// twiddle table, so it should come before any stream capture.
//
// Every call overwrites the shared array (the spectrum of its own series), so
// calls whose work overlaps on the GPU race: order them on one stream, or
// synchronise between them.  Nothing in the array has to start at zero: each
// call rewrites every entry it reads.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/ssa.h"
#include "fft_block.cuh"
#include "launch.h"

namespace ssa {
namespace {

constexpr int NA_LOG2_MAX = 14;                    // longest FFT grid: 16384 samples
constexpr int NA_HMAX = 1 << (NA_LOG2_MAX - 1);    // complex length of the packed transform
constexpr size_t NA_TW_BYTES = sizeof(Cx<float>) * TW_N;
constexpr size_t NA_SPEC_BYTES = sizeof(Cx<float>) * (NA_HMAX + 1);
constexpr size_t NA_BYTES = NA_TW_BYTES + ((NA_SPEC_BYTES + 255) / 256) * 256;

// twiddles (TW_N complex float) followed by one half spectrum (H+1 complex)
static __device__ __align__(256) unsigned char g_na_scratch[NA_BYTES];

struct NaDevice { bool ready = false; unsigned char* base = nullptr; };
static NaDevice g_na_dev[64];
static std::mutex g_na_mu;

__global__ void k_na_twiddles(Cx<float>* tw) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < TW_N; j += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(-2.0 * (double)j / (double)TW_N, &s, &c);
    tw[j] = cx((float)c, (float)s);
  }
}

// Half spectrum of the zero-padded series, scaled by 1/M (one CTA).
__global__ void __launch_bounds__(512) k_na_spectrum(const float* __restrict__ x, int n, int log2M,
                                                     const Cx<float>* __restrict__ tw, Cx<float>* xh) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int log2H = log2M - 1, H = 1 << log2H, M = 2 * H;
  Cx<float>* A = reinterpret_cast<Cx<float>*>(smem);
  Cx<float>* B = A + (H + 1);
  float* rb = reinterpret_cast<float*>(A);
  const float scale = 1.0f / (float)M;
  for (int i = threadIdx.x; i < M; i += blockDim.x) rb[i] = (i < n) ? x[i] * scale : 0.0f;
  __syncthreads();
  Cx<float>* Z = block_fft<float, false>(A, B, log2H, 1, tw);
  for (int k = threadIdx.x; k <= H; k += blockDim.x) xh[k] = untwist_fwd(Z, k, log2H, tw);
}

// u = X v (transpose 0: v on the origins 0..K-1, u on the window 0..L-1) or
// v = X^T u (transpose 1): scatter, packed FFT, product with the conjugate,
// inverse, gather -- the Hankel product of Sec. 6.1.2, Alg. hmul_u.
__global__ void __launch_bounds__(512) k_na_product(const float* __restrict__ in, int nin,
                                                    float* __restrict__ out, int nout, int log2M,
                                                    const Cx<float>* __restrict__ tw,
                                                    const Cx<float>* __restrict__ xh) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int log2H = log2M - 1, H = 1 << log2H, M = 2 * H;
  Cx<float>* A = reinterpret_cast<Cx<float>*>(smem);
  Cx<float>* B = A + (H + 1);
  float* rb = reinterpret_cast<float*>(A);
  for (int i = threadIdx.x; i < M; i += blockDim.x) rb[i] = (i < nin) ? in[i] : 0.0f;
  __syncthreads();
  Cx<float>* Z = block_fft<float, false>(A, B, log2H, 1, tw);
  Cx<float>* G = (Z == A) ? B : A;
  for (int k = threadIdx.x; k <= H; k += blockDim.x) G[k] = xh[k] * conj(untwist_fwd(Z, k, log2H, tw));
  __syncthreads();
  for (int k = threadIdx.x; k < H; k += blockDim.x) Z[k] = twist_inv(G, k, log2H, tw);
  __syncthreads();
  Cx<float>* R = block_fft<float, true>(Z, G, log2H, 1, tw);
  const float* r = reinterpret_cast<const float*>(R);
  for (int i = threadIdx.x; i < nout; i += blockDim.x) out[i] = r[i];
}

// Once per device, with that device current: the scratch array's device
// address (cudaGetSymbolAddress), the shared-memory limit of both kernels and
// the twiddle table.  Returns an SSA code.
static int na_setup(int dev, cudaStream_t st, unsigned char** base, char* err, size_t errn) {
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (dev < 0 || dev >= 64) { snprintf(err, errn, "device index %d out of range", dev); return SSA_EINVAL; }
  NaDevice& d = g_na_dev[dev];
  if (d.ready) { *base = d.base; return SSA_OK; }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
  if (e != cudaSuccess || !p) {
    snprintf(err, errn, "cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(e));
    return SSA_ECUDA;
  }
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) {
    snprintf(err, errn, "shared-memory limit query failed: %s", cudaGetErrorString(e));
    return SSA_ECUDA;
  }
  const int need = (int)(2 * (NA_HMAX + 1) * sizeof(Cx<float>));
  if (optin < need) { snprintf(err, errn, "device allows %d bytes of shared memory, %d needed", optin, need); return SSA_EUNSUPPORTED; }
  // both kernels need the raised limit: a failure here is reported with its
  // cause and the device stays unprepared (the next call tries again)
  const void* fns[2] = {(const void*)k_na_spectrum, (const void*)k_na_product};
  for (const void* fn : fns) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
    if (e != cudaSuccess) {
      snprintf(err, errn, "raising the shared-memory limit of a product kernel failed: %s", cudaGetErrorString(e));
      return SSA_ECUDA;
    }
  }
  k_na_twiddles<<<64, 256, 0, st>>>(reinterpret_cast<Cx<float>*>(p)); count_launch();
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { snprintf(err, errn, "twiddle set-up failed: %s", cudaGetErrorString(e)); return SSA_ECUDA; }
  d.base = reinterpret_cast<unsigned char*>(p);
  d.ready = true;
  *base = d.base;
  return SSA_OK;
}

}  // namespace
}  // namespace ssa

static thread_local char g_na_err[256] = "";

extern "C" const char* ssa_noalloc_last_error(void) { return g_na_err; }

extern "C" int ssa_matvec_series_noalloc(const float* x, int64_t n, int64_t L, int32_t transpose,
                                         const float* in, float* out, void* cuda_stream) {
  using namespace ssa;
  if (!x || !in || !out) { snprintf(g_na_err, sizeof(g_na_err), "null pointer"); return SSA_EINVAL; }
  if (n < 3 || L < 2 || L >= n) {
    snprintf(g_na_err, sizeof(g_na_err), "need 1 < L < n and n >= 3 (n=%lld, L=%lld)", (long long)n, (long long)L);
    return SSA_EINVAL;
  }
  if (n > (int64_t(1) << NA_LOG2_MAX)) {
    snprintf(g_na_err, sizeof(g_na_err), "series of %lld samples exceeds the fixed scratch limit of %d",
             (long long)n, 1 << NA_LOG2_MAX);
    return SSA_EUNSUPPORTED;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { snprintf(g_na_err, sizeof(g_na_err), "no current device"); return SSA_ECUDA; }
  unsigned char* base = nullptr;
  int rc = na_setup(dev, st, &base, g_na_err, sizeof(g_na_err));
  if (rc != SSA_OK) return rc;
  const int64_t K = n - L + 1;
  int log2M = 4;
  while ((int64_t(1) << log2M) < n) ++log2M;
  const int H = 1 << (log2M - 1);
  const Cx<float>* tw = reinterpret_cast<const Cx<float>*>(base);
  Cx<float>* xh = reinterpret_cast<Cx<float>*>(base + NA_TW_BYTES);
  const size_t smem = 2 * (size_t)(H + 1) * sizeof(Cx<float>);
  k_na_spectrum<<<1, 512, smem, st>>>(x, (int)n, log2M, tw, xh); count_launch();
  const int nin = (int)(transpose ? L : K), nout = (int)(transpose ? K : L);
  k_na_product<<<1, 512, smem, st>>>(in, nin, out, nout, log2M, tw, xh); count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(g_na_err, sizeof(g_na_err), "launch failed: %s", cudaGetErrorString(e));
    return SSA_ECUDA;
  }
  return SSA_OK;
}
