// Host-side entry points of the kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>
#include "kernels.cuh"
#include "fft_block.cuh"

namespace ssa {

// Kernel-launch counter (process-wide) and per-phase device timing.
void count_launch(int n = 1);
enum Phase : int { PH_SHAPES = 0, PH_SPECTRUM = 1, PH_MATVEC = 2, PH_SHORT = 3, PH_LONG = 4, PH_RITZ = 5,
                   PH_RECON = 6, PH_COUNT = 7 };
struct PhaseScope {
  int ph; cudaStream_t st; void* a; long long l0;
  PhaseScope(int ph, cudaStream_t st);
  ~PhaseScope();
};

// Lift the dynamic shared-memory limit of a kernel to the device maximum
// (once per kernel and device).
void set_max_smem(const void* fn);
int device_max_smem();

// twiddle table (per device, built once)
template <typename T> const Cx<T>* twiddles(int device);

// matvec / spectrum
// Series products of one code path `mode` (mv1d_mode): every item shares it.
template <typename T>
void launch_mv1d(const MvItem<T>* items, int n, int max_log2Mx, int s, const Cx<T>* tw, cudaStream_t st, int mode);
// Forward transforms of the window-side vector shared by the X^T u products.
template <typename T>
void launch_uspec(const UzItem<T>* items, int n, int max_log2M, int s, const Cx<T>* tw, cudaStream_t st);

// Bulk-copy waits in the series product that gave up since the last call
// (each sets a device counter instead of spinning on); read and reset, -1 on
// a CUDA error.  Synchronises the stream.
int mv_async_timeouts(cudaStream_t st);
// y-pass blocks that refused a tile larger than their launch's staging
// buffers (a sizing fault of the host, reported rather than run) since the
// last call; read and reset, -1 on a CUDA error.
int ypass_bad_tiles(cudaStream_t st);

// y-pass blocks stage tk x-frequencies (all My rows) in two buffers of
// YPASS_BUF_BYTES (grown to one padded column where a column is larger), so
// three blocks fit an SM.  tk: x-frequencies per block, 1..64.
constexpr int YPASS_BUF_BYTES = 36 * 1024;
template <typename T>
inline int ypass_tk(int log2My) {
  const int buf = YPASS_BUF_BYTES / (int)sizeof(Cx<T>);
  int tk = buf / padded_len(1 << log2My);
  return tk < 1 ? 1 : (tk > 64 ? 64 : tk);
}
// buffer elements of a y-pass launch whose largest grid has 2^max_log2My rows
template <typename T>
inline int ypass_buf(int max_log2My) {
  const int b = YPASS_BUF_BYTES / (int)sizeof(Cx<T>), c = padded_len(1 << max_log2My);
  return b > c ? b : c;
}
// blocks of one y-pass item: ceil((H + 1) / tk)
inline int ypass_blocks(int log2Mx, int tk) { return ((1 << (log2Mx - 1)) + 1 + tk - 1) / tk; }

// 2D products: tiles of the x-pass forward (y_in_hi blocks per item), the
// y-pass (ypass_blocks) and the x-pass inverse (y_out_hi blocks).
// max_buf: the largest tk * padded_len(My) among the y-pass items (complex
// elements), which sizes the launch's staging buffers with ypass_buf
template <typename T>
void launch_mv2d(const MvItem<T>* items, const YItem<T>* yitems, int n, Tiles xf, Tiles yp, Tiles xi,
                 int max_log2Mx, int max_log2My, int s, const Cx<T>* tw, cudaStream_t st, int max_buf);
template <typename T>
void launch_ypass(const YItem<T>* items, Tiles tl, int mode, int max_log2My, int s, const Cx<T>* tw,
                  cudaStream_t st, int max_buf);
// spectra: sx gives ny blocks per item, sy ypass_blocks per 2D item
template <typename T>
void launch_spec(const SpecItem<T>* items, Tiles sx, const YItem<T>* yitems, Tiles sy, int max_log2Mx,
                 int max_log2My, const Cx<T>* tw, cudaStream_t st, int max_buf);

}  // namespace ssa
