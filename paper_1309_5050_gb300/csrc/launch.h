// Host-side entry points of the kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>
#include "kernels.cuh"

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
template <typename T>
void launch_mv1d(const MvItem<T>* items, int n, int max_log2Mx, int s, const Cx<T>* tw, cudaStream_t st);
template <typename T>
void launch_mv2d(const MvItem<T>* items, const YItem<T>* yitems, int n, int max_log2Mx, int max_log2My,
                 int max_y_in, int max_y_out, int s, const Cx<T>* tw, cudaStream_t st);
template <typename T>
void launch_ypass(const YItem<T>* items, int n, int mode, int max_log2Mx, int max_log2My, int s,
                  const Cx<T>* tw, cudaStream_t st);
template <typename T>
void launch_spec(const SpecItem<T>* items, int n, const YItem<T>* yitems, int ny, int max_log2Mx, int max_log2My,
                 int max_ny, const Cx<T>* tw, cudaStream_t st);

}  // namespace ssa
