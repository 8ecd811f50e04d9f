// Host-side entry points of the shape / weight kernels (internal).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ssa {
void launch_obs_bits(const void* data, int data_double, const uint8_t* mask, int nx, int ny, int words,
                     uint32_t* bits, int* err, cudaStream_t st);
void launch_origins(const uint32_t* obs, int nwords_obs, const uint32_t* wrows, int wwords, int ey, int cx,
                    int cy, int kwords, uint32_t* kbits, cudaStream_t st);
void launch_col_counts(const uint32_t* bits, int words, int ncols, int32_t* cnt, int32_t* colbase,
                       cudaStream_t st);
void launch_weights(const uint32_t* kbits, int kwords, int kcols, const uint32_t* rrows, int rwords, int ex,
                    int ey, int nx, int ny, int32_t* w, uint32_t* nbits, int nwords, cudaStream_t st);
}  // namespace ssa
