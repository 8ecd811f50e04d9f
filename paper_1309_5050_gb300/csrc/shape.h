// Host-side entry points of the shape / weight kernels (internal).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ssa {

// Batched forms: one launch for many grids (blockIdx.z = item).
struct ObsItem {
  const void* data; int32_t data_double, nx, ny, words;
  uint32_t* bits; int* err;
  double* sq;               // per block of the item: sum of the squared observed values
};
// ||x||_2 of one problem from the observation kernel's block sums (fixed order)
struct NormItem { const double* sq; int64_t n; double* out; };
// Window columns that are one run of elements [a, b] (every rectangle, disc
// or triangle) let the origin and weight tests count set bits in a range
// from per-word prefix counts instead of matching every window word.
struct OriginItem {
  const uint32_t* obs; int32_t nwords_obs; int32_t wwords;
  const uint32_t* wrows; int32_t ey, cx, cy, kwords;
  uint32_t* kbits;
  const int32_t* opre;      // observed bits: per column, prefix popcounts of words (nwords_obs + 1)
  const int32_t* wint;      // per window column: a, b (a < 0: empty column)
  int32_t interval;         // 1: every window column is a run (opre, wint valid)
  int32_t pad_;
};
struct CountItem {            // per-column popcounts and their exclusive scan
  const uint32_t* bits; int32_t words, ncols;
  int32_t* cnt; int32_t* colbase; int32_t* total;
};
struct WeightItem {
  const uint32_t* kbits; int32_t kwords, kcols;
  const uint32_t* rrows; int32_t rwords, ex, ey, nx, ny, nwords;
  int32_t* w; uint32_t* nbits;
  const int32_t* kpre;      // origin bits: per column, prefix popcounts of words (kwords + 1)
  const int32_t* wint;
  int32_t interval;
  int32_t pad_;
};
struct PrefixItem {           // per-column exclusive prefix popcounts of a bit set
  const uint32_t* bits; int32_t words, ncols;
  int32_t* pre;               // ncols x (words + 1)
};
void launch_prefix_batch(const PrefixItem* it, const int32_t* pre, int n, int tiles, cudaStream_t st);
// pre: item i owns blocks [pre[i], pre[i+1]) (tiles = pre[n]): obs and
// weights ceil(nx/256) * ny, origins ceil(cx/256) * cy, counts and prefixes
// one block per column.
void launch_obs_batch(const ObsItem* it, const int32_t* pre, int n, int tiles, cudaStream_t st);
void launch_norm_batch(const NormItem* it, int n, cudaStream_t st);
void launch_origins_batch(const OriginItem* it, const int32_t* pre, int n, int tiles, cudaStream_t st);
void launch_counts_batch(const CountItem* it, const int32_t* pre, int n, int tiles, cudaStream_t st);
void launch_weights_batch(const WeightItem* it, const int32_t* pre, int n, int tiles, cudaStream_t st);

void launch_obs_bits(const void* data, int data_double, const uint8_t* mask, int nx, int ny, int words,
                     uint32_t* bits, int* err, cudaStream_t st);
void launch_origins(const uint32_t* obs, int nwords_obs, const uint32_t* wrows, int wwords, int ey, int cx,
                    int cy, int kwords, uint32_t* kbits, cudaStream_t st);
void launch_col_counts(const uint32_t* bits, int words, int ncols, int32_t* cnt, int32_t* colbase,
                       cudaStream_t st);
void launch_weights(const uint32_t* kbits, int kwords, int kcols, const uint32_t* rrows, int rwords, int ex,
                    int ey, int nx, int ny, int32_t* w, uint32_t* nbits, int nwords, cudaStream_t st);
}  // namespace ssa
