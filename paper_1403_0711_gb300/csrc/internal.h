// Internal types shared by the host API and the kernel launchers.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/coulps.h"

namespace coulps {

// Bits of the per-lattice device error word.
constexpr int kErrTimeout = 1;
constexpr int kErrNonFinite = 2;

// Field storage of one lattice (all chains):
//   field[chain][colour][z][y][h],  h in [0, W)
// colour c = (x + y + z) & 1, and site x of row (y, z) of colour c sits at
// h = x >> 1 (the row holds x = 2h + ((c + y + z) & 1)).  W is ceil(Lx/2)
// rounded up to whole 4-site quads and to 32 bytes; elements past the last
// site of a row are kept at zero, which doubles as the phi = 0 ghost beyond
// x = Lx - 1.  The ghosts at y = -1, Ly and z = -1, Lz are supplied by the
// TMA unit's out-of-bounds zero fill.
struct Geometry {
  int Lx, Ly, Lz;
  int n_chains;
  int precision;  // COULPS_F32 / COULPS_F64
  int es;         // element size in bytes
  int W;          // row stride in elements
  int Wq;         // logical quads per row, ceil(Lx / 8) (RNG numbering)
  size_t colour_elems;  // Lz * Ly * W
  size_t chain_elems;   // 2 * colour_elems
};

struct Tile {
  int ty;  // rows of y per CTA
  int dz;  // planes of z per CTA
};

struct SweepArgs {
  void *field;
  int Lx, Ly, Lz, W, Wq, QW, TY, DZ;
  int colour;
  uint32_t seed_lo, seed_hi;
  const uint32_t *pass_ptr;  // device pass counter
  uint32_t pass_off;         // added to *pass_ptr
  size_t chain_elems, colour_elems;
  int *err;
};

// Estimator state, per chain, in doubles.
constexpr int kBatchMin = 32;  // batches kept per chain: between kBatchMin and 2*kBatchMin
constexpr int kStatN = 0, kStatSum = 1, kStatSum2 = 2, kStatCurSum = 3, kStatCurN = 4,
              kStatBatchLen = 5, kStatNBatch = 6, kStatBatch0 = 8;
constexpr int kStatStride = kStatBatch0 + 2 * kBatchMin;
static_assert(kStatStride == COULPS_STAT_STRIDE, "stat layout");

struct Allocator {
  coulps_alloc_fn alloc;
  coulps_free_fn free_fn;
  void *ctx;
};

void *dev_alloc(const Allocator &a, size_t bytes, cudaStream_t s);
void dev_free(const Allocator &a, void *p, cudaStream_t s);

// Launchers (return cudaError_t of the launch).
cudaError_t launch_halfsweep(const Geometry &g, const Tile &t, const CUtensorMap &tm_halo,
                             const CUtensorMap &tm_own, const SweepArgs &a, bool overrelax,
                             cudaStream_t s);
size_t halfsweep_smem_bytes(const Geometry &g, const Tile &t, bool overrelax);
cudaError_t launch_advance_pass(uint32_t *pass, uint32_t n, cudaStream_t s);

cudaError_t launch_gather(const Geometry &g, const void *field, const uint32_t *idx,
                          const double *q, int64_t n, double *partials, int nblk,
                          cudaStream_t s);
cudaError_t launch_finalize(const double *partials, int nblk, int n_chains, double *stats,
                            double *log, int64_t log_cap, int *err, cudaStream_t s);
cudaError_t launch_reset_stats(double *stats, int n_chains, cudaStream_t s);

int gather_blocks(int64_t n);

}  // namespace coulps
