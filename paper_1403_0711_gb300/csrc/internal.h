// Internal types shared by the host API and the kernel launchers.
#pragma once

#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>
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

// Round keys of Philox4x32-10's Weyl schedule: (k0 + r W0, k1 + r W1), r = 0..9.
struct PhiloxKeys {
  uint32_t k[20];
};

__host__ __device__ inline PhiloxKeys philox_keys(uint32_t k0, uint32_t k1) {
  PhiloxKeys K;
  for (int r = 0; r < 10; ++r) {
    K.k[2 * r] = k0 + (uint32_t)r * 0x9E3779B9u;
    K.k[2 * r + 1] = k1 + (uint32_t)r * 0xBB67AE85u;
  }
  return K;
}

// Number of chains chain0, chain0 + stride, ... below n_chains (grid z).
inline unsigned launch_chains(int n_chains, int chain0, int stride) {
  return chain0 >= n_chains || stride < 1 ? 0u : (unsigned)((n_chains - chain0 + stride - 1) / stride);
}

struct SweepArgs {
  void *field;
  int Lx, Ly, Lz, W, Wq, QW, TY, DZ;
  int colour;
  // chains of the launch: chain0, chain0 + chain_stride, ... < n_chains
  // (grid z runs over them)
  int chain0, chain_stride;
  uint32_t round_keys[20];  // Philox round keys of the lattice's seed
  const uint32_t *pass_ptr;  // device pass counter
  uint32_t pass_off;         // added to *pass_ptr
  size_t chain_elems, colour_elems;
  int *err;
  // Fused gather (used on the last half-sweep of a measured compound sweep;
  // null otherwise).  Charges are grouped by (y tile, z plane) of the launch's
  // tile shape: entries of tile column ty_idx and plane z are
  // [g_off[ty_idx*Lz + z], g_off[ty_idx*Lz + z + 1]).  An entry packs the
  // colour in bit 31 and the site's offset within its colour's array,
  // (z*Ly + y)*W + h (h = x >> 1), in bits 0..30.
  const uint32_t *g_off;
  const uint32_t *g_ent;
  const double *g_q;
  double *g_partials;  // [chain][y tiles * z slabs][2]
};

// Fused pass (pass_fused.cu): both half-sweeps of one pass, colour 0 then
// colour 1, read from src and written to dst (two copies of the field, same
// layout).  TMA maps are built on src with boxes of TY + 4 rows (colour 1)
// and TY + 2 rows (colour 0).
struct PassArgs {
  void *dst;
  int Lx, Ly, Lz, W, Wq, QW, TY, DZ;
  int chain0, chain_stride;  // chains of the launch, as in SweepArgs
  uint32_t round_keys[20];
  const uint32_t *pass_ptr;
  uint32_t pass_off;
  size_t chain_elems, colour_elems;
  int *err;
  // Fused gather on the last kernel of a measured compound sweep (null
  // otherwise), grouped by (y tile, z plane) of this kernel's tile as in
  // SweepArgs; both colours are read from dst.
  const uint32_t *g_off;
  const uint32_t *g_ent;
  const double *g_q;
  double *g_partials;  // [chain][y tiles * z slabs][2]
};
cudaError_t launch_pass(const Geometry &g, const Tile &t, const CUtensorMap &tm_c1,
                        const CUtensorMap &tm_c0, const PassArgs &a, bool overrelax,
                        cudaStream_t s);
int pass_threads(const Geometry &g, const Tile &t);
size_t pass_smem_bytes(const Geometry &g, const Tile &t, bool overrelax);

// Pass pair (pass_pair.cu): two consecutive passes A (pass index
// *pass_ptr + pass_off) and B (the next) in one z-march from src to dst, each
// site read and written once for both.  TMA maps on src with boxes of TY + 8
// rows (colour 1) and TY + 6 rows (colour 0, read when A is over-relaxation).
cudaError_t launch_pair(const Geometry &g, const Tile &t, const CUtensorMap &tm_c1,
                        const CUtensorMap &tm_c0, const PassArgs &a, bool a_or, bool b_or,
                        cudaStream_t s);
int pair_threads(const Geometry &g, const Tile &t);
size_t pair_smem_bytes(const Geometry &g, const Tile &t, bool a_or);
// largest thread count of a pair CTA (FP32 / FP64)
constexpr int kPairMaxThreads32 = 512, kPairMaxThreads64 = 256;

// Phase-shifted schedule: chain k belongs to group k % groups; per group the
// launch does nothing (mode 0), a heatbath (1) or an over-relaxation (2)
// half-sweep with pass index *pass_ptr + pass_delta, gathering Q, P if
// gather != 0.
constexpr int kMaxGroups = 8;
struct MixedArgs {
  SweepArgs base;  // pass_off and g_* of base are ignored except g_off/g_ent/g_q/g_partials
  int groups;
  int mode[kMaxGroups];
  uint32_t pass_delta[kMaxGroups];
  int gather[kMaxGroups];
};
cudaError_t launch_halfsweep_mixed(const Geometry &g, const Tile &t, const CUtensorMap &tm_halo,
                                   const CUtensorMap &tm_own, const MixedArgs &a, cudaStream_t s);
// the gather for the chains first, first + stride, ... only
cudaError_t launch_gather_group(const Geometry &g, const void *field, const uint32_t *idx,
                                const double *q, int64_t n, double *partials, int nblk, int first,
                                int stride, cudaStream_t s);
cudaError_t launch_finalize_group(const double *partials, int nblk, int n_chains, int first,
                                  int stride, double *stats, double *log, int64_t log_cap,
                                  int *err, cudaStream_t s);

// Several charge sets measured on the same fields in one gather launch and one
// finalize launch (per set: its storage offsets, charges, CTA partials,
// blocks per chain, estimator state and optional log).
constexpr int kMaxSets = 32;
struct SetTable {
  const uint32_t *idx[kMaxSets];
  const double *q[kMaxSets];
  int64_t n[kMaxSets];
  double *partials[kMaxSets];
  int nblk[kMaxSets];
  double *stats[kMaxSets];
  double *log[kMaxSets];
  int64_t log_cap[kMaxSets];
  int n_sets;
};
cudaError_t launch_measure_sets(const Geometry &g, const void *field, const SetTable &t,
                                int *err, cudaStream_t s);

// Global control variate (gcv.cu).  gcv_solve: red/black SOR on A u = -rho
// (natural order, FP64, u_nat and rho_nat Lx*Ly*Lz doubles), h32 = u rounded
// to a fixed-point grid (exact FP32), v_layout = A h32 (exact in FP32) in one
// chain's field layout (chain_elems floats), res[0] = h32 . rho,
// res[1] = |A u + rho| / |rho|, res[2] = max |u| (res: 3 doubles); scratch
// >= 4 * nblk_red doubles; synchronises once.  gcv_eval: per chain
// T g = res[0] - Q (v . phi) into tg; partials >= 2 * nblk * n_chains
// doubles, nblk = gcv_blocks(g).
int gcv_blocks(const Geometry &g);
// Dirichlet Green function of the (2R+1)^3 cube at its centre (FP32,
// [dz][dy][dx] from -R; api.cu), the local P term's kernel.
std::vector<float> cube_green(int R);
cudaError_t gcv_solve(const Geometry &g, const double *rho_nat, double *u_nat, float *h32,
                      float *v_layout, double *scratch, int nblk_red, int n_iter, double *res,
                      cudaStream_t s);
// With R > 0 also the local term of P (kt: (2R+1)^3 floats, index
// (dz + R)(2R+1)^2 + (dy + R)(2R+1) + dx + R; cP = kt[centre] sum q^2; ppart
// >= ceil(n_q / 8) * n_chains doubles).
cudaError_t gcv_eval(const Geometry &g, const void *field, const float *v_layout,
                     const uint32_t *idx, const double *q, int64_t n_q, double *partials,
                     int nblk, const double *c0, const float *kt, int R, double cP,
                     double *ppart, double *tg, cudaStream_t s, cudaStream_t side,
                     cudaEvent_t fork, cudaEvent_t join);

// Entry packing of the fused gather.
constexpr uint32_t kGatherColourBit = 0x80000000u;

// Estimator state, per chain, in doubles.
constexpr int kBatchMin = 32;  // batches kept per chain: between kBatchMin and 2*kBatchMin
constexpr int kStatN = 0, kStatSum = 1, kStatSum2 = 2, kStatCurSum = 3, kStatCurN = 4,
              kStatBatchLen = 5, kStatNBatch = 6, kStatLast = 7, kStatBatch0 = 8;
constexpr int kStatStride = kStatBatch0 + 2 * kBatchMin;
static_assert(kStatStride == COULPS_STAT_STRIDE, "stat layout");

struct Allocator {
  coulps_alloc_fn alloc;
  coulps_free_fn free_fn;
  void *ctx;
};

// cuTensorMapEncodeTiled from the driver, looked up once (NULL if missing).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

// The allocation hooks installed by coulps_set_allocator (NULLs = default).
Allocator current_allocator();

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
// The same gather over all chains with offsets checked on the device: an
// offset >= chain_elems is skipped and counted in *bad (device memory).
cudaError_t launch_gather_checked(const Geometry &g, const void *field, const uint32_t *idx,
                                  const double *q, int64_t n, double *partials, int nblk,
                                  unsigned *bad, cudaStream_t s);
// Off-lattice charge sets (trilinear weights over eight corner sites; per
// particle 8 storage offsets, 8 weights, 8 x 3 weight gradients).
// off-lattice sets: partial blocks of a chain are `row` apart; the gather
// fills blocks [0, nblk) and (tout != NULL) keeps t_i = q_i phi~_i per chain;
// launch_near fills blocks [first, first + near_blocks(n)) with (0, s_N).
cudaError_t launch_gather_off(const Geometry &g, const void *field, const uint32_t *oidx,
                              const double *ow, const double *q, int64_t n, double *partials,
                              int nblk, int row, double *tout, cudaStream_t s);
int near_blocks(int64_t n);
cudaError_t launch_near(const double *t, const int64_t *nptr, const uint32_t *nbr, int64_t n,
                        int n_chains, double *u, double *partials, int row, int first,
                        cudaStream_t s);
cudaError_t launch_force_off(const Geometry &g, const void *field, const uint32_t *oidx,
                             const double *ow, const double *og, const double *q, int64_t n,
                             const double *Qc, const double *u, double *fsum, cudaStream_t s);
cudaError_t launch_finalize(const double *partials, int nblk, int n_chains, double *stats,
                            double *log, int64_t log_cap, int *err, cudaStream_t s,
                            double *Qout = nullptr);
cudaError_t launch_reset_stats(double *stats, int n_chains, cudaStream_t s);
// cv[chain] gets the sample y = e_last - c * tg[chain], e_last the chain's
// most recent Eq. (nsum2) sample in stats
cudaError_t launch_cv_record(const double *stats, const double *tg, double c, double *cv,
                             int n_chains, int *err, cudaStream_t s);

int gather_blocks(int64_t n);

// Control variate input packing (cv_ops.cu) for a lattice's FP32 field.
int coulps_cv_pack_field_impl(const void *field, const Geometry &g, const float *rho,
                              void *act_bf16, float *Aphi, const int *origin, const int *dims,
                              int interleave, cudaStream_t s);

}  // namespace coulps
