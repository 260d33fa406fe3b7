// Many independent systems of uneven size in one launch per half-sweep.
//
// Each system is its own lattice (own box, own charge set, one chain) with
// its own estimator.  The work of one half-sweep over all systems is a list
// of tiles (system, y0, z0, nz), ordered by system; a persistent grid (as
// many CTAs as fit on the GPU at once) walks the list with a fixed stride, so
// every CTA streams a sequence of tiles of different systems through one
// shared-memory TMA ring (tile_march.cuh), with the mbarrier phases carried
// from tile to tile.  Each system has its own pair of 4D tensor maps, kept in
// global memory, and its own tile shape (ty rows, dz planes), chosen by the
// caller or the autotuner.  The measured compound sweep gathers Q, P in its
// last half-sweep (one partial per tile) and a finalize kernel adds each
// system's partials in tile order.  The whole measured compound sweep is one
// CUDA graph.
//
// Fused over-relaxation passes (coulps_batch_set_fused): the
// over-relaxation passes run from one copy of the fields to a second one and
// back, either as fused passes (both half-sweeps of a pass in one z-march,
// pass_march.cuh; mode 1) or as pass pairs (two passes in one z-march,
// pair_march.cuh) with a fused pass for an odd remainder (mode 2, the
// default where every system admits a pair tile), by persistent kernels that
// walk lists of tiles (each system with its own tile shapes and tensor maps
// on both copies).  The heatbath passes stay half-sweeps, written out of
// place into the second copy when the count of out-of-place kernels is odd,
// so that the compound sweep ends in the first copy.  The sample is gathered
// by the last kernel.  Pair tiles vary about tenfold in size between
// systems, so the pair kernel takes them largest first from an atomic
// counter rather than by a fixed stride.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "batch_internal.h"
#include "device_common.cuh"
#include "internal.h"
#include "pair_march.cuh"
#include "pass_march.cuh"
#include "tile_march.cuh"

namespace coulps {
namespace {

using namespace tile;

constexpr int kBatchThreads = 256;
constexpr int kBatchPassThreads = 256;

// Dynamic tile scheduler of the persistent kernels: a CTA takes the next
// tile of the launch's list (tiles ordered largest first) from ctr[0]; after
// its last fetch it counts itself in ctr[1], and the last CTA of the grid
// sets both back to 0 for the next launch (launches on the batch's stream
// never overlap).  Partials are stored by tile index, so sums do not depend
// on which CTA ran a tile.
__device__ __forceinline__ int next_tile(int *ctr, const int *order, int n_items) {
  __shared__ int slot;
  if (threadIdx.x == 0) slot = atomicAdd(&ctr[0], 1);
  __syncthreads();
  const int k = slot;
  __syncthreads();  // every thread has read slot before the next fetch
  return k < n_items ? order[k] : -1;
}

__device__ __forceinline__ void tiles_done(int *ctr) {
  if (threadIdx.x == 0) {
    __threadfence();  // this CTA's last fetch comes before its count
    if (atomicAdd(&ctr[1], 1) == (int)gridDim.x - 1) {
      ctr[0] = 0;
      ctr[1] = 0;
    }
  }
}

struct BatchArgs {
  void *field;  // written: the own colour of each tile
  const BatchSystem *sys;
  const BatchItem *items;
  int n_items;
  const CUtensorMap *maps;  // 2 per system: other-colour box (TY+2 rows), own box (TY rows)
  const int *order;         // tile indices, largest tile first
  int *ctr;                 // scheduler counters (next_tile)
  int colour;
  uint32_t round_keys[20];
  const uint32_t *pass_ptr;
  uint32_t pass_off;
  int *err;
  const uint32_t *g_off, *g_ent;
  const double *g_q;
  double *g_partials;  // [item][2]
};

// V quads per thread (march_tile): 2 for the FP32 heatbath half-sweep
// without a gather (issue-bound, as in the single-lattice kernel), else 1.
template <typename T, bool OR, bool GATHER>
constexpr int batch_quads_per_thread() {
  return (sizeof(T) == 4 && !OR && !GATHER) ? 2 : 1;
}

template <typename T, bool OR, bool GATHER, int V>
__global__ void __launch_bounds__(kBatchThreads) batch_halfsweep_kernel(const BatchArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = align_smem128(smem_raw);
  const PhiloxKeys &K = *reinterpret_cast<const PhiloxKeys *>(a.round_keys);
  const uint32_t pass = OR ? 0u : (*a.pass_ptr + a.pass_off);
  int gbase = 0;
  ring_init(smem);
  for (int it; (it = next_tile(a.ctr, a.order, a.n_items)) >= 0;) {
    const BatchItem item = a.items[it];
    const BatchSystem S = a.sys[item.sys];
    TileJob<T> j;
    j.tm_halo_ = &a.maps[2 * item.sys];
    j.tm_own_ = &a.maps[2 * item.sys + 1];
    j.colour_ = a.colour;
    j.map_other_ = a.colour ^ 1;
    j.map_own_ = a.colour;
    j.out_ = reinterpret_cast<T *>(a.field) + S.field_off + (long long)a.colour * S.colour_elems;
    j.Lx_ = S.Lx; j.Ly_ = S.Ly; j.Lz_ = S.Lz; j.W_ = S.W; j.Wq_ = S.Wq; j.QW_ = S.QW; j.TY_ = S.TY;
    j.y0_ = item.y0;
    j.z0_ = item.z0;
    j.nz_ = item.nz;
    j.rng_id_ = (uint32_t)item.sys;
    j.pass_ = pass;
    if (GATHER) {
      j.g_off_ = a.g_off + S.goff_base + (size_t)(item.y0 / S.TY) * S.Lz;
      j.g_ent_ = a.g_ent;
      j.other_ = reinterpret_cast<const T *>(a.field) + S.field_off +
                (long long)(a.colour ^ 1) * S.colour_elems;
      j.g_q_ = a.g_q;
    }
    double sq = 0.0, sp = 0.0;
    const bool ok = march_tile<T, OR, GATHER, V>(j, K, smem, a.err, gbase, sq, sp);
    if (GATHER) block_partials(sq, sp, smem, a.g_partials + 2 * (size_t)it);
    if (!ok) break;
  }
  tiles_done(a.ctr);
}

// Fused passes over all systems: a persistent grid walks the pass tiles
// (system, y0, z0, nz), each CTA running march_pass tile after tile with its
// ring phases carried over; the source copy's tensor maps are 2 per system
// (colour-1 box PTY + 4 rows, colour-0 box PTY + 2 rows), dst the other copy.
struct BatchPassArgs {
  void *dst;
  const BatchSystem *sys;
  const BatchItem *items;
  const int *order;  // tile indices, largest tile first
  int *ctr;          // scheduler counters (next_tile)
  int n_items;
  const CUtensorMap *maps;
  uint32_t round_keys[20];
  const uint32_t *pass_ptr;
  uint32_t pass_off;
  int *err;
  const uint32_t *g_off, *g_ent;  // grouped by (pass y tile, z) per system
  const double *g_q;
  double *g_partials;  // [pass tile][2]
};

template <typename T, bool OR, bool GATHER>
__global__ void __launch_bounds__(kBatchPassThreads) batch_pass_kernel(const BatchPassArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = align_smem128(smem_raw);
  const PhiloxKeys &K = *reinterpret_cast<const PhiloxKeys *>(a.round_keys);
  const uint32_t pass = OR ? 0u : (*a.pass_ptr + a.pass_off);
  int gbase = 0;
  pass_ring_init(smem);
  for (int it; (it = next_tile(a.ctr, a.order, a.n_items)) >= 0;) {
    const BatchItem item = a.items[it];
    const BatchSystem S = a.sys[item.sys];
    PassTile<T> j;
    j.tm_c1_ = &a.maps[2 * item.sys];
    j.tm_c0_ = &a.maps[2 * item.sys + 1];
    j.map_c1_ = 1;
    j.map_c0_ = 0;
    j.dst_ = reinterpret_cast<T *>(a.dst) + S.field_off;
    j.colour_elems_ = S.colour_elems;
    j.Lx_ = S.Lx; j.Ly_ = S.Ly; j.Lz_ = S.Lz; j.W_ = S.W; j.Wq_ = S.Wq; j.QW_ = S.QW; j.TY_ = S.PTY;
    j.y0_ = item.y0;
    j.z0_ = item.z0;
    j.nz_ = item.nz;
    j.rng_id_ = (uint32_t)item.sys;
    j.pass_ = pass;
    j.g_off_ = GATHER ? a.g_off + S.pgoff_base + (size_t)(item.y0 / S.PTY) * S.Lz : nullptr;
    j.g_ent_ = a.g_ent;
    j.g_q_ = a.g_q;
    double sq = 0.0, sp = 0.0;
    const bool ok = march_pass<T, OR, GATHER>(j, K, smem, a.err, gbase, sq, sp);
    if (GATHER) block_partials(sq, sp, smem, a.g_partials + 2 * (size_t)it);
    if (!ok) break;
  }
  tiles_done(a.ctr);
}

// Over-relaxation pass pairs over all systems: a persistent grid (one CTA
// per SM) takes pair tiles (system, y0, z0, nz) in order of decreasing size
// from an atomic counter, each CTA running march_pair tile after tile with
// its ring phases carried over; the source copy's tensor maps are 2 per
// system (colour-1 box QTY + 8 rows, colour-0 box QTY + 6 rows), dst the
// other copy.  Partials are stored by tile index, so the gathered sums do
// not depend on which CTA ran a tile.
struct BatchPairArgs {
  void *dst;
  const uint32_t *pass_ptr;  // Philox pass of pass A: *pass_ptr + pass_off
  uint32_t pass_off;
  const BatchSystem *sys;
  const BatchItem *items;  // pair tiles in system order
  const int *order;        // tile indices, largest tile first
  int n_items;
  const CUtensorMap *maps;
  uint32_t round_keys[20];
  int *err;
  int *ctr;  // scheduler counters (next_tile)
  const uint32_t *g_off, *g_ent;  // grouped by (pair y tile, z) per system
  const double *g_q;
  double *g_partials;  // [pair tile][2]
};

template <typename T, bool A_OR, bool B_OR, bool GATHER>
__global__ void __launch_bounds__(sizeof(T) == 4 ? kPairMaxThreads32 : kPairMaxThreads64, 1)
    batch_pair_kernel(const BatchPairArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = align_smem128(smem_raw);
  const PhiloxKeys &K = *reinterpret_cast<const PhiloxKeys *>(a.round_keys);
  int gbase = 0;
  pair_ring_init(smem);
  for (int it; (it = next_tile(a.ctr, a.order, a.n_items)) >= 0;) {
    const BatchItem item = a.items[it];
    const BatchSystem S = a.sys[item.sys];
    PairTile<T> j;
    j.tm_c1_ = &a.maps[2 * item.sys];
    j.tm_c0_ = &a.maps[2 * item.sys + 1];
    j.map_c1_ = 1;
    j.map_c0_ = 0;
    j.dst_ = reinterpret_cast<T *>(a.dst) + S.field_off;
    j.colour_elems_ = S.colour_elems;
    j.Lx_ = S.Lx; j.Ly_ = S.Ly; j.Lz_ = S.Lz; j.W_ = S.W; j.Wq_ = S.Wq; j.QW_ = S.QW; j.TY_ = S.QTY;
    j.y0_ = item.y0;
    j.z0_ = item.z0;
    j.nz_ = item.nz;
    j.rng_id_ = (uint32_t)item.sys;
    j.pass_ = (A_OR && B_OR) ? 0u : (*a.pass_ptr + a.pass_off);
    j.g_off_ = GATHER ? a.g_off + S.qgoff_base + (size_t)(item.y0 / S.QTY) * S.Lz : nullptr;
    j.g_ent_ = a.g_ent;
    j.g_q_ = a.g_q;
    double sq = 0.0, sp = 0.0;
    const bool ok = march_pair<T, A_OR, B_OR, GATHER>(j, K, smem, a.err, gbase, sq, sp);
    if (GATHER) block_partials(sq, sp, smem, a.g_partials + 2 * (size_t)it);
    if (!ok) break;
  }
  tiles_done(a.ctr);
}

// Each system's tile partials added up by one warp (lane l takes tiles
// l, l + 32, ... of the system, then a fixed butterfly), for the tiling of
// the kernel that gathered; lane 0 records the sample.
__global__ void batch_finalize_kernel(const double *__restrict__ partials,
                                      const BatchSystem *__restrict__ sys, int n_sys, int n_items,
                                      int tiling, double *__restrict__ stats,
                                      double *__restrict__ log, int64_t log_cap, int *err) {
  const int s = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= n_sys) return;  // whole warps
  auto begin = [&](int t) {
    return tiling == kTilePair ? sys[t].qitem_begin
                               : (tiling == kTilePass ? sys[t].pitem_begin : sys[t].item_begin);
  };
  const int b0 = begin(s);
  const int b1 = s + 1 < n_sys ? begin(s + 1) : n_items;
  double Q = 0.0, P = 0.0;
  for (int b = b0 + lane; b < b1; b += 32) {
    Q += partials[2 * (size_t)b];
    P += partials[2 * (size_t)b + 1];
  }
  Q = warp_sum(Q);
  P = warp_sum(P);
  if (lane != 0) return;
  double *st = stats + (size_t)s * kStatStride;
  const int64_t k = (int64_t)st[kStatN];
  double *row = (log != nullptr && k < log_cap) ? log + 3 * ((size_t)k * n_sys + s) : nullptr;
  record_sample(st, Q, P, row, err);
}

__global__ void batch_reset_stats_kernel(double *stats, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * kStatStride) return;
  stats[i] = (i % kStatStride == kStatBatchLen) ? 1.0 : 0.0;
}

#define CK(expr)                          \
  do {                                    \
    cudaError_t e_ = (expr);              \
    if (e_ != cudaSuccess) {              \
      cudaGetLastError();                 \
      return COULPS_ECUDA;                \
    }                                     \
  } while (0)

}  // namespace
}  // namespace coulps

using namespace coulps;


namespace {

void batch_drop_graph(coulps_batch *B) {
  if (B->graph) cudaGraphExecDestroy(B->graph);
  B->graph = nullptr;
}

void release(coulps_batch *B, void *&p) {
  dev_free(B->alloc, p, B->stream);
  p = nullptr;
}

template <typename P>
void release(coulps_batch *B, P *&p) {
  void *v = p;
  release(B, v);
  p = nullptr;
}

int batch_row_stride(int Lx, int es) {
  const int a = 32 / es;
  return ((4 * ((Lx + 7) / 8) + a - 1) / a) * a;
}

size_t batch_smem_bytes(const coulps_batch *B, bool orx) {
  size_t m = 0;
  for (const auto &S : B->sys) {
    const SmemLayout lay = smem_layout(S.TY, S.W, B->es, orx);
    m = std::max(m, (size_t)lay.total);
  }
  return m + 128;
}

// 4D map over one system's fields [colour][z][y][h] at `base` with boxes of
// `rows` rows of W elements of one plane (zero fill outside the box).
int batch_map(const coulps_batch *B, const BatchSystem &S, void *field, int rows, CUtensorMap *m) {
  auto enc = tensor_map_encoder();
  if (!enc) return COULPS_ECUDA;
  cuuint64_t dims[4] = {(cuuint64_t)S.W, (cuuint64_t)S.Ly, (cuuint64_t)S.Lz, 2};
  cuuint64_t strides[3] = {(cuuint64_t)S.W * B->es, (cuuint64_t)S.W * S.Ly * B->es,
                           (cuuint64_t)S.colour_elems * B->es};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  void *base = (char *)field + (size_t)S.field_off * B->es;
  cuuint32_t box[4] = {(cuuint32_t)S.W, (cuuint32_t)rows, 1, 1};
  CUresult r = enc(m,
                   B->precision == COULPS_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                              : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                   4, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? COULPS_OK : COULPS_ECUDA;
}

// Gather lists of the charges grouped by (y tile, z) per system for the tile
// rows of one tiling: offsets `off` (system base + y tile * Lz + z) and
// entries (colour bit 31, offset within the colour's array).
void batch_gather_lists(const coulps_batch *B, int tiling, int n_off, std::vector<uint32_t> &off,
                        std::vector<uint32_t> &ent, std::vector<double> &gq) {
  off.assign((size_t)n_off + 1, 0);
  const int64_t ntot = B->offsets[B->n_sys];
  ent.assign((size_t)ntot, 0);
  gq.assign((size_t)ntot, 0.0);
  auto key = [&](const BatchSystem &S, int y, int z) {
    const int ty = tiling == kTilePair ? S.QTY : (tiling == kTilePass ? S.PTY : S.TY);
    const int base = tiling == kTilePair ? S.qgoff_base
                                         : (tiling == kTilePass ? S.pgoff_base : S.goff_base);
    return (size_t)base + (size_t)(y / ty) * S.Lz + z;
  };
  for (int s = 0; s < B->n_sys; ++s)
    for (int64_t i = B->offsets[s]; i < B->offsets[s + 1]; ++i)
      off[key(B->sys[s], B->sites[3 * i + 1], B->sites[3 * i + 2]) + 1]++;
  for (size_t k = 1; k < off.size(); ++k) off[k] += off[k - 1];
  std::vector<uint32_t> pos(off.begin(), off.end());
  for (int s = 0; s < B->n_sys; ++s) {
    const BatchSystem &S = B->sys[s];
    for (int64_t i = B->offsets[s]; i < B->offsets[s + 1]; ++i) {
      const int x = B->sites[3 * i], y = B->sites[3 * i + 1], z = B->sites[3 * i + 2];
      const uint32_t p = pos[key(S, y, z)]++;
      ent[p] = ((uint32_t)((x + y + z) & 1) << 31) |
               (uint32_t)(((size_t)z * S.Ly + y) * S.W + (x >> 1));
      gq[p] = B->q[i];
    }
  }
}

// Upload one set of gather lists (reallocated to their sizes).
int batch_upload_lists(coulps_batch *B, const std::vector<uint32_t> &off,
                       const std::vector<uint32_t> &ent, const std::vector<double> &gq,
                       uint32_t *&d_off, uint32_t *&d_ent, double *&d_q) {
  release(B, d_off);
  release(B, d_ent);
  release(B, d_q);
  d_off = (uint32_t *)dev_alloc(B->alloc, off.size() * sizeof(uint32_t), B->stream);
  d_ent = (uint32_t *)dev_alloc(B->alloc, std::max<size_t>(1, ent.size()) * sizeof(uint32_t),
                                B->stream);
  d_q = (double *)dev_alloc(B->alloc, std::max<size_t>(1, gq.size()) * sizeof(double), B->stream);
  if (!d_off || !d_ent || !d_q) return COULPS_ENOMEM;
  CK(cudaMemcpyAsync(d_off, off.data(), off.size() * sizeof(uint32_t), cudaMemcpyHostToDevice,
                     B->stream));
  if (!ent.empty()) {
    CK(cudaMemcpyAsync(d_ent, ent.data(), ent.size() * sizeof(uint32_t), cudaMemcpyHostToDevice,
                       B->stream));
    CK(cudaMemcpyAsync(d_q, gq.data(), gq.size() * sizeof(double), cudaMemcpyHostToDevice,
                       B->stream));
  }
  return COULPS_OK;
}

size_t batch_pass_smem_bytes(const coulps_batch *B) {
  size_t m = 0;
  for (const auto &S : B->sys)
    m = std::max(m, (size_t)pass_layout(S.PTY, S.W, B->es, true).total);
  return m + 128;
}

int batch_pair_threads(int es) { return es == 4 ? kPairMaxThreads32 : kPairMaxThreads64; }

// A pair tile of ty rows fits: (ty + 6) rows of quads in one CTA, colour-1
// box rows <= 256, shared memory <= 227 KiB.
bool batch_pair_fits(const BatchSystem &S, int ty, int es) {
  return ty >= 1 && ty <= S.Ly && S.QW * (ty + 6) <= batch_pair_threads(es) && ty + 8 <= 256 &&
         pair_layout(ty, S.W, es, true).total + 128 <= 227 * 1024;
}

bool batch_pairs_ok(const coulps_batch *B) {
  for (const auto &S : B->sys)
    if (!batch_pair_fits(S, S.QTY, B->es)) return false;
  return true;
}

size_t batch_pair_smem_bytes(const coulps_batch *B) {
  size_t m = 0;
  for (const auto &S : B->sys)
    m = std::max(m, (size_t)pair_layout(S.QTY, S.W, B->es, true).total);
  return m + 128;
}

// Tile lists, tensor maps and gather lists for the current tile shapes.
int batch_layout(coulps_batch *B) {
  if (!B->layout_dirty) return COULPS_OK;
  batch_drop_graph(B);
  B->items.clear();
  B->pitems.clear();
  B->qitems.clear();
  const bool pairs = B->fused >= 2;
  int goff = 0, pgoff = 0, qgoff = 0;
  for (int s = 0; s < B->n_sys; ++s) {
    BatchSystem &S = B->sys[s];
    S.item_begin = (int)B->items.size();
    S.goff_base = goff;
    goff += ((S.Ly + S.TY - 1) / S.TY) * S.Lz;
    for (int z0 = 0; z0 < S.Lz; z0 += S.DZ)
      for (int y0 = 0; y0 < S.Ly; y0 += S.TY)
        B->items.push_back(BatchItem{s, y0, z0, std::min(S.DZ, S.Lz - z0)});
    S.pitem_begin = (int)B->pitems.size();
    S.pgoff_base = pgoff;
    pgoff += ((S.Ly + S.PTY - 1) / S.PTY) * S.Lz;
    for (int z0 = 0; z0 < S.Lz; z0 += S.PDZ)
      for (int y0 = 0; y0 < S.Ly; y0 += S.PTY)
        B->pitems.push_back(BatchItem{s, y0, z0, std::min(S.PDZ, S.Lz - z0)});
    S.qitem_begin = (int)B->qitems.size();
    S.qgoff_base = qgoff;
    if (pairs) {
      qgoff += ((S.Ly + S.QTY - 1) / S.QTY) * S.Lz;
      for (int z0 = 0; z0 < S.Lz; z0 += S.QDZ)
        for (int y0 = 0; y0 < S.Ly; y0 += S.QTY)
          B->qitems.push_back(BatchItem{s, y0, z0, std::min(S.QDZ, S.Lz - z0)});
    }
  }
  // each tile list largest first (sites of the tile, ties in list order)
  auto largest_first = [&](const std::vector<BatchItem> &items, int tiling) {
    std::vector<int> order(items.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    auto sites = [&](int i) {
      const BatchItem &t = items[i];
      const BatchSystem &S = B->sys[t.sys];
      const int ty = tiling == kTilePair ? S.QTY : (tiling == kTilePass ? S.PTY : S.TY);
      return (long long)std::min(ty, S.Ly - t.y0) * t.nz * S.Lx;
    };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return sites(x) > sites(y); });
    return order;
  };
  const std::vector<int> order = largest_first(B->items, kTileHalf);
  const std::vector<int> porder = largest_first(B->pitems, kTilePass);
  const std::vector<int> qorder = largest_first(B->qitems, kTilePair);
  // half-sweep maps on both copies (the second only with fused passes)
  std::vector<CUtensorMap> maps(4 * (size_t)B->n_sys);
  std::vector<CUtensorMap> pmaps(4 * (size_t)B->n_sys);
  std::vector<CUtensorMap> qmaps(4 * (size_t)B->n_sys);
  for (int c = 0; c < (B->field2 ? 2 : 1); ++c) {
    void *f = c ? B->field2 : B->field;
    for (int s = 0; s < B->n_sys; ++s) {
      const BatchSystem &S = B->sys[s];
      CUtensorMap *m = &maps[2 * ((size_t)c * B->n_sys + s)];
      int st = batch_map(B, S, f, S.TY + 2, &m[0]);
      if (!st) st = batch_map(B, S, f, S.TY, &m[1]);
      if (!st && B->field2) {
        CUtensorMap *pm = &pmaps[2 * ((size_t)c * B->n_sys + s)];
        st = batch_map(B, S, f, S.PTY + 4, &pm[0]);
        if (!st) st = batch_map(B, S, f, S.PTY + 2, &pm[1]);
      }
      if (!st && pairs) {
        CUtensorMap *qm = &qmaps[2 * ((size_t)c * B->n_sys + s)];
        st = batch_map(B, S, f, S.QTY + 8, &qm[0]);
        if (!st) st = batch_map(B, S, f, S.QTY + 6, &qm[1]);
      }
      if (st) return st;
    }
  }
  release(B, B->d_items);
  release(B, B->d_part);
  release(B, B->d_pitems);
  release(B, B->d_ppart);
  B->d_items = (BatchItem *)dev_alloc(B->alloc, B->items.size() * sizeof(BatchItem), B->stream);
  B->d_part = (double *)dev_alloc(B->alloc, B->items.size() * 2 * sizeof(double), B->stream);
  B->d_pitems = (BatchItem *)dev_alloc(B->alloc, B->pitems.size() * sizeof(BatchItem), B->stream);
  B->d_ppart = (double *)dev_alloc(B->alloc, B->pitems.size() * 2 * sizeof(double), B->stream);
  release(B, B->d_order);
  release(B, B->d_porder);
  B->d_order = (int *)dev_alloc(B->alloc, order.size() * sizeof(int), B->stream);
  B->d_porder = (int *)dev_alloc(B->alloc, porder.size() * sizeof(int), B->stream);
  if (!B->d_items || !B->d_part || !B->d_pitems || !B->d_ppart || !B->d_order || !B->d_porder)
    return COULPS_ENOMEM;
  CK(cudaMemcpyAsync(B->d_order, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice,
                     B->stream));
  CK(cudaMemcpyAsync(B->d_porder, porder.data(), porder.size() * sizeof(int),
                     cudaMemcpyHostToDevice, B->stream));
  release(B, B->d_qitems);
  release(B, B->d_qorder);
  release(B, B->d_qpart);
  if (pairs) {
    B->d_qitems = (BatchItem *)dev_alloc(B->alloc, B->qitems.size() * sizeof(BatchItem), B->stream);
    B->d_qorder = (int *)dev_alloc(B->alloc, qorder.size() * sizeof(int), B->stream);
    B->d_qpart = (double *)dev_alloc(B->alloc, B->qitems.size() * 2 * sizeof(double), B->stream);
    if (!B->d_qitems || !B->d_qorder || !B->d_qpart) return COULPS_ENOMEM;
    CK(cudaMemcpyAsync(B->d_qitems, B->qitems.data(), B->qitems.size() * sizeof(BatchItem),
                       cudaMemcpyHostToDevice, B->stream));
    CK(cudaMemcpyAsync(B->d_qorder, qorder.data(), qorder.size() * sizeof(int),
                       cudaMemcpyHostToDevice, B->stream));
    CK(cudaMemcpyAsync(B->d_qmaps, qmaps.data(), qmaps.size() * sizeof(CUtensorMap),
                       cudaMemcpyHostToDevice, B->stream));
  }
  CK(cudaMemcpyAsync(B->d_sys, B->sys.data(), B->sys.size() * sizeof(BatchSystem),
                     cudaMemcpyHostToDevice, B->stream));
  CK(cudaMemcpyAsync(B->d_items, B->items.data(), B->items.size() * sizeof(BatchItem),
                     cudaMemcpyHostToDevice, B->stream));
  CK(cudaMemcpyAsync(B->d_pitems, B->pitems.data(), B->pitems.size() * sizeof(BatchItem),
                     cudaMemcpyHostToDevice, B->stream));
  CK(cudaMemcpyAsync(B->d_maps, maps.data(), maps.size() * sizeof(CUtensorMap),
                     cudaMemcpyHostToDevice, B->stream));
  CK(cudaMemcpyAsync(B->d_pmaps, pmaps.data(), pmaps.size() * sizeof(CUtensorMap),
                     cudaMemcpyHostToDevice, B->stream));
  // gather lists for every tiling in use
  std::vector<uint32_t> off, ent, poff, pent, qoff, qent;
  std::vector<double> gq, pgq, qgq;
  if (B->has_charges) {
    batch_gather_lists(B, kTileHalf, goff, off, ent, gq);
    int st = batch_upload_lists(B, off, ent, gq, B->d_goff, B->d_gent, B->d_gq);
    if (st) return st;
    batch_gather_lists(B, kTilePass, pgoff, poff, pent, pgq);
    st = batch_upload_lists(B, poff, pent, pgq, B->d_pgoff, B->d_pgent, B->d_pgq);
    if (st) return st;
    if (pairs) {
      batch_gather_lists(B, kTilePair, qgoff, qoff, qent, qgq);
      st = batch_upload_lists(B, qoff, qent, qgq, B->d_qgoff, B->d_qgent, B->d_qgq);
      if (st) return st;
    }
  }
  // persistent grids: as many CTAs as are co-resident at the largest smem need
  B->smem = batch_smem_bytes(B, true);
  B->psmem = batch_pass_smem_bytes(B);
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int per_sm = std::max(1, std::min(8, (int)((200 * 1024) / B->smem)));
  B->grid = std::max(1, std::min((int)B->items.size(), sms * per_sm));
  // two quads per thread: ceil(QW / 2) threads a row, the widest tile's count
  B->threads2 = 32;
  for (const auto &S : B->sys)
    B->threads2 = std::max(B->threads2, (S.QW + 1) / 2 * S.TY);
  B->threads2 = (B->threads2 + 31) / 32 * 32;
  {
    int per_sm2 = 0;
    auto hk = B->precision == COULPS_F32 ? batch_halfsweep_kernel<float, false, false, 2>
                                         : batch_halfsweep_kernel<double, false, false, 2>;
    if (cudaFuncSetAttribute(hk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B->smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, hk, B->threads2, B->smem) !=
            cudaSuccess ||
        per_sm2 < 1) {
      cudaGetLastError();
      per_sm2 = per_sm;
    }
    B->grid2 = std::max(1, std::min((int)B->items.size(), sms * per_sm2));
  }
  // pass CTAs per SM: as many as registers, threads and shared memory allow
  int pper_sm = 0;
  auto pk = B->precision == COULPS_F32 ? batch_pass_kernel<float, true, false>
                                       : batch_pass_kernel<double, true, false>;
  if (cudaFuncSetAttribute(pk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B->psmem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pper_sm, pk, kBatchPassThreads, B->psmem) !=
          cudaSuccess ||
      pper_sm < 1) {
    cudaGetLastError();
    pper_sm = 1;
  }
  B->pgrid = std::max(1, std::min((int)B->pitems.size(), sms * pper_sm));
  // pair CTAs: one per SM (512 threads of over 100 registers each)
  if (pairs) {
    B->qsmem = batch_pair_smem_bytes(B);
    // the block: the widest pair tile's (QTY + 6) rows of quads, whole warps
    B->qthreads = 32;
    for (const auto &S : B->sys) B->qthreads = std::max(B->qthreads, S.QW * (S.QTY + 6));
    B->qthreads = (B->qthreads + 31) / 32 * 32;
    // CTAs per SM: the fewest over the pair kinds the mode runs
    auto per_sm_of = [&](const void *k) {
      int n = 0;
      if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B->qsmem) !=
              cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, B->qthreads, B->qsmem) !=
              cudaSuccess ||
          n < 1) {
        cudaGetLastError();
        n = 1;
      }
      return n;
    };
    const bool f32 = B->precision == COULPS_F32;
    int qper_sm = per_sm_of(f32 ? (const void *)batch_pair_kernel<float, true, true, false>
                                : (const void *)batch_pair_kernel<double, true, true, false>);
    if (B->fused == 3) {
      qper_sm = std::min(qper_sm, per_sm_of(f32 ? (const void *)batch_pair_kernel<float, false, true, false>
                                                : (const void *)batch_pair_kernel<double, false, true, false>));
      qper_sm = std::min(qper_sm, per_sm_of(f32 ? (const void *)batch_pair_kernel<float, false, false, false>
                                                : (const void *)batch_pair_kernel<double, false, false, false>));
    }
    B->qgrid = std::max(1, std::min((int)B->qitems.size(), sms * qper_sm));
  }
  CK(cudaStreamSynchronize(B->stream));  // host vectors leave scope
  B->layout_dirty = false;
  return COULPS_OK;
}

template <typename T, bool OR, bool GATHER>
cudaError_t launch_batch_t(coulps_batch *B, const BatchArgs &a) {
  constexpr int V = batch_quads_per_thread<T, OR, GATHER>();
  auto kfn = batch_halfsweep_kernel<T, OR, GATHER, V>;
  static size_t configured = 0;
  if (B->smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)B->smem);
    if (e != cudaSuccess) return e;
    configured = B->smem;
  }
  if (V == 2)
    kfn<<<B->grid2, B->threads2, B->smem, B->stream>>>(a);
  else
    kfn<<<B->grid, kBatchThreads, B->smem, B->stream>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_batch_p(coulps_batch *B, const BatchArgs &a, bool orx) {
  const bool gather = a.g_partials != nullptr;
  if (orx) return gather ? launch_batch_t<T, true, true>(B, a) : launch_batch_t<T, true, false>(B, a);
  return gather ? launch_batch_t<T, false, true>(B, a) : launch_batch_t<T, false, false>(B, a);
}

template <typename T, bool OR, bool GATHER>
cudaError_t launch_bpass_t(coulps_batch *B, const BatchPassArgs &a) {
  auto kfn = batch_pass_kernel<T, OR, GATHER>;
  static size_t configured = 0;
  if (B->psmem > configured) {
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)B->psmem);
    if (e != cudaSuccess) return e;
    configured = B->psmem;
  }
  kfn<<<B->pgrid, kBatchPassThreads, B->psmem, B->stream>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bpass_p(coulps_batch *B, const BatchPassArgs &a, bool orx) {
  const bool gather = a.g_partials != nullptr;
  if (orx) return gather ? launch_bpass_t<T, true, true>(B, a) : launch_bpass_t<T, true, false>(B, a);
  return gather ? launch_bpass_t<T, false, true>(B, a) : launch_bpass_t<T, false, false>(B, a);
}

template <typename T, bool A_OR, bool B_OR, bool GATHER>
cudaError_t launch_bpair_t(coulps_batch *B, const BatchPairArgs &a) {
  auto kfn = batch_pair_kernel<T, A_OR, B_OR, GATHER>;
  static size_t configured = 0;
  if (B->qsmem > configured) {
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)B->qsmem);
    if (e != cudaSuccess) return e;
    configured = B->qsmem;
  }
  kfn<<<B->qgrid, B->qthreads, B->qsmem, B->stream>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bpair_p(coulps_batch *B, const BatchPairArgs &a, bool a_or, bool b_or) {
  const bool gather = a.g_partials != nullptr;
  if (a_or)  // over-relaxation passes come after the heatbath passes: B too
    return gather ? launch_bpair_t<T, true, true, true>(B, a)
                  : launch_bpair_t<T, true, true, false>(B, a);
  if (b_or)
    return gather ? launch_bpair_t<T, false, true, true>(B, a)
                  : launch_bpair_t<T, false, true, false>(B, a);
  return gather ? launch_bpair_t<T, false, false, true>(B, a)
                : launch_bpair_t<T, false, false, false>(B, a);
}

cudaError_t launch_bpair(coulps_batch *B, const BatchPairArgs &a, bool a_or, bool b_or) {
  return B->precision == COULPS_F32 ? launch_bpair_p<float>(B, a, a_or, b_or)
                                    : launch_bpair_p<double>(B, a, a_or, b_or);
}

// One compound sweep of every system (and its sample when `measure`).  The
// passes [0, head) run as half-sweeps, then d pass pairs and s fused passes
// between the two copies, then the rest as in-place half-sweeps on the
// first copy.  fused = 1, 2: head = n_hb and the over-relaxation block runs
// as d = n_or / 2 pairs (fused = 2, else d = 0) and s = n_or - 2 d fused
// passes.  Every such kernel changes copy, so when d + s is odd the heatbath
// passes write the second copy (the first of them reading colour 1 from the
// first copy); with no heatbath pass one pair becomes two fused passes, or
// (no pair) the last pass runs as in-place half-sweeps.  fused = 3: all n
// passes as pairs and fused passes (head = 0; an even count of kernels, by
// n mod 4: n / 2 pairs; (n - 3) / 2 and 3; n / 2 - 1 and 2; (n - 1) / 2 and 1),
// half-sweeps only for n = 1.  The sweep ends in the first copy.
int batch_enqueue_compound(coulps_batch *B, int n_hb, int n_or, bool measure) {
  const int n = n_hb + n_or;
  int head = n_hb, d = 0, s = 0;
  bool flip = false;
  if (B->fused == 3 && B->field2 && n >= 2) {
    head = 0;
    switch (n % 4) {
      case 0: d = n / 2; s = 0; break;
      case 1: d = (n - 3) / 2; s = 3; break;
      case 2: d = n / 2 - 1; s = 2; break;
      default: d = (n - 1) / 2; s = 1; break;
    }
  } else if (B->fused && B->field2) {
    d = B->fused >= 2 ? n_or / 2 : 0;
    s = n_or - 2 * d;
    if ((d + s) % 2 == 1) {
      if (n_hb > 0) {
        flip = true;
      } else if (d >= 1) {
        d -= 1;
        s += 2;
      } else {
        s -= 1;
      }
    }
  }
  const int nf = 2 * d + s;  // passes run out of place
  const bool gather_fused = measure && nf > 0 && head + nf == n;
  const int gather_tiling = !gather_fused ? kTileHalf : (s > 0 ? kTilePass : kTilePair);
  BatchArgs a;
  std::memset(&a, 0, sizeof(a));
  a.sys = B->d_sys;
  a.items = B->d_items;
  a.order = B->d_order;
  a.ctr = B->d_ctr;
  a.n_items = (int)B->items.size();
  const PhiloxKeys K = philox_keys((uint32_t)(B->seed & 0xffffffffu), (uint32_t)(B->seed >> 32));
  for (int i = 0; i < 20; ++i) a.round_keys[i] = K.k[i];
  a.pass_ptr = B->d_pass;
  a.err = B->d_err;
  auto half_sweeps = [&](int i, bool on2, bool gather) -> int {
    const bool orx = i >= n_hb;
    for (int c = 0; c < 2; ++c) {
      a.colour = c;
      a.pass_off = (uint32_t)i;
      a.field = on2 ? B->field2 : B->field;
      // the other colour's rows: from the second copy once it holds them
      const bool halo2 = on2 && (i > 0 || c == 1);
      a.maps = B->d_maps + (halo2 ? 2 * (size_t)B->n_sys : 0);
      const bool last = gather && c == 1;
      a.g_off = last ? B->d_goff : nullptr;
      a.g_ent = last ? B->d_gent : nullptr;
      a.g_q = last ? B->d_gq : nullptr;
      a.g_partials = last ? B->d_part : nullptr;
      CK(B->precision == COULPS_F32 ? launch_batch_p<float>(B, a, orx)
                                    : launch_batch_p<double>(B, a, orx));
    }
    return COULPS_OK;
  };
  for (int i = 0; i < head; ++i) {
    const int r = half_sweeps(i, flip, measure && nf == 0 && i == n - 1);
    if (r) return r;
  }
  int src = flip ? 1 : 0;  // copy the next out-of-place kernel reads
  BatchPairArgs q;
  std::memset(&q, 0, sizeof(q));
  q.sys = B->d_sys;
  q.items = B->d_qitems;
  q.order = B->d_qorder;
  q.n_items = (int)B->qitems.size();
  for (int i = 0; i < 20; ++i) q.round_keys[i] = K.k[i];
  q.err = B->d_err;
  q.ctr = B->d_ctr;
  q.pass_ptr = B->d_pass;
  for (int t = 0; t < d; ++t, src ^= 1) {
    const int i = head + 2 * t;  // passes i (A) and i + 1 (B)
    q.pass_off = (uint32_t)i;
    q.dst = src ? B->field : B->field2;
    q.maps = B->d_qmaps + 2 * (size_t)src * B->n_sys;
    const bool last = gather_fused && s == 0 && t == d - 1;
    q.g_off = last ? B->d_qgoff : nullptr;
    q.g_ent = last ? B->d_qgent : nullptr;
    q.g_q = last ? B->d_qgq : nullptr;
    q.g_partials = last ? B->d_qpart : nullptr;
    CK(launch_bpair(B, q, i >= n_hb, i + 1 >= n_hb));
  }
  BatchPassArgs p;
  std::memset(&p, 0, sizeof(p));
  p.sys = B->d_sys;
  p.items = B->d_pitems;
  p.order = B->d_porder;
  p.ctr = B->d_ctr;
  p.n_items = (int)B->pitems.size();
  for (int i = 0; i < 20; ++i) p.round_keys[i] = K.k[i];
  p.pass_ptr = B->d_pass;
  p.err = B->d_err;
  for (int t = 0; t < s; ++t, src ^= 1) {
    const int i = head + 2 * d + t;
    const int b = src;
    p.dst = b ? B->field : B->field2;
    p.maps = B->d_pmaps + 2 * (size_t)b * B->n_sys;
    p.pass_off = (uint32_t)i;
    const bool last = gather_fused && t == s - 1;
    p.g_off = last ? B->d_pgoff : nullptr;
    p.g_ent = last ? B->d_pgent : nullptr;
    p.g_q = last ? B->d_pgq : nullptr;
    p.g_partials = last ? B->d_ppart : nullptr;
    CK(B->precision == COULPS_F32 ? launch_bpass_p<float>(B, p, i >= n_hb)
                                  : launch_bpass_p<double>(B, p, i >= n_hb));
  }
  for (int i = head + nf; i < n; ++i) {
    const int r = half_sweeps(i, false, measure && i == n - 1);
    if (r) return r;
  }
  if (n > 0) CK(launch_advance_pass(B->d_pass, (uint32_t)n, B->stream));
  if (measure) {
    const double *part = gather_tiling == kTilePair
                             ? B->d_qpart
                             : (gather_tiling == kTilePass ? B->d_ppart : B->d_part);
    const int n_items = (int)(gather_tiling == kTilePair
                                  ? B->qitems.size()
                                  : (gather_tiling == kTilePass ? B->pitems.size() : B->items.size()));
    batch_finalize_kernel<<<(B->n_sys + 3) / 4, 128, 0, B->stream>>>(
        part, B->d_sys, B->n_sys, n_items, gather_tiling, B->d_stats, B->d_log, B->log_cap,
        B->d_err);
    CK(cudaGetLastError());
  }
  return COULPS_OK;
}

int batch_check_error(coulps_batch *B) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, B->d_err, sizeof(int), cudaMemcpyDeviceToHost, B->stream));
  CK(cudaStreamSynchronize(B->stream));
  if (h & kErrTimeout) return COULPS_ETIMEOUT;
  if (h & kErrNonFinite) return COULPS_ENONFINITE;
  return COULPS_OK;
}

}  // namespace

namespace coulps {
int batch_enqueue(coulps_batch *B, int n_hb, int n_or, bool measure) {
  return batch_enqueue_compound(B, n_hb, n_or, measure);
}
int batch_sync(coulps_batch *B) { return batch_check_error(B); }
}  // namespace coulps

namespace {

}  // namespace

extern "C" {

int coulps_batch_create(int n_systems, const int32_t *dims, int precision, uint64_t seed,
                        void *stream, coulps_batch_t *out) {
  if (!out) return COULPS_EINVAL;
  *out = nullptr;
  if (n_systems < 1 || n_systems > 65535 || !dims) return COULPS_EINVAL;
  if (precision != COULPS_F32 && precision != COULPS_F64) return COULPS_EINVAL;
  coulps_batch *B = new (std::nothrow) coulps_batch();
  if (!B) return COULPS_ENOMEM;
  B->n_sys = n_systems;
  B->precision = precision;
  B->es = precision == COULPS_F32 ? 4 : 8;
  B->seed = seed;
  B->stream = (cudaStream_t)stream;
  B->alloc = current_allocator();
  long long off = 0;
  for (int s = 0; s < n_systems; ++s) {
    BatchSystem S;
    std::memset(&S, 0, sizeof(S));
    S.Lx = dims[3 * s];
    S.Ly = dims[3 * s + 1];
    S.Lz = dims[3 * s + 2];
    if (S.Lx < 1 || S.Ly < 1 || S.Lz < 1 || S.Lx > 512 || S.Ly > 65535 || S.Lz > 65535 ||
        (uint64_t)S.Lz * S.Ly * ((S.Lx + 7) / 8) > 0xffffffffull) {
      delete B;
      return COULPS_EINVAL;
    }
    S.W = batch_row_stride(S.Lx, B->es);
    S.Wq = (S.Lx + 7) / 8;
    S.QW = S.W / 4;
    S.TY = std::max(1, std::min(std::min(S.Ly, kBatchThreads / S.QW), 254));
    S.DZ = std::min(S.Lz, 16);
    // fused-pass tile: (PTY + 2) rows of quads within one 256-thread CTA, an
    // odd row count (the fastest in measurements of the single-lattice pass)
    S.PTY = kBatchPassThreads / S.QW - 2;
    if (S.PTY > 1 && S.PTY % 2 == 0) --S.PTY;
    S.PTY = std::max(1, std::min(std::min(S.PTY, S.Ly), 252));
    S.PDZ = S.Lz >= 64 ? 32 : S.Lz;
    // pass-pair tile: (QTY + 6) rows of quads within one CTA of the pair
    // kernel's width, whole z up to 127 planes (the ring's 8 halo planes
    // are then outside the box and cost no DRAM traffic), else 64
    S.QTY = std::min(std::min(batch_pair_threads(B->es) / S.QW - 6, S.Ly), 248);
    if (!batch_pair_fits(S, S.QTY, B->es)) S.QTY = 0;
    S.QDZ = S.Lz < 128 ? S.Lz : 64;
    S.colour_elems = (long long)S.Lz * S.Ly * S.W;
    S.field_off = off;
    off += 2 * S.colour_elems;
    B->sys.push_back(S);
  }
  B->field_bytes = (size_t)off * B->es;
  B->field = dev_alloc(B->alloc, B->field_bytes, B->stream);
  B->d_sys = (BatchSystem *)dev_alloc(B->alloc, n_systems * sizeof(BatchSystem), B->stream);
  B->d_maps = (CUtensorMap *)dev_alloc(B->alloc, 4 * (size_t)n_systems * sizeof(CUtensorMap),
                                       B->stream);
  B->d_pmaps = (CUtensorMap *)dev_alloc(B->alloc, 4 * (size_t)n_systems * sizeof(CUtensorMap),
                                        B->stream);
  B->d_qmaps = (CUtensorMap *)dev_alloc(B->alloc, 4 * (size_t)n_systems * sizeof(CUtensorMap),
                                        B->stream);
  B->d_ctr = (int *)dev_alloc(B->alloc, 64, B->stream);
  B->d_pass = (uint32_t *)dev_alloc(B->alloc, 64, B->stream);
  B->d_err = (int *)dev_alloc(B->alloc, 64, B->stream);
  B->d_stats = (double *)dev_alloc(B->alloc, (size_t)n_systems * kStatStride * sizeof(double),
                                   B->stream);
  if (!B->field || !B->d_sys || !B->d_maps || !B->d_pmaps || !B->d_qmaps || !B->d_ctr ||
      !B->d_pass || !B->d_err || !B->d_stats) {
    coulps_batch_destroy(B);
    return COULPS_ENOMEM;
  }
  B->bytes = B->field_bytes;
  if (cudaMemsetAsync(B->field, 0, B->field_bytes, B->stream) != cudaSuccess ||
      cudaMemsetAsync(B->d_pass, 0, 64, B->stream) != cudaSuccess ||
      cudaMemsetAsync(B->d_ctr, 0, 64, B->stream) != cudaSuccess ||
      cudaMemsetAsync(B->d_err, 0, 64, B->stream) != cudaSuccess) {
    cudaGetLastError();
    coulps_batch_destroy(B);
    return COULPS_ECUDA;
  }
  batch_reset_stats_kernel<<<(n_systems * kStatStride + 255) / 256, 256, 0, B->stream>>>(
      B->d_stats, n_systems);
  int st = coulps_batch_set_fused(B, batch_pairs_ok(B) ? 2 : 1);
  if (!st) st = batch_layout(B);
  if (st) {
    coulps_batch_destroy(B);
    return st;
  }
  *out = B;
  return COULPS_OK;
}

int coulps_batch_set_fused(coulps_batch_t B, int enable) {
  if (!B || enable < 0 || enable > 3) return COULPS_EINVAL;
  if (enable >= 2 && !batch_pairs_ok(B)) return COULPS_EINVAL;
  batch_drop_graph(B);
  if (!enable) {
    if (B->field2) {
      release(B, B->field2);
      B->bytes -= B->field_bytes;
    }
    B->fused = 0;
  } else {
    if (!B->field2) {
      B->field2 = dev_alloc(B->alloc, B->field_bytes, B->stream);
      if (!B->field2) return COULPS_ENOMEM;
      B->bytes += B->field_bytes;
      // row padding and never-written quads stay 0 in both copies
      CK(cudaMemsetAsync(B->field2, 0, B->field_bytes, B->stream));
    }
    B->fused = enable;
  }
  B->layout_dirty = true;
  return batch_layout(B);
}

int coulps_batch_set_pass_tiles(coulps_batch_t B, const int32_t *ty_dz) {
  if (!B || !ty_dz) return COULPS_EINVAL;
  std::vector<BatchSystem> next = B->sys;
  for (int s = 0; s < B->n_sys; ++s) {
    BatchSystem &S = next[s];
    const int ty = ty_dz[2 * s], dz = ty_dz[2 * s + 1];
    if (ty < 0 || dz < 0) return COULPS_EINVAL;
    if (ty > 0) S.PTY = ty;
    if (dz > 0) S.PDZ = dz;
    if (S.PTY + 4 > 256 || S.QW * (S.PTY + 2) > kBatchPassThreads) return COULPS_EINVAL;
    if (pass_layout(S.PTY, S.W, B->es, true).total + 128 > 227 * 1024) return COULPS_EINVAL;
  }
  B->sys = next;
  B->layout_dirty = true;
  return batch_layout(B);
}

int coulps_batch_system_pass_tile(coulps_batch_t B, int system, int32_t *ty_dz) {
  if (!B || !ty_dz || system < 0 || system >= B->n_sys) return COULPS_EINVAL;
  ty_dz[0] = B->sys[system].PTY;
  ty_dz[1] = B->sys[system].PDZ;
  return COULPS_OK;
}

int coulps_batch_set_pair_tiles(coulps_batch_t B, const int32_t *ty_dz) {
  if (!B || !ty_dz) return COULPS_EINVAL;
  std::vector<BatchSystem> next = B->sys;
  for (int s = 0; s < B->n_sys; ++s) {
    BatchSystem &S = next[s];
    const int ty = ty_dz[2 * s], dz = ty_dz[2 * s + 1];
    if (ty < 0 || dz < 0) return COULPS_EINVAL;
    if (ty > 0) S.QTY = ty;
    if (dz > 0) S.QDZ = dz;
    if (!batch_pair_fits(S, S.QTY, B->es)) return COULPS_EINVAL;
  }
  B->sys = next;
  B->layout_dirty = true;
  return batch_layout(B);
}

int coulps_batch_system_pair_tile(coulps_batch_t B, int system, int32_t *ty_dz) {
  if (!B || !ty_dz || system < 0 || system >= B->n_sys) return COULPS_EINVAL;
  ty_dz[0] = B->sys[system].QTY;
  ty_dz[1] = B->sys[system].QDZ;
  return COULPS_OK;
}

int coulps_batch_fused(coulps_batch_t B) { return B ? B->fused : -1; }

void coulps_batch_destroy(coulps_batch_t B) {
  if (!B) return;
  batch_drop_graph(B);
  release(B, B->field);
  release(B, B->d_sys);
  release(B, B->d_items);
  release(B, B->d_maps);
  release(B, B->d_pmaps);
  release(B, B->field2);
  release(B, B->d_pitems);
  release(B, B->d_pgoff);
  release(B, B->d_pgent);
  release(B, B->d_pgq);
  release(B, B->d_ppart);
  release(B, B->d_qmaps);
  release(B, B->d_qitems);
  release(B, B->d_qorder);
  release(B, B->d_order);
  release(B, B->d_porder);
  release(B, B->d_qgoff);
  release(B, B->d_qgent);
  release(B, B->d_qgq);
  release(B, B->d_qpart);
  release(B, B->d_ctr);
  release(B, B->d_pass);
  release(B, B->d_err);
  release(B, B->d_goff);
  release(B, B->d_gent);
  release(B, B->d_gq);
  release(B, B->d_part);
  release(B, B->d_stats);
  release(B, B->d_log);
  delete B;
}

int coulps_batch_set_tiles(coulps_batch_t B, const int32_t *ty_dz) {
  if (!B || !ty_dz) return COULPS_EINVAL;
  std::vector<BatchSystem> next = B->sys;
  for (int s = 0; s < B->n_sys; ++s) {
    BatchSystem &S = next[s];
    const int ty = ty_dz[2 * s], dz = ty_dz[2 * s + 1];
    if (ty < 0 || dz < 0) return COULPS_EINVAL;
    if (ty > 0) S.TY = ty;
    if (dz > 0) S.DZ = dz;
    if (S.TY + 2 > 256 || S.QW * S.TY > kBatchThreads) return COULPS_EINVAL;
  }
  B->sys = next;
  B->layout_dirty = true;
  if (batch_smem_bytes(B, true) > 227 * 1024) return COULPS_EINVAL;
  return batch_layout(B);
}

int coulps_batch_info(coulps_batch_t B, int64_t *info) {
  if (!B || !info) return COULPS_EINVAL;
  info[0] = B->n_sys;
  info[1] = (int64_t)B->items.size();
  info[2] = B->grid;
  info[3] = (int64_t)B->smem;
  info[4] = (int64_t)B->pass;
  info[5] = (int64_t)B->field_bytes;
  int64_t sites = 0;
  for (const auto &S : B->sys) sites += (int64_t)S.Lx * S.Ly * S.Lz;
  info[6] = sites;
  info[7] = B->pgrid;
  info[8] = B->fused >= 2 ? B->qgrid : 0;
  info[9] = B->fused >= 2 ? B->qthreads : 0;
  return COULPS_OK;
}

int coulps_batch_system_tile(coulps_batch_t B, int system, int32_t *ty_dz) {
  if (!B || !ty_dz || system < 0 || system >= B->n_sys) return COULPS_EINVAL;
  ty_dz[0] = B->sys[system].TY;
  ty_dz[1] = B->sys[system].DZ;
  return COULPS_OK;
}

int coulps_batch_charges(coulps_batch_t B, const int64_t *offsets, const int32_t *site,
                         const double *q, int64_t log_capacity) {
  if (!B || !offsets || log_capacity < 0) return COULPS_EINVAL;
  if (offsets[0] != 0) return COULPS_EINVAL;
  for (int s = 0; s < B->n_sys; ++s)
    if (offsets[s + 1] < offsets[s]) return COULPS_EINVAL;
  const int64_t n = offsets[B->n_sys];
  if (n > 0 && (!site || !q)) return COULPS_EINVAL;
  if (n >= ((int64_t)1 << 31)) return COULPS_EINVAL;
  for (int s = 0; s < B->n_sys; ++s) {
    const BatchSystem &S = B->sys[s];
    for (int64_t i = offsets[s]; i < offsets[s + 1]; ++i) {
      const int x = site[3 * i], y = site[3 * i + 1], z = site[3 * i + 2];
      if (x < 0 || x >= S.Lx || y < 0 || y >= S.Ly || z < 0 || z >= S.Lz || !std::isfinite(q[i]))
        return COULPS_EINVAL;
    }
  }
  B->offsets.assign(offsets, offsets + B->n_sys + 1);
  B->sites.assign(site, site + 3 * n);
  B->q.assign(q, q + n);
  B->has_charges = true;
  release(B, B->d_log);
  B->log_cap = log_capacity;
  if (log_capacity > 0) {
    B->d_log = (double *)dev_alloc(B->alloc, sizeof(double) * 3 * (size_t)log_capacity * B->n_sys,
                                   B->stream);
    if (!B->d_log) return COULPS_ENOMEM;
  }
  batch_reset_stats_kernel<<<(B->n_sys * kStatStride + 255) / 256, 256, 0, B->stream>>>(
      B->d_stats, B->n_sys);
  CK(cudaGetLastError());
  B->layout_dirty = true;
  return batch_layout(B);
}

int coulps_batch_sweep(coulps_batch_t B, int n_compound, int n_hb, int n_or) {
  if (!B || n_compound < 0 || n_hb < 0 || n_or < 0) return COULPS_EINVAL;
  int st = batch_layout(B);
  if (st) return st;
  for (int k = 0; k < n_compound; ++k) {
    st = batch_enqueue_compound(B, n_hb, n_or, false);
    if (st) return st;
    B->pass += (uint64_t)(n_hb + n_or);
  }
  return COULPS_OK;
}

int coulps_batch_run(coulps_batch_t B, int n_therm, int n_meas, int n_hb, int n_or) {
  if (!B || n_therm < 0 || n_meas < 0 || n_hb < 0 || n_or < 0) return COULPS_EINVAL;
  if (n_meas > 0 && (!B->has_charges || n_hb + n_or == 0)) return COULPS_EINVAL;
  int st = coulps_batch_sweep(B, n_therm, n_hb, n_or);
  if (st || n_meas == 0) return st;
  const bool capturable = B->stream != nullptr;
  if (capturable && (!B->graph || B->graph_hb != n_hb || B->graph_or != n_or)) {
    batch_drop_graph(B);
    cudaGraph_t gr = nullptr;
    CK(cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
    const int s1 = batch_enqueue_compound(B, n_hb, n_or, true);
    cudaError_t e = cudaStreamEndCapture(B->stream, &gr);
    if (s1 || e != cudaSuccess) {
      cudaGetLastError();
      if (gr) cudaGraphDestroy(gr);
      return s1 ? s1 : COULPS_ECUDA;
    }
    e = cudaGraphInstantiate(&B->graph, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
      cudaGetLastError();
      B->graph = nullptr;
      return COULPS_ECUDA;
    }
    B->graph_hb = n_hb;
    B->graph_or = n_or;
  }
  for (int k = 0; k < n_meas; ++k) {
    if (capturable) {
      CK(cudaGraphLaunch(B->graph, B->stream));
    } else {
      st = batch_enqueue_compound(B, n_hb, n_or, true);
      if (st) return st;
    }
    B->pass += (uint64_t)(n_hb + n_or);
  }
  return COULPS_OK;
}

int coulps_batch_sync(coulps_batch_t B) {
  if (!B) return COULPS_EINVAL;
  return batch_check_error(B);
}

int coulps_batch_estimate(coulps_batch_t B, double *mean, double *stderr_bm, double *tau_int,
                          int64_t *n) {
  if (!B) return COULPS_EINVAL;
  std::vector<double> st((size_t)B->n_sys * kStatStride);
  CK(cudaMemcpyAsync(st.data(), B->d_stats, st.size() * sizeof(double), cudaMemcpyDeviceToHost,
                     B->stream));
  int s = batch_check_error(B);
  if (s) return s;
  for (int k = 0; k < B->n_sys; ++k) {
    double m, e, t;
    int64_t c;
    s = coulps_pool_stats(st.data() + (size_t)k * kStatStride, 1, &m, &e, &t, &c);
    if (s && s != COULPS_ENONFINITE) return s;
    if (mean) mean[k] = m;
    if (stderr_bm) stderr_bm[k] = e;
    if (tau_int) tau_int[k] = t;
    if (n) n[k] = c;
  }
  return COULPS_OK;
}

int coulps_batch_samples(coulps_batch_t B, double *QPe, int64_t cap, int64_t *n) {
  if (!B || cap < 0 || (cap > 0 && !QPe)) return COULPS_EINVAL;
  double ns = 0;
  CK(cudaMemcpyAsync(&ns, B->d_stats + kStatN, sizeof(double), cudaMemcpyDeviceToHost,
                     B->stream));
  int s = batch_check_error(B);
  if (s) return s;
  int64_t m = std::min<int64_t>((int64_t)ns, std::min(cap, B->log_cap));
  if (m > 0) {
    CK(cudaMemcpyAsync(QPe, B->d_log, sizeof(double) * 3 * (size_t)m * B->n_sys,
                       cudaMemcpyDeviceToHost, B->stream));
    CK(cudaStreamSynchronize(B->stream));
  }
  if (n) *n = m;
  return COULPS_OK;
}

int coulps_batch_field_set(coulps_batch_t B, int system, const double *host) {
  if (!B || !host || system < 0 || system >= B->n_sys) return COULPS_EINVAL;
  const BatchSystem &S = B->sys[system];
  std::vector<unsigned char> buf((size_t)2 * S.colour_elems * B->es, 0);
  for (int z = 0; z < S.Lz; ++z)
    for (int y = 0; y < S.Ly; ++y)
      for (int x = 0; x < S.Lx; ++x) {
        const size_t k = (size_t)((x + y + z) & 1) * S.colour_elems + ((size_t)z * S.Ly + y) * S.W +
                         (x >> 1);
        const double v = host[x + (size_t)S.Lx * (y + (size_t)S.Ly * z)];
        if (B->precision == COULPS_F32)
          reinterpret_cast<float *>(buf.data())[k] = (float)v;
        else
          reinterpret_cast<double *>(buf.data())[k] = v;
      }
  CK(cudaMemcpyAsync((char *)B->field + (size_t)S.field_off * B->es, buf.data(), buf.size(),
                     cudaMemcpyHostToDevice, B->stream));
  return batch_check_error(B);  // buf leaves scope
}

int coulps_batch_stats(coulps_batch_t B, double *out, int64_t cap) {
  if (!B || !out) return COULPS_EINVAL;
  const int64_t need = (int64_t)B->n_sys * kStatStride;
  if (cap < need) return COULPS_EINVAL;
  CK(cudaMemcpyAsync(out, B->d_stats, need * sizeof(double), cudaMemcpyDeviceToHost, B->stream));
  return batch_check_error(B);
}

int coulps_batch_reset_stats(coulps_batch_t B) {
  if (!B) return COULPS_EINVAL;
  batch_reset_stats_kernel<<<(B->n_sys * kStatStride + 255) / 256, 256, 0, B->stream>>>(B->d_stats,
                                                                                      B->n_sys);
  CK(cudaGetLastError());
  return COULPS_OK;
}

int coulps_batch_field_get(coulps_batch_t B, int system, double *host) {
  if (!B || !host || system < 0 || system >= B->n_sys) return COULPS_EINVAL;
  const BatchSystem &S = B->sys[system];
  std::vector<unsigned char> buf((size_t)2 * S.colour_elems * B->es);
  CK(cudaMemcpyAsync(buf.data(), (const char *)B->field + (size_t)S.field_off * B->es, buf.size(),
                     cudaMemcpyDeviceToHost, B->stream));
  int s = batch_check_error(B);
  if (s) return s;
  for (int z = 0; z < S.Lz; ++z)
    for (int y = 0; y < S.Ly; ++y)
      for (int x = 0; x < S.Lx; ++x) {
        const size_t k = (size_t)((x + y + z) & 1) * S.colour_elems + ((size_t)z * S.Ly + y) * S.W +
                         (x >> 1);
        host[x + (size_t)S.Lx * (y + (size_t)S.Ly * z)] =
            B->precision == COULPS_F32 ? (double)reinterpret_cast<const float *>(buf.data())[k]
                                       : reinterpret_cast<const double *>(buf.data())[k];
      }
  return COULPS_OK;
}

}  // extern "C"
