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
// Fused over-relaxation passes (coulps_batch_set_fused, on by default): the
// over-relaxation passes run as fused passes (both half-sweeps of a pass in
// one z-march, pass_march.cuh) from one copy of the fields to a second one
// and back, by a persistent kernel that walks a list of pass tiles (each
// system with its own pass tile shape and tensor maps on both copies); the
// heatbath passes stay half-sweeps, the first written out of place into the
// second copy when the over-relaxation count is odd, so that the compound
// sweep ends in the first copy.  The sample is gathered by the last kernel.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "device_common.cuh"
#include "internal.h"
#include "pass_march.cuh"
#include "tile_march.cuh"

namespace coulps {
namespace {

using namespace tile;

constexpr int kBatchThreads = 256;
constexpr int kBatchPassThreads = 256;

struct BatchSystem {
  int Lx, Ly, Lz, W, Wq, QW, TY, DZ;
  long long field_off;     // first element of the system's field ([colour][z][y][h])
  long long colour_elems;  // Lz * Ly * W
  int goff_base;           // first gather offset of the system (y tile * Lz + z)
  int item_begin;          // first tile of the system in the work list
  int PTY, PDZ;            // fused-pass tile: rows, planes
  int pgoff_base;          // first pass-tile gather offset of the system
  int pitem_begin;         // first pass tile of the system in the pass work list
};

struct BatchItem {
  int sys, y0, z0, nz;
};

struct BatchArgs {
  void *field;  // written: the own colour of each tile
  const BatchSystem *sys;
  const BatchItem *items;
  int n_items;
  const CUtensorMap *maps;  // 2 per system: other-colour box (TY+2 rows), own box (TY rows)
  int colour;
  uint32_t round_keys[20];
  const uint32_t *pass_ptr;
  uint32_t pass_off;
  int *err;
  const uint32_t *g_off, *g_ent;
  const double *g_q;
  double *g_partials;  // [item][2]
};

template <typename T, bool OR, bool GATHER>
__global__ void __launch_bounds__(kBatchThreads) batch_halfsweep_kernel(const BatchArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = align_smem128(smem_raw);
  const PhiloxKeys &K = *reinterpret_cast<const PhiloxKeys *>(a.round_keys);
  const uint32_t pass = OR ? 0u : (*a.pass_ptr + a.pass_off);
  int gbase = 0;
  ring_init(smem);
  for (int it = blockIdx.x; it < a.n_items; it += gridDim.x) {
    const BatchItem item = a.items[it];
    const BatchSystem S = a.sys[item.sys];
    TileJob<T> j;
    j.tm_halo = &a.maps[2 * item.sys];
    j.tm_own = &a.maps[2 * item.sys + 1];
    j.colour = a.colour;
    j.map_other = a.colour ^ 1;
    j.map_own = a.colour;
    j.out = reinterpret_cast<T *>(a.field) + S.field_off + (long long)a.colour * S.colour_elems;
    j.Lx = S.Lx; j.Ly = S.Ly; j.Lz = S.Lz; j.W = S.W; j.Wq = S.Wq; j.QW = S.QW; j.TY = S.TY;
    j.y0 = item.y0;
    j.z0 = item.z0;
    j.nz = item.nz;
    j.rng_id = (uint32_t)item.sys;
    j.pass = pass;
    if (GATHER) {
      j.g_off = a.g_off + S.goff_base + (size_t)(item.y0 / S.TY) * S.Lz;
      j.g_ent = a.g_ent;
      j.other = reinterpret_cast<const T *>(a.field) + S.field_off +
                (long long)(a.colour ^ 1) * S.colour_elems;
      j.g_q = a.g_q;
    }
    double sq = 0.0, sp = 0.0;
    const bool ok = march_tile<T, OR, GATHER>(j, K, smem, a.err, gbase, sq, sp);
    if (GATHER) block_partials(sq, sp, smem, a.g_partials + 2 * (size_t)it);
    if (!ok) break;
  }
}

// Fused passes over all systems: a persistent grid walks the pass tiles
// (system, y0, z0, nz), each CTA running march_pass tile after tile with its
// ring phases carried over; the source copy's tensor maps are 2 per system
// (colour-1 box PTY + 4 rows, colour-0 box PTY + 2 rows), dst the other copy.
struct BatchPassArgs {
  void *dst;
  const BatchSystem *sys;
  const BatchItem *items;
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
  for (int it = blockIdx.x; it < a.n_items; it += gridDim.x) {
    const BatchItem item = a.items[it];
    const BatchSystem S = a.sys[item.sys];
    PassJob<T> j;
    j.tm_c1 = &a.maps[2 * item.sys];
    j.tm_c0 = &a.maps[2 * item.sys + 1];
    j.map_c1 = 1;
    j.map_c0 = 0;
    j.dst0 = reinterpret_cast<T *>(a.dst) + S.field_off;
    j.dst1 = j.dst0 + S.colour_elems;
    j.Lx = S.Lx; j.Ly = S.Ly; j.Lz = S.Lz; j.W = S.W; j.Wq = S.Wq; j.QW = S.QW; j.TY = S.PTY;
    j.y0 = item.y0;
    j.z0 = item.z0;
    j.nz = item.nz;
    j.rng_id = (uint32_t)item.sys;
    j.pass = pass;
    j.g_off = GATHER ? a.g_off + S.pgoff_base + (size_t)(item.y0 / S.PTY) * S.Lz : nullptr;
    j.g_ent = a.g_ent;
    j.g_q = a.g_q;
    double sq = 0.0, sp = 0.0;
    const bool ok = march_pass<T, OR, GATHER>(j, K, smem, a.err, gbase, sq, sp);
    if (GATHER) block_partials(sq, sp, smem, a.g_partials + 2 * (size_t)it);
    if (!ok) break;
  }
}

// Each system's tile partials added in tile order: the half-sweep tiles, or
// (pass_tiles) the fused-pass tiles.
__global__ void batch_finalize_kernel(const double *__restrict__ partials,
                                      const BatchSystem *__restrict__ sys, int n_sys, int n_items,
                                      bool pass_tiles, double *__restrict__ stats,
                                      double *__restrict__ log, int64_t log_cap, int *err) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_sys) return;
  const int b0 = pass_tiles ? sys[s].pitem_begin : sys[s].item_begin;
  const int b1 = s + 1 < n_sys ? (pass_tiles ? sys[s + 1].pitem_begin : sys[s + 1].item_begin)
                               : n_items;
  double Q = 0.0, P = 0.0;
  for (int b = b0; b < b1; ++b) {
    Q += partials[2 * (size_t)b];
    P += partials[2 * (size_t)b + 1];
  }
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

struct coulps_batch {
  int n_sys = 0;
  int precision = COULPS_F32, es = 4;
  uint64_t seed = 0;
  cudaStream_t stream = nullptr;
  Allocator alloc = {nullptr, nullptr, nullptr};
  std::vector<BatchSystem> sys;
  std::vector<BatchItem> items;
  void *field = nullptr;
  size_t field_bytes = 0;
  BatchSystem *d_sys = nullptr;
  BatchItem *d_items = nullptr;
  CUtensorMap *d_maps = nullptr;  // half-sweep maps: [copy][system][2]
  // fused over-relaxation passes (fused = 1): a second copy of the fields,
  // the pass tiles, their maps [copy][system][2] and gather lists
  int fused = 0;
  void *field2 = nullptr;
  std::vector<BatchItem> pitems;
  BatchItem *d_pitems = nullptr;
  CUtensorMap *d_pmaps = nullptr;
  uint32_t *d_pgoff = nullptr, *d_pgent = nullptr;
  double *d_pgq = nullptr, *d_ppart = nullptr;
  int pgrid = 0;
  size_t psmem = 0;
  uint32_t *d_pass = nullptr;
  int *d_err = nullptr;
  uint64_t pass = 0;
  int grid = 0;        // persistent CTAs
  size_t smem = 0;     // dynamic shared memory per CTA (largest system)
  bool layout_dirty = true;
  // charges and estimator
  bool has_charges = false;
  std::vector<int64_t> offsets;
  std::vector<int32_t> sites;
  std::vector<double> q;
  uint32_t *d_goff = nullptr, *d_gent = nullptr;
  double *d_gq = nullptr, *d_part = nullptr, *d_stats = nullptr, *d_log = nullptr;
  int64_t log_cap = 0;
  size_t bytes = 0;
  cudaGraphExec_t graph = nullptr;
  int graph_hb = -1, graph_or = -1;
};

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
// rows of `pass` (fused-pass tiles) or of the half-sweep tiles: offsets
// `off` (system base + y tile * Lz + z) and entries (colour bit 31, offset
// within the colour's array).
void batch_gather_lists(const coulps_batch *B, bool pass, int n_off, std::vector<uint32_t> &off,
                        std::vector<uint32_t> &ent, std::vector<double> &gq) {
  off.assign((size_t)n_off + 1, 0);
  const int64_t ntot = B->offsets[B->n_sys];
  ent.assign((size_t)ntot, 0);
  gq.assign((size_t)ntot, 0.0);
  auto key = [&](const BatchSystem &S, int y, int z) {
    const int ty = pass ? S.PTY : S.TY;
    return (size_t)(pass ? S.pgoff_base : S.goff_base) + (size_t)(y / ty) * S.Lz + z;
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

// Tile lists, tensor maps and gather lists for the current tile shapes.
int batch_layout(coulps_batch *B) {
  if (!B->layout_dirty) return COULPS_OK;
  batch_drop_graph(B);
  B->items.clear();
  B->pitems.clear();
  int goff = 0, pgoff = 0;
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
  }
  // half-sweep maps on both copies (the second only with fused passes)
  std::vector<CUtensorMap> maps(4 * (size_t)B->n_sys);
  std::vector<CUtensorMap> pmaps(4 * (size_t)B->n_sys);
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
  if (!B->d_items || !B->d_part || !B->d_pitems || !B->d_ppart) return COULPS_ENOMEM;
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
  // gather lists for both tilings
  std::vector<uint32_t> off, ent, poff, pent;
  std::vector<double> gq, pgq;
  if (B->has_charges) {
    batch_gather_lists(B, false, goff, off, ent, gq);
    int st = batch_upload_lists(B, off, ent, gq, B->d_goff, B->d_gent, B->d_gq);
    if (st) return st;
    batch_gather_lists(B, true, pgoff, poff, pent, pgq);
    st = batch_upload_lists(B, poff, pent, pgq, B->d_pgoff, B->d_pgent, B->d_pgq);
    if (st) return st;
  }
  // persistent grids: as many CTAs as are co-resident at the largest smem need
  B->smem = batch_smem_bytes(B, true);
  B->psmem = batch_pass_smem_bytes(B);
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int per_sm = std::max(1, std::min(8, (int)((200 * 1024) / B->smem)));
  B->grid = std::max(1, std::min((int)B->items.size(), sms * per_sm));
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
  CK(cudaStreamSynchronize(B->stream));  // host vectors leave scope
  B->layout_dirty = false;
  return COULPS_OK;
}

template <typename T, bool OR, bool GATHER>
cudaError_t launch_batch_t(coulps_batch *B, const BatchArgs &a) {
  auto kfn = batch_halfsweep_kernel<T, OR, GATHER>;
  static size_t configured = 0;
  if (B->smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)B->smem);
    if (e != cudaSuccess) return e;
    configured = B->smem;
  }
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

// One compound sweep of every system (and its sample when `measure`).  With
// fused passes the over-relaxation block runs as fused passes between the
// two copies: all of it after the heatbath passes when n_or is even, or when
// it is odd and a heatbath pass precedes it (then the heatbath passes write
// the second copy, the first of them reading colour 1 from the first copy);
// otherwise all but the last, which runs as in-place half-sweeps.  The
// sweep ends in the first copy.
int batch_enqueue_compound(coulps_batch *B, int n_hb, int n_or, bool measure) {
  const int n = n_hb + n_or;
  int nf = 0;
  bool flip = false;
  if (B->fused && B->field2) {
    nf = n_or & ~1;
    if ((n_or & 1) && n_hb > 0) {
      nf = n_or;
      flip = true;
    }
  }
  const bool gather_pass = measure && nf > 0 && n_hb + nf == n;
  BatchArgs a;
  std::memset(&a, 0, sizeof(a));
  a.sys = B->d_sys;
  a.items = B->d_items;
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
  for (int i = 0; i < n_hb; ++i) {
    const int r = half_sweeps(i, flip, measure && nf == 0 && i == n - 1);
    if (r) return r;
  }
  BatchPassArgs p;
  std::memset(&p, 0, sizeof(p));
  p.sys = B->d_sys;
  p.items = B->d_pitems;
  p.n_items = (int)B->pitems.size();
  for (int i = 0; i < 20; ++i) p.round_keys[i] = K.k[i];
  p.pass_ptr = B->d_pass;
  p.err = B->d_err;
  for (int t = 0; t < nf; ++t) {
    const int i = n_hb + t;
    const int b = (t + (flip ? 1 : 0)) & 1;  // source copy
    p.dst = b ? B->field : B->field2;
    p.maps = B->d_pmaps + 2 * (size_t)b * B->n_sys;
    p.pass_off = (uint32_t)i;
    const bool last = gather_pass && t == nf - 1;
    p.g_off = last ? B->d_pgoff : nullptr;
    p.g_ent = last ? B->d_pgent : nullptr;
    p.g_q = last ? B->d_pgq : nullptr;
    p.g_partials = last ? B->d_ppart : nullptr;
    CK(B->precision == COULPS_F32 ? launch_bpass_p<float>(B, p, true)
                                  : launch_bpass_p<double>(B, p, true));
  }
  for (int i = n_hb + nf; i < n; ++i) {
    const int r = half_sweeps(i, false, measure && i == n - 1);
    if (r) return r;
  }
  if (n > 0) CK(launch_advance_pass(B->d_pass, (uint32_t)n, B->stream));
  if (measure) {
    batch_finalize_kernel<<<(B->n_sys + 127) / 128, 128, 0, B->stream>>>(
        gather_pass ? B->d_ppart : B->d_part, B->d_sys, B->n_sys,
        gather_pass ? (int)B->pitems.size() : (int)B->items.size(), gather_pass, B->d_stats,
        B->d_log, B->log_cap, B->d_err);
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
  B->d_pass = (uint32_t *)dev_alloc(B->alloc, 64, B->stream);
  B->d_err = (int *)dev_alloc(B->alloc, 64, B->stream);
  B->d_stats = (double *)dev_alloc(B->alloc, (size_t)n_systems * kStatStride * sizeof(double),
                                   B->stream);
  if (!B->field || !B->d_sys || !B->d_maps || !B->d_pmaps || !B->d_pass || !B->d_err ||
      !B->d_stats) {
    coulps_batch_destroy(B);
    return COULPS_ENOMEM;
  }
  B->bytes = B->field_bytes;
  if (cudaMemsetAsync(B->field, 0, B->field_bytes, B->stream) != cudaSuccess ||
      cudaMemsetAsync(B->d_pass, 0, 64, B->stream) != cudaSuccess ||
      cudaMemsetAsync(B->d_err, 0, 64, B->stream) != cudaSuccess) {
    cudaGetLastError();
    coulps_batch_destroy(B);
    return COULPS_ECUDA;
  }
  batch_reset_stats_kernel<<<(n_systems * kStatStride + 255) / 256, 256, 0, B->stream>>>(
      B->d_stats, n_systems);
  int st = coulps_batch_set_fused(B, 1);
  if (!st) st = batch_layout(B);
  if (st) {
    coulps_batch_destroy(B);
    return st;
  }
  *out = B;
  return COULPS_OK;
}

int coulps_batch_set_fused(coulps_batch_t B, int enable) {
  if (!B || enable < 0 || enable > 1) return COULPS_EINVAL;
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
    B->fused = 1;
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
