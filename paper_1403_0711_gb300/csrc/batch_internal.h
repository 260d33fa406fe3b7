// The many-system batch's state, shared by batch.cu (the sweeps) and
// batch_gcv.cu (the global control variate of every system).
#pragma once

#include <cstdint>
#include <vector>

#include "internal.h"

namespace coulps {

struct BatchSystem {
  int Lx, Ly, Lz, W, Wq, QW, TY, DZ;
  long long field_off;     // first element of the system's field ([colour][z][y][h])
  long long colour_elems;  // Lz * Ly * W
  int goff_base;           // first gather offset of the system (y tile * Lz + z)
  int item_begin;          // first tile of the system in the work list
  int PTY, PDZ;            // fused-pass tile: rows, planes
  int pgoff_base;          // first pass-tile gather offset of the system
  int pitem_begin;         // first pass tile of the system in the pass work list
  int QTY, QDZ;            // pass-pair tile: rows, planes (QTY = 0: no pair tile fits)
  int qgoff_base;          // first pair-tile gather offset of the system
  int qitem_begin;         // first pair tile of the system in the pair work list
};

// Tilings of one system's lattice: half-sweep, fused-pass, pass-pair tiles.
enum Tiling { kTileHalf = 0, kTilePass = 1, kTilePair = 2 };

struct BatchItem {
  int sys, y0, z0, nz;
};

}  // namespace coulps

struct coulps_batch {
  int n_sys = 0;
  int precision = COULPS_F32, es = 4;
  uint64_t seed = 0;
  cudaStream_t stream = nullptr;
  coulps::Allocator alloc = {nullptr, nullptr, nullptr};
  std::vector<coulps::BatchSystem> sys;
  std::vector<coulps::BatchItem> items;
  void *field = nullptr;
  size_t field_bytes = 0;
  coulps::BatchSystem *d_sys = nullptr;
  coulps::BatchItem *d_items = nullptr;
  int *d_order = nullptr, *d_porder = nullptr;  // tile lists largest first
  CUtensorMap *d_maps = nullptr;  // half-sweep maps: [copy][system][2]
  // fused over-relaxation passes (fused >= 1): a second copy of the fields,
  // the pass tiles, their maps [copy][system][2] and gather lists; with
  // fused = 2 also the pair tiles
  int fused = 0;
  void *field2 = nullptr;
  std::vector<coulps::BatchItem> pitems;
  coulps::BatchItem *d_pitems = nullptr;
  CUtensorMap *d_pmaps = nullptr;
  uint32_t *d_pgoff = nullptr, *d_pgent = nullptr;
  double *d_pgq = nullptr, *d_ppart = nullptr;
  int pgrid = 0;
  size_t psmem = 0;
  std::vector<coulps::BatchItem> qitems;
  coulps::BatchItem *d_qitems = nullptr;
  int *d_qorder = nullptr;
  CUtensorMap *d_qmaps = nullptr;
  uint32_t *d_qgoff = nullptr, *d_qgent = nullptr;
  double *d_qgq = nullptr, *d_qpart = nullptr;
  int *d_ctr = nullptr;
  int qgrid = 0, qthreads = 0;
  size_t qsmem = 0;
  uint32_t *d_pass = nullptr;
  int *d_err = nullptr;
  uint64_t pass = 0;
  int grid = 0;        // persistent CTAs
  size_t smem = 0;     // dynamic shared memory per CTA (largest system)
  int grid2 = 0, threads2 = 0;  // the same with two quads per thread
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

namespace coulps {
// One compound sweep of every system (and its sample when `measure`),
// enqueued on the batch's stream (batch.cu).
int batch_enqueue(coulps_batch *B, int n_hb, int n_or, bool measure);
// Synchronises the batch's stream and returns its device error status.
int batch_sync(coulps_batch *B);
}  // namespace coulps
