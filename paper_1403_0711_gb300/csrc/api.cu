// Host side of the C ABI declared in include/coulps.h.
//
// Owns the device buffers, validates arguments, builds the TMA tensor maps,
// sequences the half-sweep / gather / finalize launches on the handle's
// stream, captures the measured loop into a CUDA graph, and turns the
// per-chain running sums into the pooled estimate with its batch-means error
// (the host-side counterpart of the paper's final mpi_reduce).
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "device_common.cuh"
#include "internal.h"

using namespace coulps;

namespace coulps {

static Allocator g_allocator = {nullptr, nullptr, nullptr};

Allocator current_allocator() { return g_allocator; }

void *dev_alloc(const Allocator &a, size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 16;
  if (a.alloc) return a.alloc(bytes, (void *)s, a.ctx);
  void *p = nullptr;
  if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(const Allocator &a, void *p, cudaStream_t s) {
  if (!p) return;
  if (a.free_fn) {
    a.free_fn(p, (void *)s, a.ctx);
    return;
  }
  cudaFreeAsync(p, s);
}

}  // namespace coulps

struct coulps_lattice {
  Geometry g;
  Tile tile;
  uint64_t seed;
  cudaStream_t stream;
  Allocator alloc;
  void *field = nullptr;
  uint32_t *d_pass = nullptr;
  int *d_err = nullptr;
  uint64_t pass = 0;  // host mirror of *d_pass
  CUtensorMap tm_halo, tm_own;
  // fused passes (pass_fused.cu): a second copy of the field; a compound
  // sweep starts and ends in `field`, and field2 is scratch within it
  // (an odd block of fused passes starts from field2, which the first
  // heatbath pass then writes out of place)
  void *field2 = nullptr;
  CUtensorMap tm_halo2;  // halo map of field2 (tile ty + 2 rows)
  // split > 1 streams: chains k with k % split == j on stream j (stream 0 is
  // the lattice's own; xstream[j - 1] the library's; coulps_set_streams)
  int split = 1;
  cudaStream_t xstream[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr, ev_join[3] = {nullptr, nullptr, nullptr};
  int fused = 0;  // 0 off, 1 over-relaxation passes, 2 all passes, 3 over-relaxation
                  // pass pairs, 4 all passes as pairs (pass_plan)
  Tile ptile = {0, 0};
  CUtensorMap tm_p1[2], tm_p0[2];  // source field / field2; boxes ty + 4, ty + 2 rows
  // pass pairs (pass_pair.cu): tile ({0, 0} when the row is too wide for a
  // pair CTA) and maps on field / field2 with boxes ty + 8 and ty + 6 rows
  Tile qtile = {0, 0};
  CUtensorMap tm_q1[2], tm_q0[2];
  size_t bytes = 0;
  int n_charge_sets = 0;
  // measured compound sweep captured as a graph
  cudaGraphExec_t graph = nullptr;
  const void *graph_key = nullptr;
  int graph_hb = -1, graph_or = -1;
  Tile graph_tile = {0, 0};
  // per-kernel event timing
  bool profiling = false;
  struct Timed {
    cudaEvent_t a, b;
    int kind;  // 0 heatbath, 1 over-relaxation, 2 mixed (phase-shifted schedule),
               // 3 fused heatbath pass, 4 fused over-relaxation pass,
               // 5 pass pair with a heatbath pass, 6 over-relaxation pass pair
  };
  std::vector<cudaEvent_t> spare_events;
  std::vector<Timed> pending;
  static constexpr int kTimeSlots = 14;
  double times[kTimeSlots] = {0};
  // measured-phase schedule (COULPS_SCHEDULE_*) and its steady-state graph
  int schedule = COULPS_SCHEDULE_ALIGNED;
  cudaGraphExec_t sgraph = nullptr;
  const void *sgraph_key = nullptr;
  int sgraph_hb = -1, sgraph_or = -1;
  Tile sgraph_tile = {0, 0};
  // shifted schedule: prologue, steady step and epilogue graphs
  cudaGraphExec_t hgraph[3] = {nullptr, nullptr, nullptr};
  const void *hgraph_key = nullptr;
  int hgraph_hb = -1, hgraph_or = -1;
  // measured compound sweep + multi-set gather (coulps_run_sets) as a graph
  cudaGraphExec_t mgraph = nullptr;
  std::vector<const void *> mgraph_key;
  int mgraph_hb = -1, mgraph_or = -1;
};

struct coulps_charges {
  coulps_lattice *lat = nullptr;
  int64_t n = 0;
  uint32_t *d_idx = nullptr;
  double *d_q = nullptr;
  int nblk = 1;
  double *d_partials = nullptr;  // scratch: [chain][nblk][2]
  double *d_stats = nullptr;     // [chain][kStatStride]
  double *d_cvstats = nullptr;   // [chain][kStatStride], control-variate samples
  // coulps_estimate_post / _take: two pinned slots of the estimator state
  // and the lattice's error word, each with the event that completes its copy
  double *h_post = nullptr;  // [2][chain][kStatStride]
  int *h_post_err = nullptr; // [2]
  cudaEvent_t ev_post[2] = {nullptr, nullptr};
  int64_t posted = 0, taken = 0;
  // off-lattice set: per particle 8 corner offsets, weights, weight gradients;
  // the last sample's Q per chain; running force sums [chain][particle][3]
  bool off = false;
  uint32_t *d_oidx = nullptr;
  double *d_ow = nullptr, *d_og = nullptr, *d_lastQ = nullptr, *d_fsum = nullptr;
  std::vector<double> pos;  // off-lattice positions (x, y, z) per particle
  // near pairs (CSR over particles, both directions); gather blocks nblk_g,
  // near-pair blocks after them (nblk = row length of the partials)
  int nblk_g = 0;
  int64_t n_pairs = 0;
  int64_t *d_nptr = nullptr;
  uint32_t *d_nbr = nullptr;
  double *d_t = nullptr, *d_u = nullptr;
  double *d_log = nullptr;       // [sample][chain][3]
  int64_t log_cap = 0;
  size_t bytes = 0;
  // pinned staging for coulps_charges_update
  uint32_t *h_idx = nullptr;
  double *h_q = nullptr;
  cudaEvent_t staged = nullptr;  // recorded after the last upload's copies
  // host copy of the set (to regroup it for the fused gather)
  std::vector<int32_t> sites;
  std::vector<double> qv;
  // fused gather: charges grouped by (y tile, z plane) of the lattice's tile
  bool gather_dirty = true;
  Tile gather_tile = {0, 0};
  size_t goff_n = 0;
  uint32_t *d_goff = nullptr, *d_gent = nullptr;
  double *d_gq = nullptr;
  double *d_fpart = nullptr;  // [chain][y tiles * z slabs][2]
  size_t fpart_n = 0;
  int fused_nblk = 0;
  uint32_t *h_goff = nullptr, *h_gent = nullptr;
  double *h_gq = nullptr;
  size_t h_goff_cap = 0;
  cudaEvent_t gstaged = nullptr;
};

namespace {

#define CK(expr)                          \
  do {                                    \
    cudaError_t e_ = (expr);              \
    if (e_ != cudaSuccess) {              \
      cudaGetLastError();                 \
      return COULPS_ECUDA;                \
    }                                     \
  } while (0)

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 coulps::tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  }
  return fn;
}

namespace {

// 4D map over field[chain*2 + colour][z][y][h] with a box of `rows` rows of W
// elements of one plane.  Out-of-range boxes read as zeros.
int make_map(CUtensorMap *m, const Geometry &g, void *base, int rows) {
  auto fn = tensor_map_encoder();
  if (!fn) return COULPS_ECUDA;
  cuuint64_t dims[4] = {(cuuint64_t)g.W, (cuuint64_t)g.Ly, (cuuint64_t)g.Lz,
                        (cuuint64_t)g.n_chains * 2};
  cuuint64_t strides[3] = {(cuuint64_t)g.W * g.es, (cuuint64_t)g.W * g.Ly * g.es,
                           (cuuint64_t)g.W * g.Ly * g.Lz * g.es};
  cuuint32_t box[4] = {(cuuint32_t)g.W, (cuuint32_t)rows, 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = fn(m,
                  g.precision == COULPS_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                            : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                  4, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? COULPS_OK : COULPS_ECUDA;
}

int rebuild_maps(coulps_lattice *L) {
  int st = make_map(&L->tm_halo, L->g, L->field, L->tile.ty + 2);
  if (st) return st;
  if (L->field2) {
    st = make_map(&L->tm_halo2, L->g, L->field2, L->tile.ty + 2);
    if (st) return st;
  }
  return make_map(&L->tm_own, L->g, L->field, L->tile.ty);
}

// Fused-pass tile: rows + 2 halo rows of quads per CTA within 256 threads,
// an odd row count (measured a little faster at 128^3: 13 rows 0.202 ms, 14
// rows 0.211 ms per pass of 64 chains); z slabs of 32 planes (several CTAs
// per column fill the GPU's slots evenly).  Rows of more than 42 quads leave
// fewer than 5 rows in 256 threads, and the 4 halo rows of colour 1 are then
// re-read for every row or two: such rows take up to 512 threads (measured,
// one chain: 512^3 0.321 ms per pass with 1 row, 0.221 with 3, 0.183 with 5;
// 384^3 0.104 with 7 rows; at 256^3 the 256-thread 5 rows are faster than 9
// or 13 rows: 0.039, 0.041, 0.049 ms).
Tile default_pass_tile(const Geometry &g) {
  const int qw = g.W / 4;
  int ty = 256 / qw - 2;
  if (ty < 4) ty = 512 / qw - 2;
  if (ty > 1 && ty % 2 == 0) --ty;
  if (ty < 1) ty = 1;
  if (ty > g.Ly) ty = g.Ly;
  if (ty > 252) ty = 252;  // TMA box rows ty + 4 <= 256
  int dz = g.Lz >= 64 ? 32 : g.Lz;
  while (ty > 1 && pass_smem_bytes(g, Tile{ty, dz}, true) > 227 * 1024) ty -= ty > 2 ? 2 : 1;
  return Tile{ty, dz};
}

// Pass-pair tile: the CTA computes ty + 6 rows (3 halo rows each side) of
// W / 4 quads, one thread per quad, within 512 threads (FP32) or 256 (FP64);
// {0, 0} when fewer than 4 rows fit (the halo would dominate).  z slabs of
// 64 planes from Lz = 128 (measured at 128^3 x 64 chains, two streams: 0.802
// ms per 1 HB : 3 OR compound sweep against 0.828 with 32 planes).
Tile default_pair_tile(const Geometry &g) {
  const int qw = g.W / 4;
  const int max_threads = g.precision == COULPS_F32 ? kPairMaxThreads32 : kPairMaxThreads64;
  int ty = max_threads / qw - 6;
  if (ty > g.Ly) ty = g.Ly;
  if (ty > 248) ty = 248;  // TMA box rows ty + 8 <= 256
  const int dz = g.Lz >= 128 ? 64 : (g.Lz >= 64 ? 32 : g.Lz);
  while (ty >= 1 && pair_smem_bytes(g, Tile{ty, dz}, true) > 227 * 1024) --ty;
  if (ty < 4 && ty < g.Ly) return Tile{0, 0};
  if (ty < 1) return Tile{0, 0};
  return Tile{ty, dz};
}

// SMs of the current device (0 if the query fails).
int device_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// Halves a default tile's z slab (not below min_dz) while one launch over all
// chains would have fewer than `target` CTAs: a single 128^3 chain otherwise
// gives the pass pair 10 CTAs and the heatbath half-sweep 64 on 152 SMs.
// Shorter slabs add halo planes (1 for a half-sweep or fused pass, 3 for a
// pair), so lattices with enough CTAs keep the measured slabs.
Tile fill_grid(const Geometry &g, Tile t, int target, int min_dz) {
  if (t.ty < 1 || t.dz < 1) return t;
  const int64_t rows = (g.Ly + t.ty - 1) / t.ty;
  while (t.dz > min_dz && rows * ((g.Lz + t.dz - 1) / t.dz) * g.n_chains < target)
    t.dz = std::max(min_dz, (t.dz + 1) / 2);
  return t;
}

int rebuild_pass_maps(coulps_lattice *L) {
  if (!L->fused) return COULPS_OK;
  for (int b = 0; b < 2; ++b) {
    void *base = b ? L->field2 : L->field;
    int st = make_map(&L->tm_p1[b], L->g, base, L->ptile.ty + 4);
    if (st) return st;
    st = make_map(&L->tm_p0[b], L->g, base, L->ptile.ty + 2);
    if (st) return st;
    if (L->fused >= 3 && L->qtile.ty > 0) {
      st = make_map(&L->tm_q1[b], L->g, base, L->qtile.ty + 8);
      if (st) return st;
      st = make_map(&L->tm_q0[b], L->g, base, L->qtile.ty + 6);
      if (st) return st;
    }
  }
  return COULPS_OK;
}

// Trips of n >= 2 passes run as pass pairs: `pairs` pass pairs, then
// `singles` fused single passes, with pairs + singles even so that the
// passes, which flip between the two copies on every trip, end in the copy
// they started from.
void pair_plan(int n, int &pairs, int &singles) {
  switch (n % 4) {
    case 0: pairs = n / 2; singles = 0; break;
    case 1: pairs = (n - 3) / 2; singles = 3; break;
    case 2: pairs = n / 2 - 1; singles = 2; break;
    default: pairs = (n - 1) / 2; singles = 1; break;
  }
}

// How the passes of one compound sweep run: passes [0, head) as
// half-sweeps (in place on the field, or, with flip, the first one out of
// place into field2 and the rest in place there), then `pairs` pass pairs and
// `singles` fused single passes (the trips, alternating between the copies,
// from field2 with flip and from the field otherwise, ending in the field),
// then the remaining passes as in-place half-sweeps on the field.
struct PassPlan {
  int head = 0;
  bool flip = false;
  int pairs = 0, singles = 0;
};

PassPlan pass_plan(const coulps_lattice *L, int n_hb, int n_or) {
  const int n = n_hb + n_or;
  PassPlan P;
  const bool pairs_ok = L->qtile.ty > 0;
  int mode = L->fused;
  if (mode == 3 && !pairs_ok) mode = 1;
  if (mode == 4 && !pairs_ok) mode = 2;
  if (mode == 1 || mode == 3) {
    // heatbath passes as half-sweeps, the over-relaxation block as trips
    P.head = n_hb;
    int d = mode == 3 ? n_or / 2 : 0, s = mode == 3 ? n_or % 2 : n_or;
    if ((d + s) % 2 == 1) {
      if (n_hb > 0) {
        P.flip = true;  // the heatbath passes write field2: an odd trip count ends in the field
      } else if (d >= 1) {
        d -= 1;
        s += 2;
      } else {
        s -= 1;  // one pass left: it runs as half-sweeps after the trips
      }
    }
    P.pairs = d;
    P.singles = s;
  } else if (mode == 2) {
    P.singles = n & ~1;
  } else if (mode == 4 && n >= 2) {
    pair_plan(n, P.pairs, P.singles);
  }
  return P;
}

// The tile by which the last kernel of a measured compound sweep (aligned
// schedule) gathers Q and P: the pass pair's, the fused pass's, or the
// half-sweep's.
Tile fused_gather_tile(const coulps_lattice *L, int n_hb, int n_or) {
  const int n = n_hb + n_or;
  const PassPlan P = pass_plan(L, n_hb, n_or);
  if (P.head + 2 * P.pairs + P.singles < n || P.pairs + P.singles == 0) return L->tile;
  return P.singles > 0 ? L->ptile : L->qtile;
}

Tile default_tile(const Geometry &g) {
  // About 256 threads per CTA (W/4 threads per row), 16 z planes per CTA.
  const int qw = g.W / 4;
  int ty = 256 / qw;
  if (ty < 1) ty = 1;
  if (ty > 254) ty = 254;  // TMA box rows ty + 2 <= 256
  if (ty > g.Ly) ty = g.Ly;
  while (ty > 1 && qw * ty > 1024) --ty;
  int dz = g.Lz < 16 ? g.Lz : 16;
  return Tile{ty, dz};
}

// Self-test of the failure path of a bounded device wait: one thread polls a
// word that nothing ever sets, gives up after limit_ns of %globaltimer time
// and records a timeout in the lattice's error word, as every sweep kernel's
// bounded mbarrier wait does.
__device__ int g_never_set = 0;

__global__ void selftest_wait_kernel(int *err, uint64_t limit_ns) {
  if (threadIdx.x != 0) return;
  volatile int *flag = &g_never_set;
  const uint64_t t0 = global_timer_ns();
  while (*flag == 0) {
    if (global_timer_ns() - t0 > limit_ns) {
      atomicOr(err, kErrTimeout);
      return;
    }
    __nanosleep(1000);
  }
}

int check_device_error(coulps_lattice *L) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, L->d_err, sizeof(int), cudaMemcpyDeviceToHost, L->stream));
  CK(cudaStreamSynchronize(L->stream));
  if (h & kErrTimeout) return COULPS_ETIMEOUT;
  if (h & kErrNonFinite) return COULPS_ENONFINITE;
  return COULPS_OK;
}

// Queue the half-sweeps of one compound sweep.  The pass index of every
// half-sweep is read on the device as *d_pass + offset, and the counter is
// advanced at the end, so the same launches can be captured once and
// replayed.
cudaEvent_t take_event(coulps_lattice *L) {
  if (!L->spare_events.empty()) {
    cudaEvent_t e = L->spare_events.back();
    L->spare_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// The passes of one compound sweep for the chains chain0, chain0 + stride,
// ... on stream `st`, with their measurement when `fuse` is given: its Q, P
// are gathered by the sweep's last kernel, by the tile fused_gather_tile
// names (the pass counter is advanced by the caller).
// Which passes of the plan enqueue_part queues: all of them, the head only
// (the heatbath half-sweeps of modes 1 and 3), or the rest only (the trips
// and tail, with their gather), the rest's pass indices offset by `shift`.
enum PartRange { kPartAll = 0, kPartHead = 1, kPartRest = 2 };

int enqueue_part(coulps_lattice *L, cudaStream_t st, int n_hb, int n_or, coulps_charges *fuse,
                 int chain0, int stride, int range = kPartAll, uint32_t shift = 0u) {
  SweepArgs a;
  a.chain0 = chain0;
  a.chain_stride = stride;
  a.field = L->field;
  a.Lx = L->g.Lx; a.Ly = L->g.Ly; a.Lz = L->g.Lz;
  a.W = L->g.W; a.Wq = L->g.Wq; a.QW = L->g.W / 4;
  a.TY = L->tile.ty; a.DZ = L->tile.dz;
  {
    const PhiloxKeys K = philox_keys((uint32_t)(L->seed & 0xffffffffu), (uint32_t)(L->seed >> 32));
    for (int i = 0; i < 20; ++i) a.round_keys[i] = K.k[i];
  }
  a.pass_ptr = L->d_pass;
  a.chain_elems = L->g.chain_elems;
  a.colour_elems = L->g.colour_elems;
  a.err = L->d_err;
  a.g_off = nullptr;
  a.g_ent = nullptr;
  a.g_q = nullptr;
  a.g_partials = nullptr;
  const int n_pass = n_hb + n_or;
  if (fuse) {
    // the charges must be grouped by the tile of the kernel that gathers
    const Tile gt = fused_gather_tile(L, n_hb, n_or);
    if (fuse->gather_dirty || fuse->gather_tile.ty != gt.ty || fuse->gather_tile.dz != gt.dz)
      return COULPS_EINVAL;
  }
  PassArgs p;
  p.chain0 = chain0;
  p.chain_stride = stride;
  p.Lx = a.Lx; p.Ly = a.Ly; p.Lz = a.Lz;
  p.W = a.W; p.Wq = a.Wq; p.QW = a.QW;
  for (int i = 0; i < 20; ++i) p.round_keys[i] = a.round_keys[i];
  p.pass_ptr = L->d_pass;
  p.chain_elems = a.chain_elems;
  p.colour_elems = a.colour_elems;
  p.err = L->d_err;
  p.g_off = nullptr;
  p.g_ent = nullptr;
  p.g_q = nullptr;
  p.g_partials = nullptr;
  auto set_gather = [&](PassArgs &q) {
    q.g_off = fuse->d_goff;
    q.g_ent = fuse->d_gent;
    q.g_q = fuse->d_gq;
    q.g_partials = fuse->d_fpart;
  };
  auto timed = [&](int kind, auto &&launch) -> int {
    cudaEvent_t ea = nullptr, eb = nullptr;
    if (L->profiling) {
      ea = take_event(L);
      eb = take_event(L);
      if (!ea || !eb) return COULPS_ECUDA;
      CK(cudaEventRecord(ea, st));
    }
    CK(launch());
    if (L->profiling) {
      CK(cudaEventRecord(eb, st));
      L->pending.push_back({ea, eb, kind});
    }
    return COULPS_OK;
  };

  const PassPlan plan = pass_plan(L, n_hb, n_or);
  const int trips = plan.pairs + plan.singles;
  const int tail0 = plan.head + 2 * plan.pairs + plan.singles;  // first pass of the tail
  // one pass as two half-sweeps: on2 -- the pass runs on field2 (heatbath
  // passes ahead of trips that start from field2: the first of them reads
  // colour 1 from the field and writes colour 0 into field2, a heatbath update
  // does not read the site's old value, so this moves no extra bytes)
  auto half_sweeps = [&](int i, bool on2, bool gather) -> int {
    const bool orx = i >= n_hb;
    a.field = on2 ? L->field2 : L->field;
    for (int c = 0; c < 2; ++c) {
      a.colour = c;
      a.pass_off = (uint32_t)i + (i >= plan.head ? shift : 0u);
      // the other colour's rows come from field, except once field2 holds
      // them: colour 1 of the first pass, and every later pass
      const CUtensorMap &halo = on2 && (i > 0 || c == 1) ? L->tm_halo2 : L->tm_halo;
      if (gather && c == 1) {
        a.g_off = fuse->d_goff;
        a.g_ent = fuse->d_gent;
        a.g_q = fuse->d_gq;
        a.g_partials = fuse->d_fpart;
      }
      const int r = timed(orx ? 1 : 0, [&]() {
        return launch_halfsweep(L->g, L->tile, halo, L->tm_own, a, orx, st);
      });
      if (r) return r;
    }
    a.field = L->field;
    return COULPS_OK;
  };
  if (range != kPartRest)
    for (int i = 0; i < plan.head; ++i) {
      const int r =
          half_sweeps(i, plan.flip, fuse && trips == 0 && tail0 == n_pass && i == n_pass - 1);
      if (r) return r;
    }
  if (range == kPartHead) return COULPS_OK;
  // trips: pass pairs, then single fused passes, each from one copy to the other
  int i = plan.head;
  for (int t = 0; t < trips; ++t) {
    const int b = (t + (plan.flip ? 1 : 0)) & 1;  // source copy: 0 the field, 1 field2
    p.dst = b ? L->field : L->field2;
    p.pass_off = (uint32_t)i + shift;
    if (fuse && t == trips - 1 && tail0 == n_pass) set_gather(p);
    int r;
    if (t < plan.pairs) {
      const bool a_or = i >= n_hb, b_or = i + 1 >= n_hb;
      p.TY = L->qtile.ty; p.DZ = L->qtile.dz;
      r = timed(a_or && b_or ? 6 : 5, [&]() {
        return launch_pair(L->g, L->qtile, L->tm_q1[b], L->tm_q0[b], p, a_or, b_or, st);
      });
      i += 2;
    } else {
      const bool orx = i >= n_hb;
      p.TY = L->ptile.ty; p.DZ = L->ptile.dz;
      r = timed(orx ? 4 : 3, [&]() {
        return launch_pass(L->g, L->ptile, L->tm_p1[b], L->tm_p0[b], p, orx, st);
      });
      i += 1;
    }
    if (r) return r;
  }
  for (; i < n_pass; ++i) {
    const int r = half_sweeps(i, false, fuse && i == n_pass - 1);
    if (r) return r;
  }
  if (fuse && n_pass > 0) {  // (range is kPartAll or kPartRest here)
    if (chain0 == 0 && stride == 1)
      CK(launch_finalize(fuse->d_fpart, fuse->fused_nblk, L->g.n_chains, fuse->d_stats,
                         fuse->d_log, fuse->log_cap, L->d_err, st));
    else
      CK(launch_finalize_group(fuse->d_fpart, fuse->fused_nblk, L->g.n_chains, chain0, stride,
                               fuse->d_stats, fuse->d_log, fuse->log_cap, L->d_err, st));
  }
  return COULPS_OK;
}

// One compound sweep of every chain (and its sample when `fuse` is given).
// With k > 1 streams chain c runs on stream c % k: stream 0 is the lattice's,
// the others are forked from it at the start and joined back at the end
// (also under graph capture), so the groups' heatbath and over-relaxation
// kernels can share the GPU; each chain's passes, draws and sample are
// unchanged.  The pass counter is advanced once, after the join.
int enqueue_compound(coulps_lattice *L, int n_hb, int n_or, coulps_charges *fuse = nullptr) {
  const int k = L->split < L->g.n_chains ? L->split : L->g.n_chains;
  if (k >= 2) {
    CK(cudaEventRecord(L->ev_fork, L->stream));
    int r = COULPS_OK;
    for (int j = 1; j < k; ++j) {
      CK(cudaStreamWaitEvent(L->xstream[j - 1], L->ev_fork, 0));
      if (!r) r = enqueue_part(L, L->xstream[j - 1], n_hb, n_or, fuse, j, k);
    }
    if (!r) r = enqueue_part(L, L->stream, n_hb, n_or, fuse, 0, k);
    // join whatever was queued on the other streams, also on failure
    for (int j = 1; j < k; ++j) {
      CK(cudaEventRecord(L->ev_join[j - 1], L->xstream[j - 1]));
      CK(cudaStreamWaitEvent(L->stream, L->ev_join[j - 1], 0));
    }
    if (r) return r;
  } else {
    int r = enqueue_part(L, L->stream, n_hb, n_or, fuse, 0, 1);
    if (r) return r;
  }
  if (n_hb + n_or > 0) CK(launch_advance_pass(L->d_pass, (uint32_t)(n_hb + n_or), L->stream));
  return COULPS_OK;
}


// The shifted schedule (coulps_set_schedule): with two streams, the odd
// chains run half a compound sweep behind the even ones, so that one group's
// heatbath half-sweeps (instruction-bound) meet the other's over-relaxation
// kernels (memory-bound) throughout.  A run of n >= 2 measured compound
// sweeps is a prologue (even chains: sweep 0; odd chains: the heatbath
// passes of sweep 0), n - 1 steady steps (even: sweep k; odd: the
// over-relaxation passes and the sample of sweep k - 1, then the heatbath
// passes of sweep k) and an epilogue (odd: the over-relaxation passes and
// sample of the last sweep).  Every chain does exactly the passes, draws and
// samples of the aligned schedule; the pass counter advances by one sweep per
// prologue and steady step.
bool shifted_ok(const coulps_lattice *L, int n_hb, int n_or) {
  if (L->schedule != COULPS_SCHEDULE_SHIFTED || L->split != 2 || L->g.n_chains < 2) return false;
  if (n_hb < 1 || n_or < 1) return false;
  const PassPlan P = pass_plan(L, n_hb, n_or);
  return P.head == n_hb && P.head < n_hb + n_or;
}

int enqueue_shifted(coulps_lattice *L, int n_hb, int n_or, coulps_charges *fuse, int phase) {
  const int n = n_hb + n_or;
  const uint32_t back = (uint32_t)(-(int64_t)n);  // pass offsets of the previous sweep
  CK(cudaEventRecord(L->ev_fork, L->stream));
  CK(cudaStreamWaitEvent(L->xstream[0], L->ev_fork, 0));
  int r = COULPS_OK;
  if (phase == 0) {
    r = enqueue_part(L, L->xstream[0], n_hb, n_or, nullptr, 1, 2, kPartHead);
  } else {
    r = enqueue_part(L, L->xstream[0], n_hb, n_or, fuse, 1, 2, kPartRest, back);
    if (!r && phase == 1) r = enqueue_part(L, L->xstream[0], n_hb, n_or, nullptr, 1, 2, kPartHead);
  }
  if (!r && phase != 2) r = enqueue_part(L, L->stream, n_hb, n_or, fuse, 0, 2);
  CK(cudaEventRecord(L->ev_join[0], L->xstream[0]));
  CK(cudaStreamWaitEvent(L->stream, L->ev_join[0], 0));
  if (r) return r;
  if (phase != 2) CK(launch_advance_pass(L->d_pass, (uint32_t)n, L->stream));
  return COULPS_OK;
}



void drop_graph(coulps_lattice *L);

// Group the charge set by (y tile, z plane) of tile t (that of the kernel
// that gathers) and queue the upload of the lists the fused gather reads.
// Buffers are reused when their sizes do not change, so a captured graph
// stays valid.
int stage_gather(coulps_lattice *L, coulps_charges *C, Tile t) {
  const Geometry &g = L->g;
  if (!C->gather_dirty && C->gather_tile.ty == t.ty && C->gather_tile.dz == t.dz) return COULPS_OK;
  const int ytiles = (g.Ly + t.ty - 1) / t.ty, zslabs = (g.Lz + t.dz - 1) / t.dz;
  const size_t goff_n = (size_t)ytiles * g.Lz + 1;
  const size_t n = (size_t)C->n;
  const size_t fpart_n = (size_t)g.n_chains * ytiles * zslabs * 2;
  if (goff_n != C->goff_n || !C->d_goff) {
    drop_graph(L);
    dev_free(L->alloc, C->d_goff, L->stream);
    C->d_goff = (uint32_t *)dev_alloc(L->alloc, goff_n * sizeof(uint32_t), L->stream);
    if (!C->d_goff) return COULPS_ENOMEM;
    C->goff_n = goff_n;
  }
  if (!C->d_gent) {
    C->d_gent = (uint32_t *)dev_alloc(L->alloc, n * sizeof(uint32_t), L->stream);
    C->d_gq = (double *)dev_alloc(L->alloc, n * sizeof(double), L->stream);
    if (!C->d_gent || !C->d_gq) return COULPS_ENOMEM;
  }
  if (fpart_n != C->fpart_n || !C->d_fpart) {
    drop_graph(L);
    dev_free(L->alloc, C->d_fpart, L->stream);
    C->d_fpart = (double *)dev_alloc(L->alloc, fpart_n * sizeof(double), L->stream);
    if (!C->d_fpart) return COULPS_ENOMEM;
    C->fpart_n = fpart_n;
  }
  C->fused_nblk = ytiles * zslabs;
  if (!C->gstaged) {
    // all three or none: a failure leaves the set as it was
    uint32_t *he = nullptr;
    double *hq = nullptr;
    cudaEvent_t ev = nullptr;
    if (n > 0 && (cudaMallocHost((void **)&he, n * sizeof(uint32_t)) != cudaSuccess ||
                  cudaMallocHost((void **)&hq, n * sizeof(double)) != cudaSuccess)) {
      cudaGetLastError();
      if (he) cudaFreeHost(he);
      return COULPS_ENOMEM;
    }
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      if (he) cudaFreeHost(he);
      if (hq) cudaFreeHost(hq);
      return COULPS_ECUDA;
    }
    C->h_gent = he;
    C->h_gq = hq;
    C->gstaged = ev;
  } else {
    CK(cudaEventSynchronize(C->gstaged));  // the previous upload has left the staging
  }
  if (goff_n > C->h_goff_cap) {
    if (C->h_goff) cudaFreeHost(C->h_goff);
    C->h_goff = nullptr;
    if (cudaMallocHost((void **)&C->h_goff, goff_n * sizeof(uint32_t)) != cudaSuccess) {
      cudaGetLastError();
      C->h_goff_cap = 0;
      return COULPS_ENOMEM;
    }
    C->h_goff_cap = goff_n;
  }
  // counting sort by key = y_tile * Lz + z
  std::vector<uint32_t> count(goff_n, 0);
  for (size_t i = 0; i < n; ++i) {
    const int y = C->sites[3 * i + 1], z = C->sites[3 * i + 2];
    count[(size_t)(y / t.ty) * g.Lz + z + 1]++;
  }
  for (size_t k = 1; k < goff_n; ++k) count[k] += count[k - 1];
  for (size_t k = 0; k < goff_n; ++k) C->h_goff[k] = count[k];
  for (size_t i = 0; i < n; ++i) {
    const int x = C->sites[3 * i], y = C->sites[3 * i + 1], z = C->sites[3 * i + 2];
    const int yt = y / t.ty;
    const uint32_t pos = count[(size_t)yt * g.Lz + z]++;
    const uint32_t colour = (uint32_t)((x + y + z) & 1);
    C->h_gent[pos] = (colour << 31) | (uint32_t)(((size_t)z * g.Ly + y) * g.W + (x >> 1));
    C->h_gq[pos] = C->qv[i];
  }
  CK(cudaMemcpyAsync(C->d_goff, C->h_goff, goff_n * sizeof(uint32_t), cudaMemcpyHostToDevice,
                     L->stream));
  if (n > 0) {
    CK(cudaMemcpyAsync(C->d_gent, C->h_gent, n * sizeof(uint32_t), cudaMemcpyHostToDevice,
                       L->stream));
    CK(cudaMemcpyAsync(C->d_gq, C->h_gq, n * sizeof(double), cudaMemcpyHostToDevice, L->stream));
  }
  CK(cudaEventRecord(C->gstaged, L->stream));
  C->gather_tile = t;
  C->gather_dirty = false;
  return COULPS_OK;
}

int enqueue_measure(coulps_lattice *L, coulps_charges *C) {
  if (C->off) {
    const bool near = C->n_pairs > 0;
    CK(launch_gather_off(L->g, L->field, C->d_oidx, C->d_ow, C->d_q, C->n, C->d_partials,
                         C->nblk_g, C->nblk, near ? C->d_t : nullptr, L->stream));
    if (near)
      CK(launch_near(C->d_t, C->d_nptr, C->d_nbr, C->n, L->g.n_chains, C->d_u, C->d_partials,
                     C->nblk, C->nblk_g, L->stream));
    CK(launch_finalize(C->d_partials, C->nblk, L->g.n_chains, C->d_stats, C->d_log, C->log_cap,
                       L->d_err, L->stream, C->d_lastQ));
    if (C->d_fsum)
      CK(launch_force_off(L->g, L->field, C->d_oidx, C->d_ow, C->d_og, C->d_q, C->n, C->d_lastQ,
                          near ? C->d_u : nullptr, C->d_fsum, L->stream));
    return COULPS_OK;
  }
  CK(launch_gather(L->g, L->field, C->d_idx, C->d_q, C->n, C->d_partials, C->nblk, L->stream));
  CK(launch_finalize(C->d_partials, C->nblk, L->g.n_chains, C->d_stats, C->d_log, C->log_cap,
                     L->d_err, L->stream));
  return COULPS_OK;
}

// Every set samples the current fields: kMaxSets per gather launch.
int enqueue_measure_sets(coulps_lattice *L, coulps_charges *const *sets, int n_sets) {
  // off-lattice sets one by one, the others kMaxSets per launch
  std::vector<coulps_charges *> on;
  for (int k = 0; k < n_sets; ++k) {
    if (sets[k]->off) {
      int st = enqueue_measure(L, sets[k]);
      if (st) return st;
    } else {
      on.push_back(sets[k]);
    }
  }
  n_sets = (int)on.size();
  for (int k0 = 0; k0 < n_sets; k0 += kMaxSets) {
    SetTable t;
    t.n_sets = n_sets - k0 < kMaxSets ? n_sets - k0 : kMaxSets;
    for (int k = 0; k < t.n_sets; ++k) {
      coulps_charges *C = on[k0 + k];
      t.idx[k] = C->d_idx;
      t.q[k] = C->d_q;
      t.n[k] = C->n;
      t.partials[k] = C->d_partials;
      t.nblk[k] = C->nblk;
      t.stats[k] = C->d_stats;
      t.log[k] = C->d_log;
      t.log_cap[k] = C->log_cap;
    }
    CK(launch_measure_sets(L->g, L->field, t, L->d_err, L->stream));
  }
  return COULPS_OK;
}

void drop_graph(coulps_lattice *L) {
  // launches of these graphs may still be queued: let them finish first
  if (L->graph || L->sgraph || L->mgraph || L->hgraph[0]) cudaStreamSynchronize(L->stream);
  for (auto &h : L->hgraph) {
    if (h) cudaGraphExecDestroy(h);
    h = nullptr;
  }
  L->hgraph_key = nullptr;
  if (L->mgraph) cudaGraphExecDestroy(L->mgraph);
  L->mgraph = nullptr;
  L->mgraph_key.clear();
  if (L->graph) cudaGraphExecDestroy(L->graph);
  L->graph = nullptr;
  L->graph_key = nullptr;
  if (L->sgraph) cudaGraphExecDestroy(L->sgraph);
  L->sgraph = nullptr;
  L->sgraph_key = nullptr;
}

// The measured phase of coulps_run on the shifted schedule (see
// enqueue_shifted): prologue, n_meas - 1 steady steps, epilogue, each a
// cached CUDA graph when the stream can be captured.
int run_shifted(coulps_lattice *L, coulps_charges *C, int n_meas, int n_hb, int n_or) {
  const bool capturable = L->stream != nullptr && !L->profiling;
  if (capturable &&
      (L->hgraph_key != C || L->hgraph_hb != n_hb || L->hgraph_or != n_or || !L->hgraph[0])) {
    drop_graph(L);
    for (int ph = 0; ph < 3; ++ph) {
      cudaGraph_t gr = nullptr;
      CK(cudaStreamBeginCapture(L->stream, cudaStreamCaptureModeThreadLocal));
      const int s1 = enqueue_shifted(L, n_hb, n_or, C, ph);
      cudaError_t e = cudaStreamEndCapture(L->stream, &gr);
      if (s1 || e != cudaSuccess) {
        cudaGetLastError();
        if (gr) cudaGraphDestroy(gr);
        drop_graph(L);
        return s1 ? s1 : COULPS_ECUDA;
      }
      e = cudaGraphInstantiate(&L->hgraph[ph], gr, 0);
      cudaGraphDestroy(gr);
      if (e != cudaSuccess) {
        cudaGetLastError();
        L->hgraph[ph] = nullptr;
        drop_graph(L);
        return COULPS_ECUDA;
      }
    }
    L->hgraph_key = C;
    L->hgraph_hb = n_hb;
    L->hgraph_or = n_or;
  }
  auto phase = [&](int ph) -> int {
    if (capturable) {
      CK(cudaGraphLaunch(L->hgraph[ph], L->stream));
      return COULPS_OK;
    }
    return enqueue_shifted(L, n_hb, n_or, C, ph);
  };
  int st = phase(0);
  for (int k = 1; k < n_meas && !st; ++k) st = phase(1);
  if (!st) st = phase(2);
  return st;
}

// ---- phase-shifted schedule ------------------------------------------------
// Chain k is in group k % P (P = passes per compound sweep) and runs P - ...
// its pass p at slot t = p + g.  In every launch of the steady state one
// group does heatbath passes while the others do over-relaxation, so the
// ALU-bound and the memory-bound half-sweeps share the GPU.  Every chain
// still does exactly the passes and samples of the aligned schedule.
//
// One slot: red and black mixed half-sweeps, then the finalize of any group
// that completed a measured compound sweep.  The pass index of group g is
// *d_pass + (t - g - t_dev), where the device counter holds B + t_dev.
int enqueue_slot(coulps_lattice *L, coulps_charges *C, int n_hb, int n_or, int64_t t,
                 int64_t t_dev, int64_t T) {
  const int P = n_hb + n_or;
  MixedArgs m;
  std::memset(&m, 0, sizeof(m));
  SweepArgs &a = m.base;
  a.chain0 = 0;
  a.chain_stride = 1;
  a.field = L->field;
  a.Lx = L->g.Lx; a.Ly = L->g.Ly; a.Lz = L->g.Lz;
  a.W = L->g.W; a.Wq = L->g.Wq; a.QW = L->g.W / 4;
  a.TY = L->tile.ty; a.DZ = L->tile.dz;
  {
    const PhiloxKeys K = philox_keys((uint32_t)(L->seed & 0xffffffffu), (uint32_t)(L->seed >> 32));
    for (int i = 0; i < 20; ++i) a.round_keys[i] = K.k[i];
  }
  a.pass_ptr = L->d_pass;
  a.chain_elems = L->g.chain_elems;
  a.colour_elems = L->g.colour_elems;
  a.err = L->d_err;
  a.g_off = C->d_goff;
  a.g_ent = C->d_gent;
  a.g_q = C->d_gq;
  a.g_partials = C->d_fpart;
  m.groups = P;
  bool any_gather = false;
  for (int g = 0; g < P; ++g) {
    const int64_t p = t - g;
    const bool active = p >= 0 && p < T;
    m.mode[g] = active ? ((p % P) < n_hb ? 1 : 2) : 0;
    m.pass_delta[g] = (uint32_t)(p - t_dev);
  }
  for (int c = 0; c < 2; ++c) {
    a.colour = c;
    for (int g = 0; g < P; ++g) {
      const int64_t p = t - g;
      m.gather[g] = (c == 1 && m.mode[g] != 0 && p % P == P - 1) ? 1 : 0;
      any_gather = any_gather || m.gather[g];
    }
    cudaEvent_t ea = nullptr, eb = nullptr;
    if (L->profiling) {
      ea = take_event(L);
      eb = take_event(L);
      if (!ea || !eb) return COULPS_ECUDA;
      CK(cudaEventRecord(ea, L->stream));
    }
    CK(launch_halfsweep_mixed(L->g, L->tile, L->tm_halo, L->tm_own, m, L->stream));
    if (L->profiling) {
      CK(cudaEventRecord(eb, L->stream));
      L->pending.push_back({ea, eb, 2});
    }
  }
  if (any_gather)
    for (int g = 0; g < P; ++g)
      if (m.gather[g])
        CK(launch_finalize_group(C->d_fpart, C->fused_nblk, L->g.n_chains, g, P, C->d_stats,
                                 C->d_log, C->log_cap, L->d_err, L->stream));
  return COULPS_OK;
}

// The measured phase of coulps_run on the phase-shifted schedule (all chains
// start aligned at pass counter B and end aligned at B + n_meas * P).
int run_staggered(coulps_lattice *L, coulps_charges *C, int n_meas, int n_hb, int n_or) {
  const int P = n_hb + n_or;
  const int64_t T = (int64_t)n_meas * P;
  int st;
  // prologue: slots 0 .. P-2 (no group completes a compound sweep yet)
  for (int64_t t = 0; t < P - 1; ++t)
    if ((st = enqueue_slot(L, C, n_hb, n_or, t, 0, T))) return st;
  CK(launch_advance_pass(L->d_pass, (uint32_t)(P - 1), L->stream));
  int64_t t_dev = P - 1;
  // steady state: n_meas - 1 periods of P slots, one graph
  const bool capturable = L->stream != nullptr && !L->profiling;
  auto enqueue_period = [&](int64_t t0) -> int {
    for (int s = 0; s < P; ++s) {
      int r = enqueue_slot(L, C, n_hb, n_or, t0 + s, t0, T);
      if (r) return r;
    }
    CK(launch_advance_pass(L->d_pass, (uint32_t)P, L->stream));
    return COULPS_OK;
  };
  if (n_meas > 1 && capturable &&
      (L->sgraph_key != C || L->sgraph_hb != n_hb || L->sgraph_or != n_or ||
       L->sgraph_tile.ty != L->tile.ty || L->sgraph_tile.dz != L->tile.dz)) {
    if (L->sgraph) cudaGraphExecDestroy(L->sgraph);
    L->sgraph = nullptr;
    cudaGraph_t gr = nullptr;
    CK(cudaStreamBeginCapture(L->stream, cudaStreamCaptureModeThreadLocal));
    // a steady period is the same for every t0 once T is large: capture it
    // with T large enough that no group is idle
    const int s1 = enqueue_period(t_dev);
    cudaError_t e = cudaStreamEndCapture(L->stream, &gr);
    if (s1 || e != cudaSuccess) {
      cudaGetLastError();
      if (gr) cudaGraphDestroy(gr);
      return s1 ? s1 : COULPS_ECUDA;
    }
    e = cudaGraphInstantiate(&L->sgraph, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
      cudaGetLastError();
      L->sgraph = nullptr;
      return COULPS_ECUDA;
    }
    L->sgraph_key = C;
    L->sgraph_hb = n_hb;
    L->sgraph_or = n_or;
    L->sgraph_tile = L->tile;
  }
  for (int k = 0; k < n_meas - 1; ++k) {
    if (capturable) {
      CK(cudaGraphLaunch(L->sgraph, L->stream));
    } else if ((st = enqueue_period(t_dev))) {
      return st;
    }
    t_dev += P;
  }
  // epilogue: slots T - 1 .. T + P - 2
  for (int64_t t = t_dev; t < T + P - 1; ++t)
    if ((st = enqueue_slot(L, C, n_hb, n_or, t, t_dev, T))) return st;
  CK(launch_advance_pass(L->d_pass, (uint32_t)(T - t_dev), L->stream));
  return COULPS_OK;
}

// Corner storage offsets (in a chain's field), trilinear weights and weight
// gradients of n particles at real positions pos (x, y, z): base site
// b = floor(r) clipped to L - 2, f = r - b, corner c = (cx, cy, cz) with cx
// slowest, weight prod_mu (c_mu ? f_mu : 1 - f_mu).  False if a position is
// outside [0, L - 1] or not finite, or a dimension is < 2.
bool offlattice_corners(int Lx, int Ly, int Lz, int W, size_t colour_elems, int64_t n,
                        const double *pos, uint32_t *oidx, double *ow, double *og) {
  const int Ls[3] = {Lx, Ly, Lz};
  if (Lx < 2 || Ly < 2 || Lz < 2) return false;
  for (int64_t i = 0; i < n; ++i) {
    int b[3];
    double f[3];
    for (int mu = 0; mu < 3; ++mu) {
      const double r = pos[3 * i + mu];
      if (!(r >= 0.0 && r <= (double)(Ls[mu] - 1))) return false;
      int bi = (int)std::floor(r);
      if (bi > Ls[mu] - 2) bi = Ls[mu] - 2;
      b[mu] = bi;
      f[mu] = r - bi;
    }
    for (int c = 0; c < 8; ++c) {
      const int cc[3] = {(c >> 2) & 1, (c >> 1) & 1, c & 1};
      double fac[3], dfac[3];
      for (int mu = 0; mu < 3; ++mu) {
        fac[mu] = cc[mu] ? f[mu] : 1.0 - f[mu];
        dfac[mu] = cc[mu] ? 1.0 : -1.0;
      }
      const int x = b[0] + cc[0], y = b[1] + cc[1], z = b[2] + cc[2];
      const int col = (x + y + z) & 1;
      oidx[8 * i + c] =
          (uint32_t)((size_t)col * colour_elems + ((size_t)z * Ly + y) * W + (x >> 1));
      ow[8 * i + c] = fac[0] * fac[1] * fac[2];
      og[3 * (8 * i + c) + 0] = dfac[0] * fac[1] * fac[2];
      og[3 * (8 * i + c) + 1] = fac[0] * dfac[1] * fac[2];
      og[3 * (8 * i + c) + 2] = fac[0] * fac[1] * dfac[2];
    }
  }
  return true;
}

// Near partners of n particles (|r_i - r_j| < rc, j != i) as CSR, both
// directions, each list ascending: ptr (n + 1 entries) and nbr.  Pairs are
// found through a grid of cells of edge >= rc (a particle's partners lie in
// its own or the 26 adjacent cells); the grid is coarsened until it has at
// most 8 n + 64 cells.
void near_csr(const double *p, int64_t n, double rc, std::vector<int64_t> &ptr,
              std::vector<uint32_t> &nbr) {
  ptr.assign((size_t)n + 1, 0);
  nbr.clear();
  if (!(rc > 0.0) || n < 2) return;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = 0; i < n; ++i)
    for (int mu = 0; mu < 3; ++mu) {
      lo[mu] = std::min(lo[mu], p[3 * i + mu]);
      hi[mu] = std::max(hi[mu], p[3 * i + mu]);
    }
  double cs = rc;
  int64_t nd[3];
  for (;;) {
    for (int mu = 0; mu < 3; ++mu) nd[mu] = (int64_t)std::floor((hi[mu] - lo[mu]) / cs) + 1;
    if ((double)nd[0] * nd[1] * nd[2] <= 8.0 * (double)n + 64.0) break;
    cs *= 1.5;
  }
  auto cell_of = [&](int64_t i, int mu) {
    int64_t c = (int64_t)std::floor((p[3 * i + mu] - lo[mu]) / cs);
    return c < 0 ? 0 : (c >= nd[mu] ? nd[mu] - 1 : c);
  };
  const int64_t ncell = nd[0] * nd[1] * nd[2];
  std::vector<int64_t> cstart((size_t)ncell + 1, 0), cell((size_t)n), order((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    cell[i] = (cell_of(i, 2) * nd[1] + cell_of(i, 1)) * nd[0] + cell_of(i, 0);
    cstart[cell[i] + 1]++;
  }
  for (int64_t c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
  {
    std::vector<int64_t> fill(cstart.begin(), cstart.end() - 1);
    for (int64_t i = 0; i < n; ++i) order[fill[cell[i]]++] = i;
  }
  std::vector<uint32_t> mine;
  for (int64_t i = 0; i < n; ++i) {
    mine.clear();
    const int64_t cx = cell_of(i, 0), cy = cell_of(i, 1), cz = cell_of(i, 2);
    for (int64_t z = std::max<int64_t>(cz - 1, 0); z <= std::min(cz + 1, nd[2] - 1); ++z)
      for (int64_t y = std::max<int64_t>(cy - 1, 0); y <= std::min(cy + 1, nd[1] - 1); ++y)
        for (int64_t x = std::max<int64_t>(cx - 1, 0); x <= std::min(cx + 1, nd[0] - 1); ++x) {
          const int64_t c = (z * nd[1] + y) * nd[0] + x;
          for (int64_t k = cstart[c]; k < cstart[c + 1]; ++k) {
            const int64_t j = order[k];
            if (j == i) continue;
            const double dx = p[3 * i] - p[3 * j], dy = p[3 * i + 1] - p[3 * j + 1],
                         dz = p[3 * i + 2] - p[3 * j + 2];
            if (std::sqrt(dx * dx + dy * dy + dz * dz) < rc) mine.push_back((uint32_t)j);
          }
        }
    std::sort(mine.begin(), mine.end());
    nbr.insert(nbr.end(), mine.begin(), mine.end());
    ptr[i + 1] = (int64_t)nbr.size();
  }
}

uint64_t fnv1a(uint64_t h, const void *p, size_t n) {
  const unsigned char *b = static_cast<const unsigned char *>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

}  // namespace

extern "C" {

const char *coulps_error_string(int status) {
  switch (status) {
    case COULPS_OK: return "ok";
    case COULPS_EINVAL: return "invalid argument";
    case COULPS_ENOMEM: return "out of memory";
    case COULPS_ECUDA: return "CUDA runtime error";
    case COULPS_ETIMEOUT: return "device wait timed out";
    case COULPS_ENONFINITE: return "non-finite sample";
    case COULPS_EIO: return "checkpoint I/O error";
    case COULPS_ECORRUPT: return "checkpoint corrupt or mismatched";
    case COULPS_EUNSUPPORTED: return "unsupported shape or mode";
    default: return "unknown status";
  }
}

int coulps_version(void) { return 100; }

int coulps_set_allocator(coulps_alloc_fn alloc, coulps_free_fn free_fn, void *ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return COULPS_EINVAL;
  g_allocator = Allocator{alloc, free_fn, ctx};
  return COULPS_OK;
}

int coulps_lattice_create(int Lx, int Ly, int Lz, int n_chains, int precision, uint64_t seed,
                          void *stream, coulps_lattice_t *out) {
  if (!out) return COULPS_EINVAL;
  *out = nullptr;
  if (Lx < 1 || Ly < 1 || Lz < 1 || Lx > 512 || Ly > 65535 || Lz > 65535) return COULPS_EINVAL;
  if (n_chains < 1 || n_chains > 65535) return COULPS_EINVAL;
  if (precision != COULPS_F32 && precision != COULPS_F64) return COULPS_EINVAL;
  Geometry g;
  g.Lx = Lx; g.Ly = Ly; g.Lz = Lz;
  g.n_chains = n_chains;
  g.precision = precision;
  g.es = precision == COULPS_F32 ? 4 : 8;
  g.Wq = (Lx + 7) / 8;
  const int align_elems = 32 / g.es;  // 32-byte rows
  g.W = ((4 * g.Wq + align_elems - 1) / align_elems) * align_elems;
  if ((uint64_t)Lz * (uint64_t)Ly * (uint64_t)g.Wq > 0xffffffffull) return COULPS_EINVAL;
  g.colour_elems = (size_t)Lz * Ly * g.W;
  g.chain_elems = 2 * g.colour_elems;
  if (g.W > 256) return COULPS_EUNSUPPORTED;

  coulps_lattice *L = new (std::nothrow) coulps_lattice();
  if (!L) return COULPS_ENOMEM;
  L->g = g;
  const int sms = device_sms();
  L->tile = fill_grid(g, default_tile(g), 2 * sms, 4);
  L->seed = seed;
  L->stream = (cudaStream_t)stream;
  L->alloc = g_allocator;
  const size_t fbytes = g.chain_elems * g.es * (size_t)n_chains;
  L->field = dev_alloc(L->alloc, fbytes, L->stream);
  L->d_pass = (uint32_t *)dev_alloc(L->alloc, 64, L->stream);
  L->d_err = (int *)dev_alloc(L->alloc, 64, L->stream);
  if (!L->field || !L->d_pass || !L->d_err) {
    coulps_lattice_destroy(L);
    return COULPS_ENOMEM;
  }
  L->bytes = fbytes + 128;
  if (cudaMemsetAsync(L->field, 0, fbytes, L->stream) != cudaSuccess ||
      cudaMemsetAsync(L->d_pass, 0, 64, L->stream) != cudaSuccess ||
      cudaMemsetAsync(L->d_err, 0, 64, L->stream) != cudaSuccess) {
    cudaGetLastError();
    coulps_lattice_destroy(L);
    return COULPS_ECUDA;
  }
  int st = rebuild_maps(L);
  if (!st) st = coulps_set_fused(L, 3);
  if (st) {
    coulps_lattice_destroy(L);
    return st;
  }
  *out = L;
  return COULPS_OK;
}

int coulps_set_fused(coulps_lattice_t L, int enable) {
  if (!L || enable < 0 || enable > 4) return COULPS_EINVAL;
  const size_t fbytes = L->g.chain_elems * L->g.es * (size_t)L->g.n_chains;
  drop_graph(L);
  if (!enable) {
    if (L->field2) {
      dev_free(L->alloc, L->field2, L->stream);
      L->field2 = nullptr;
      L->bytes -= fbytes;
    }
    L->fused = 0;
    return COULPS_OK;
  }
  if (!L->field2) {
    L->field2 = dev_alloc(L->alloc, fbytes, L->stream);
    if (!L->field2) return COULPS_ENOMEM;
    L->bytes += fbytes;
    // row padding and never-written quads stay 0 in both copies
    CK(cudaMemsetAsync(L->field2, 0, fbytes, L->stream));
  }
  if (L->ptile.ty == 0) L->ptile = fill_grid(L->g, default_pass_tile(L->g), 2 * device_sms(), 4);
  if (enable >= 3 && L->qtile.ty == 0)
    L->qtile = fill_grid(L->g, default_pair_tile(L->g), device_sms(), 8);
  L->fused = enable;
  int st = rebuild_maps(L);
  if (st) return st;
  return rebuild_pass_maps(L);
}

int coulps_set_pair_tile(coulps_lattice_t L, int ty, int dz) {
  if (!L || ty < 1 || dz < 0 || ty + 8 > 256) return COULPS_EINVAL;
  Tile t{ty, dz > 0 ? dz : (L->qtile.dz > 0 ? L->qtile.dz : L->g.Lz)};
  const int max_threads = L->g.precision == COULPS_F32 ? kPairMaxThreads32 : kPairMaxThreads64;
  if (pair_threads(L->g, t) > max_threads) return COULPS_EINVAL;
  if (pair_smem_bytes(L->g, t, true) > 227 * 1024) return COULPS_EINVAL;
  drop_graph(L);
  L->qtile = t;
  return rebuild_pass_maps(L);
}

int coulps_pair_tile(coulps_lattice_t L, int32_t out[2]) {
  if (!L || !out) return COULPS_EINVAL;
  out[0] = L->qtile.ty;
  out[1] = L->qtile.dz;
  return COULPS_OK;
}

int coulps_set_pass_tile(coulps_lattice_t L, int ty, int dz) {
  if (!L || ty < 1 || dz < 0 || ty + 4 > 256) return COULPS_EINVAL;
  Tile t{ty, dz > 0 ? dz : L->ptile.dz};
  if (t.dz < 1) t.dz = L->g.Lz;
  if (pass_threads(L->g, t) > 512) return COULPS_EINVAL;
  if (pass_smem_bytes(L->g, t, true) > 227 * 1024) return COULPS_EINVAL;
  drop_graph(L);
  L->ptile = t;
  return rebuild_pass_maps(L);
}

void coulps_lattice_destroy(coulps_lattice_t L) {
  if (!L) return;
  drop_graph(L);
  for (auto &t : L->pending) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  for (auto e : L->spare_events) cudaEventDestroy(e);
  for (int j = 0; j < 3; ++j) {
    if (L->xstream[j]) {
      cudaStreamSynchronize(L->xstream[j]);
      cudaStreamDestroy(L->xstream[j]);
    }
    if (L->ev_join[j]) cudaEventDestroy(L->ev_join[j]);
  }
  if (L->ev_fork) cudaEventDestroy(L->ev_fork);
  dev_free(L->alloc, L->field, L->stream);
  dev_free(L->alloc, L->field2, L->stream);
  dev_free(L->alloc, L->d_pass, L->stream);
  dev_free(L->alloc, L->d_err, L->stream);
  delete L;
}

int coulps_set_stream(coulps_lattice_t L, void *stream) {
  if (!L) return COULPS_EINVAL;
  if ((cudaStream_t)stream != L->stream) drop_graph(L);
  L->stream = (cudaStream_t)stream;
  return COULPS_OK;
}

int coulps_lattice_info(coulps_lattice_t L, int64_t info[13]) {
  if (!L || !info) return COULPS_EINVAL;
  info[0] = L->g.Lx; info[1] = L->g.Ly; info[2] = L->g.Lz;
  info[3] = L->g.n_chains; info[4] = L->g.precision; info[5] = L->g.W;
  info[6] = (int64_t)L->pass; info[7] = (int64_t)L->bytes;
  info[8] = L->tile.ty; info[9] = L->tile.dz;
  info[10] = L->fused; info[11] = L->ptile.ty; info[12] = L->ptile.dz;
  return COULPS_OK;
}

int coulps_set_tile(coulps_lattice_t L, int ty, int dz) {
  if (!L) return COULPS_EINVAL;
  Tile t = L->tile;
  if (ty > 0) t.ty = ty;
  if (dz > 0) t.dz = dz;
  if (ty < 0 || dz < 0 || t.ty < 1 || t.dz < 1 || t.ty + 2 > 256) return COULPS_EINVAL;
  if ((L->g.W / 4) * t.ty > 256) return COULPS_EINVAL;
  if (halfsweep_smem_bytes(L->g, t, true) > 227 * 1024) return COULPS_EINVAL;
  L->tile = t;
  drop_graph(L);
  return rebuild_maps(L);
}

int coulps_sync(coulps_lattice_t L) {
  if (!L) return COULPS_EINVAL;
  return check_device_error(L);
}

int coulps_selftest_wait(coulps_lattice_t L, int64_t limit_ns) {
  if (!L || limit_ns < 1000 || limit_ns > 1000000000) return COULPS_EINVAL;
  selftest_wait_kernel<<<1, 32, 0, L->stream>>>(L->d_err, (uint64_t)limit_ns);
  CK(cudaGetLastError());
  return COULPS_OK;
}

int coulps_clear_error(coulps_lattice_t L) {
  if (!L) return COULPS_EINVAL;
  CK(cudaMemsetAsync(L->d_err, 0, sizeof(int), L->stream));
  CK(cudaStreamSynchronize(L->stream));
  return COULPS_OK;
}

int coulps_field_get(coulps_lattice_t L, int chain, double *host) {
  if (!L || !host || chain < 0 || chain >= L->g.n_chains) return COULPS_EINVAL;
  const Geometry &g = L->g;
  std::vector<unsigned char> buf(g.chain_elems * g.es);
  CK(cudaMemcpyAsync(buf.data(), (const char *)L->field + (size_t)chain * g.chain_elems * g.es,
                     buf.size(), cudaMemcpyDeviceToHost, L->stream));
  int st = check_device_error(L);
  if (st) return st;
  for (int z = 0; z < g.Lz; ++z)
    for (int y = 0; y < g.Ly; ++y)
      for (int x = 0; x < g.Lx; ++x) {
        const int c = (x + y + z) & 1;
        const size_t s = (size_t)c * g.colour_elems + ((size_t)z * g.Ly + y) * g.W + (x >> 1);
        double v;
        if (g.precision == COULPS_F32)
          v = reinterpret_cast<const float *>(buf.data())[s];
        else
          v = reinterpret_cast<const double *>(buf.data())[s];
        host[x + (size_t)g.Lx * (y + (size_t)g.Ly * z)] = v;
      }
  return COULPS_OK;
}

int coulps_field_set(coulps_lattice_t L, int chain, const double *host) {
  if (!L || !host || chain < 0 || chain >= L->g.n_chains) return COULPS_EINVAL;
  const Geometry &g = L->g;
  std::vector<unsigned char> buf(g.chain_elems * g.es, 0);
  for (int z = 0; z < g.Lz; ++z)
    for (int y = 0; y < g.Ly; ++y)
      for (int x = 0; x < g.Lx; ++x) {
        const int c = (x + y + z) & 1;
        const size_t s = (size_t)c * g.colour_elems + ((size_t)z * g.Ly + y) * g.W + (x >> 1);
        const double v = host[x + (size_t)g.Lx * (y + (size_t)g.Ly * z)];
        if (g.precision == COULPS_F32)
          reinterpret_cast<float *>(buf.data())[s] = (float)v;
        else
          reinterpret_cast<double *>(buf.data())[s] = v;
      }
  CK(cudaMemcpyAsync((char *)L->field + (size_t)chain * g.chain_elems * g.es, buf.data(),
                     buf.size(), cudaMemcpyHostToDevice, L->stream));
  CK(cudaStreamSynchronize(L->stream));
  return COULPS_OK;
}

int coulps_sweep(coulps_lattice_t L, int n_compound, int n_hb, int n_or) {
  if (!L || n_compound < 0 || n_hb < 0 || n_or < 0) return COULPS_EINVAL;
  for (int k = 0; k < n_compound; ++k) {
    int st = enqueue_compound(L, n_hb, n_or);
    if (st) return st;
    L->pass += (uint64_t)(n_hb + n_or);
  }
  return COULPS_OK;
}

int coulps_charges_create(coulps_lattice_t L, int64_t n, const int32_t *site, const double *q,
                          int64_t log_capacity, coulps_charges_t *out) {
  if (!L || !out || n < 0 || log_capacity < 0) return COULPS_EINVAL;
  *out = nullptr;
  if (n > 0 && (!site || !q)) return COULPS_EINVAL;
  if (n > (int64_t)1 << 31) return COULPS_EINVAL;
  const Geometry &g = L->g;
  // charge sites are kept as 32-bit offsets within one chain's field
  if (g.chain_elems > 0xffffffffull) return COULPS_EUNSUPPORTED;
  std::vector<uint32_t> idx((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    const int x = site[3 * i], y = site[3 * i + 1], z = site[3 * i + 2];
    if (x < 0 || x >= g.Lx || y < 0 || y >= g.Ly || z < 0 || z >= g.Lz) return COULPS_EINVAL;
    if (!std::isfinite(q[i])) return COULPS_EINVAL;
    const int c = (x + y + z) & 1;
    idx[i] = (uint32_t)((size_t)c * g.colour_elems + ((size_t)z * g.Ly + y) * g.W + (x >> 1));
  }
  coulps_charges *C = new (std::nothrow) coulps_charges();
  if (!C) return COULPS_ENOMEM;
  C->lat = L;
  C->n = n;
  try {
    C->sites.assign(site, site + 3 * n);
    C->qv.assign(q, q + n);
  } catch (...) {
    delete C;
    return COULPS_ENOMEM;
  }
  C->nblk = gather_blocks(n);
  C->log_cap = log_capacity;
  const size_t b_idx = sizeof(uint32_t) * (size_t)n, b_q = sizeof(double) * (size_t)n;
  const size_t b_part = sizeof(double) * 2 * (size_t)C->nblk * g.n_chains;
  const size_t b_stats = sizeof(double) * kStatStride * (size_t)g.n_chains;
  const size_t b_log = sizeof(double) * 3 * (size_t)log_capacity * g.n_chains;
  C->d_idx = (uint32_t *)dev_alloc(L->alloc, b_idx, L->stream);
  C->d_q = (double *)dev_alloc(L->alloc, b_q, L->stream);
  C->d_partials = (double *)dev_alloc(L->alloc, b_part, L->stream);
  C->d_stats = (double *)dev_alloc(L->alloc, b_stats, L->stream);
  C->d_cvstats = (double *)dev_alloc(L->alloc, b_stats, L->stream);
  if (log_capacity > 0) C->d_log = (double *)dev_alloc(L->alloc, b_log, L->stream);
  C->bytes = b_idx + b_q + b_part + 2 * b_stats + b_log;
  if (!C->d_idx || !C->d_q || !C->d_partials || !C->d_stats || !C->d_cvstats ||
      (log_capacity > 0 && !C->d_log)) {
    coulps_charges_destroy(C);
    return COULPS_ENOMEM;
  }
  L->n_charge_sets++;
  if (n > 0) {
    if (cudaMemcpyAsync(C->d_idx, idx.data(), b_idx, cudaMemcpyHostToDevice, L->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(C->d_q, q, b_q, cudaMemcpyHostToDevice, L->stream) != cudaSuccess) {
      cudaGetLastError();
      coulps_charges_destroy(C);
      return COULPS_ECUDA;
    }
  }
  if (launch_reset_stats(C->d_stats, g.n_chains, L->stream) != cudaSuccess ||
      launch_reset_stats(C->d_cvstats, g.n_chains, L->stream) != cudaSuccess) {
    cudaGetLastError();
    coulps_charges_destroy(C);
    return COULPS_ECUDA;
  }
  // host vectors are copied from pageable memory: make sure the copy is done
  if (cudaStreamSynchronize(L->stream) != cudaSuccess) {
    cudaGetLastError();
    coulps_charges_destroy(C);
    return COULPS_ECUDA;
  }
  *out = C;
  return COULPS_OK;
}

void coulps_charges_destroy(coulps_charges_t C) {
  if (!C) return;
  coulps_lattice *L = C->lat;
  if (L->graph_key == C ||
      std::find(L->mgraph_key.begin(), L->mgraph_key.end(), (const void *)C) != L->mgraph_key.end())
    drop_graph(L);
  dev_free(L->alloc, C->d_idx, L->stream);
  dev_free(L->alloc, C->d_q, L->stream);
  dev_free(L->alloc, C->d_partials, L->stream);
  dev_free(L->alloc, C->d_stats, L->stream);
  dev_free(L->alloc, C->d_cvstats, L->stream);
  dev_free(L->alloc, C->d_log, L->stream);
  for (void *p : {(void *)C->d_oidx, (void *)C->d_ow, (void *)C->d_og, (void *)C->d_lastQ,
                  (void *)C->d_fsum, (void *)C->d_nptr, (void *)C->d_nbr, (void *)C->d_t,
                  (void *)C->d_u})
    dev_free(L->alloc, p, L->stream);
  if (C->staged) {
    cudaEventSynchronize(C->staged);
    cudaEventDestroy(C->staged);
  }
  for (int k = 0; k < 2; ++k)
    if (C->ev_post[k]) {
      cudaEventSynchronize(C->ev_post[k]);
      cudaEventDestroy(C->ev_post[k]);
    }
  if (C->h_post) cudaFreeHost(C->h_post);
  if (C->h_post_err) cudaFreeHost(C->h_post_err);
  if (C->h_idx) cudaFreeHost(C->h_idx);
  if (C->h_q) cudaFreeHost(C->h_q);
  if (C->gstaged) {
    cudaEventSynchronize(C->gstaged);
    cudaEventDestroy(C->gstaged);
  }
  if (C->h_goff) cudaFreeHost(C->h_goff);
  if (C->h_gent) cudaFreeHost(C->h_gent);
  if (C->h_gq) cudaFreeHost(C->h_gq);
  dev_free(L->alloc, C->d_goff, L->stream);
  dev_free(L->alloc, C->d_gent, L->stream);
  dev_free(L->alloc, C->d_gq, L->stream);
  dev_free(L->alloc, C->d_fpart, L->stream);
  L->n_charge_sets--;
  delete C;
}

int coulps_measure(coulps_lattice_t L, coulps_charges_t C) {
  if (!L || !C || C->lat != L) return COULPS_EINVAL;
  return enqueue_measure(L, C);
}

int coulps_run(coulps_lattice_t L, coulps_charges_t C, int n_therm, int n_meas, int n_hb,
               int n_or) {
  if (!L || !C || C->lat != L || n_therm < 0 || n_meas < 0 || n_hb < 0 || n_or < 0)
    return COULPS_EINVAL;
  int st = coulps_sweep(L, n_therm, n_hb, n_or);
  if (st) return st;
  if (n_meas == 0) return COULPS_OK;
  // The measured sweeps gather Q, P inside their last kernel (on-lattice
  // sets; off-lattice ones use their own gather after the sweep).
  const bool fused = n_hb + n_or > 0 && !C->off;
  const int P = n_hb + n_or;
  const bool phased = L->schedule == COULPS_SCHEDULE_PHASED && !C->off && n_hb > 0 && n_or > 0 &&
                      P <= kMaxGroups && n_meas >= 2 && L->g.n_chains >= P;
  if (fused) {
    st = stage_gather(L, C, phased ? L->tile : fused_gather_tile(L, n_hb, n_or));
    if (st) return st;
  }
  if (phased) {
    st = run_staggered(L, C, n_meas, n_hb, n_or);
    if (!st) L->pass += (uint64_t)n_meas * P;
    return st;
  }
  if (fused && n_meas >= 2 && shifted_ok(L, n_hb, n_or)) {
    st = run_shifted(L, C, n_meas, n_hb, n_or);
    if (!st) L->pass += (uint64_t)n_meas * P;
    return st;
  }
  const bool capturable = L->stream != nullptr && !L->profiling;
  if (capturable && (L->graph_key != C || L->graph_hb != n_hb || L->graph_or != n_or ||
                     L->graph_tile.ty != L->tile.ty || L->graph_tile.dz != L->tile.dz)) {
    drop_graph(L);
    cudaGraph_t gr = nullptr;
    CK(cudaStreamBeginCapture(L->stream, cudaStreamCaptureModeThreadLocal));
    int s1 = enqueue_compound(L, n_hb, n_or, fused ? C : nullptr);
    int s2 = s1 ? s1 : (fused ? COULPS_OK : enqueue_measure(L, C));
    cudaError_t e = cudaStreamEndCapture(L->stream, &gr);
    if (s2 || e != cudaSuccess) {
      cudaGetLastError();
      if (gr) cudaGraphDestroy(gr);
      return s2 ? s2 : COULPS_ECUDA;
    }
    e = cudaGraphInstantiate(&L->graph, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
      cudaGetLastError();
      L->graph = nullptr;
      return COULPS_ECUDA;
    }
    L->graph_key = C;
    L->graph_hb = n_hb;
    L->graph_or = n_or;
    L->graph_tile = L->tile;
  }
  for (int k = 0; k < n_meas; ++k) {
    if (capturable) {
      CK(cudaGraphLaunch(L->graph, L->stream));
    } else {
      st = enqueue_compound(L, n_hb, n_or, fused ? C : nullptr);
      if (!st && !fused) st = enqueue_measure(L, C);
      if (st) return st;
    }
    L->pass += (uint64_t)(n_hb + n_or);
  }
  return COULPS_OK;
}

static int check_sets(coulps_lattice *L, const coulps_charges_t *sets, int n_sets) {
  if (!L || !sets || n_sets < 1) return COULPS_EINVAL;
  for (int k = 0; k < n_sets; ++k)
    if (!sets[k] || sets[k]->lat != L) return COULPS_EINVAL;
  return COULPS_OK;
}

int coulps_measure_sets(coulps_lattice_t L, const coulps_charges_t *sets, int n_sets) {
  int st = check_sets(L, sets, n_sets);
  if (st) return st;
  return enqueue_measure_sets(L, sets, n_sets);
}

int coulps_run_sets(coulps_lattice_t L, const coulps_charges_t *sets, int n_sets, int n_therm,
                    int n_meas, int n_hb, int n_or) {
  int st = check_sets(L, sets, n_sets);
  if (st) return st;
  if (n_therm < 0 || n_meas < 0 || n_hb < 0 || n_or < 0) return COULPS_EINVAL;
  st = coulps_sweep(L, n_therm, n_hb, n_or);
  if (st || n_meas == 0) return st;
  // one measured compound sweep + the multi-set gather as a graph, kept for
  // later calls with the same sets and mix (tile changes drop it)
  std::vector<const void *> key(sets, sets + n_sets);
  const bool capturable = L->stream != nullptr && !L->profiling && n_meas >= 4;
  if (capturable && (!L->mgraph || L->mgraph_key != key || L->mgraph_hb != n_hb ||
                     L->mgraph_or != n_or)) {
    drop_graph(L);
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t gr = nullptr;
    CK(cudaStreamBeginCapture(L->stream, cudaStreamCaptureModeThreadLocal));
    int s1 = enqueue_compound(L, n_hb, n_or, nullptr);
    int s2 = s1 ? s1 : enqueue_measure_sets(L, sets, n_sets);
    cudaError_t e = cudaStreamEndCapture(L->stream, &gr);
    if (s2 || e != cudaSuccess) {
      cudaGetLastError();
      if (gr) cudaGraphDestroy(gr);
      return s2 ? s2 : COULPS_ECUDA;
    }
    e = cudaGraphInstantiate(&exec, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return COULPS_ECUDA;
    }
    L->mgraph = exec;
    L->mgraph_key = key;
    L->mgraph_hb = n_hb;
    L->mgraph_or = n_or;
  }
  for (int k = 0; k < n_meas && !st; ++k) {
    if (capturable) {
      if (cudaGraphLaunch(L->mgraph, L->stream) != cudaSuccess) {
        cudaGetLastError();
        st = COULPS_ECUDA;
      }
    } else {
      st = enqueue_compound(L, n_hb, n_or, nullptr);
      if (!st) st = enqueue_measure_sets(L, sets, n_sets);
    }
    if (!st) L->pass += (uint64_t)(n_hb + n_or);
  }
  return st;
}

int coulps_pool_stats(const double *st, int64_t n_rows, double *mean, double *stderr_bm,
                      double *tau_int, int64_t *n) {
  if (n_rows < 0 || (n_rows > 0 && !st)) return COULPS_EINVAL;
  // Pool over rows (chains) in order.  Batches of all rows share one length.
  double N = 0, S = 0, S2 = 0;
  double nb_tot = 0, bsum = 0, bsum2 = 0, blen = 0;
  for (int64_t k = 0; k < n_rows; ++k) {
    const double *p = st + (size_t)k * kStatStride;
    N += p[kStatN];
    S += p[kStatSum];
    S2 += p[kStatSum2];
    if (k > 0 && p[kStatBatchLen] != blen) return COULPS_EINVAL;
    blen = p[kStatBatchLen];
    const int nb = (int)p[kStatNBatch];
    if (nb < 0 || nb >= 2 * kBatchMin) return COULPS_EINVAL;
    for (int b = 0; b < nb; ++b) {
      const double m = p[kStatBatch0 + b] / blen;
      bsum += m;
      bsum2 += m * m;
      nb_tot += 1;
    }
  }
  const double mu = N > 0 ? S / N : NAN;
  double se = NAN, tau = NAN;
  if (nb_tot >= 2) {
    const double bm = bsum / nb_tot;
    const double bvar = (bsum2 - nb_tot * bm * bm) / (nb_tot - 1);
    se = std::sqrt(bvar > 0 ? bvar / nb_tot : 0.0);
    const double var = N > 1 ? (S2 - N * mu * mu) / (N - 1) : NAN;
    if (var > 0) tau = 0.5 * blen * bvar / var;
  }
  if (mean) *mean = mu;
  if (stderr_bm) *stderr_bm = se;
  if (tau_int) *tau_int = tau;
  if (n) *n = (int64_t)N;
  if (N > 0 && !std::isfinite(mu)) return COULPS_ENONFINITE;
  return COULPS_OK;
}

int coulps_chain_stats(coulps_charges_t C, double *out, int64_t cap) {
  if (!C || !out) return COULPS_EINVAL;
  coulps_lattice *L = C->lat;
  const int64_t need = (int64_t)L->g.n_chains * kStatStride;
  if (cap < need) return COULPS_EINVAL;
  CK(cudaMemcpyAsync(out, C->d_stats, need * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
  return check_device_error(L);
}

int coulps_estimate(coulps_charges_t C, double *mean, double *stderr_bm, double *tau_int,
                    int64_t *n) {
  if (!C) return COULPS_EINVAL;
  coulps_lattice *L = C->lat;
  std::vector<double> st((size_t)L->g.n_chains * kStatStride);
  int s = coulps_chain_stats(C, st.data(), (int64_t)st.size());
  if (s) return s;
  return coulps_pool_stats(st.data(), L->g.n_chains, mean, stderr_bm, tau_int, n);
}

int coulps_estimate_post(coulps_charges_t C) {
  if (!C) return COULPS_EINVAL;
  coulps_lattice *L = C->lat;
  const size_t need = (size_t)L->g.n_chains * kStatStride;
  if (C->posted - C->taken >= 2) return COULPS_EINVAL;  // both slots hold untaken states
  if (!C->h_post) {
    // all four or none: a failure leaves the set as it was
    double *hp = nullptr;
    int *he = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (cudaMallocHost((void **)&hp, 2 * need * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void **)&he, 2 * sizeof(int)) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      if (hp) cudaFreeHost(hp);
      if (he) cudaFreeHost(he);
      for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
      return COULPS_ENOMEM;
    }
    C->h_post = hp;
    C->h_post_err = he;
    C->ev_post[0] = ev[0];
    C->ev_post[1] = ev[1];
  }
  const int slot = (int)(C->posted & 1);
  CK(cudaMemcpyAsync(C->h_post + slot * need, C->d_stats, need * sizeof(double),
                     cudaMemcpyDeviceToHost, L->stream));
  CK(cudaMemcpyAsync(C->h_post_err + slot, L->d_err, sizeof(int), cudaMemcpyDeviceToHost,
                     L->stream));
  CK(cudaEventRecord(C->ev_post[slot], L->stream));
  ++C->posted;
  return COULPS_OK;
}

int coulps_estimate_take(coulps_charges_t C, double *mean, double *stderr_bm, double *tau_int,
                         int64_t *n) {
  if (!C) return COULPS_EINVAL;
  if (C->taken == C->posted) return COULPS_EINVAL;  // nothing posted
  coulps_lattice *L = C->lat;
  const size_t need = (size_t)L->g.n_chains * kStatStride;
  const int slot = (int)(C->taken & 1);
  CK(cudaEventSynchronize(C->ev_post[slot]));
  ++C->taken;
  const int e = C->h_post_err[slot];
  if (e & kErrTimeout) return COULPS_ETIMEOUT;
  if (e & kErrNonFinite) return COULPS_ENONFINITE;
  return coulps_pool_stats(C->h_post + slot * need, L->g.n_chains, mean, stderr_bm, tau_int, n);
}

int coulps_samples(coulps_charges_t C, double *QPe, int64_t cap, int64_t *n) {
  if (!C || (cap > 0 && !QPe) || cap < 0) return COULPS_EINVAL;
  coulps_lattice *L = C->lat;
  const int nc = L->g.n_chains;
  double ns = 0;
  CK(cudaMemcpyAsync(&ns, C->d_stats + kStatN, sizeof(double), cudaMemcpyDeviceToHost,
                     L->stream));
  int s = check_device_error(L);
  if (s) return s;
  int64_t m = (int64_t)ns;
  if (m > C->log_cap) m = C->log_cap;
  if (m > cap) m = cap;
  if (m > 0) {
    CK(cudaMemcpyAsync(QPe, C->d_log, sizeof(double) * 3 * (size_t)m * nc,
                       cudaMemcpyDeviceToHost, L->stream));
    CK(cudaStreamSynchronize(L->stream));
  }
  if (n) *n = m;
  return COULPS_OK;
}

int coulps_reset_stats(coulps_charges_t C) {
  if (!C) return COULPS_EINVAL;
  CK(launch_reset_stats(C->d_stats, C->lat->g.n_chains, C->lat->stream));
  if (C->d_fsum)
    CK(cudaMemsetAsync(C->d_fsum, 0, sizeof(double) * 3 * (size_t)C->n * C->lat->g.n_chains,
                       C->lat->stream));
  return COULPS_OK;
}

int coulps_charges_create_off(coulps_lattice_t L, int64_t n, const double *pos, const double *q,
                              int64_t log_capacity, int forces, coulps_charges_t *out) {
  if (!L || !out || n < 0 || log_capacity < 0) return COULPS_EINVAL;
  *out = nullptr;
  if (n > 0 && (!pos || !q)) return COULPS_EINVAL;
  if (n > ((int64_t)1 << 28)) return COULPS_EINVAL;
  const Geometry &g = L->g;
  if (g.Lx < 2 || g.Ly < 2 || g.Lz < 2) return COULPS_EINVAL;
  if (g.chain_elems > 0xffffffffull) return COULPS_EUNSUPPORTED;  // 32-bit corner offsets
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(q[i])) return COULPS_EINVAL;
  // corners, trilinear weights and their gradients, in FP64 on the host
  std::vector<uint32_t> oidx((size_t)8 * n);
  std::vector<double> ow((size_t)8 * n), og((size_t)24 * n);
  if (!offlattice_corners(g.Lx, g.Ly, g.Lz, g.W, g.colour_elems, n, pos, oidx.data(), ow.data(),
                          og.data()))
    return COULPS_EINVAL;
  // the common parts of a charge set (statistics, log) with no lattice charges
  coulps_charges_t C = nullptr;
  int st = coulps_charges_create(L, 0, nullptr, nullptr, log_capacity, &C);
  if (st) return st;
  C->off = true;
  C->n = n;
  C->nblk = C->nblk_g = gather_blocks(n);
  C->pos.assign(pos, pos + 3 * n);
  dev_free(L->alloc, C->d_partials, L->stream);
  dev_free(L->alloc, C->d_q, L->stream);
  const size_t nc = (size_t)g.n_chains;
  C->d_partials = (double *)dev_alloc(L->alloc, sizeof(double) * 2 * (size_t)C->nblk * nc, L->stream);
  C->d_q = (double *)dev_alloc(L->alloc, sizeof(double) * (size_t)(n > 0 ? n : 1), L->stream);
  C->d_oidx = (uint32_t *)dev_alloc(L->alloc, sizeof(uint32_t) * 8 * (size_t)(n > 0 ? n : 1), L->stream);
  C->d_ow = (double *)dev_alloc(L->alloc, sizeof(double) * 8 * (size_t)(n > 0 ? n : 1), L->stream);
  C->d_og = (double *)dev_alloc(L->alloc, sizeof(double) * 24 * (size_t)(n > 0 ? n : 1), L->stream);
  C->d_lastQ = (double *)dev_alloc(L->alloc, sizeof(double) * nc, L->stream);
  if (forces && n > 0)
    C->d_fsum = (double *)dev_alloc(L->alloc, sizeof(double) * 3 * (size_t)n * nc, L->stream);
  if (!C->d_partials || !C->d_q || !C->d_oidx || !C->d_ow || !C->d_og || !C->d_lastQ ||
      (forces && n > 0 && !C->d_fsum)) {
    coulps_charges_destroy(C);
    return COULPS_ENOMEM;
  }
  C->qv.assign(q, q + n);
  C->bytes += (size_t)n * (sizeof(double) + 8 * (sizeof(uint32_t) + 4 * sizeof(double))) +
              sizeof(double) * nc * (1 + (C->d_fsum ? 3 * (size_t)n : 0));
  if (n > 0 &&
      (cudaMemcpyAsync(C->d_q, q, sizeof(double) * n, cudaMemcpyHostToDevice, L->stream) !=
           cudaSuccess ||
       cudaMemcpyAsync(C->d_oidx, oidx.data(), sizeof(uint32_t) * oidx.size(),
                       cudaMemcpyHostToDevice, L->stream) != cudaSuccess ||
       cudaMemcpyAsync(C->d_ow, ow.data(), sizeof(double) * ow.size(), cudaMemcpyHostToDevice,
                       L->stream) != cudaSuccess ||
       cudaMemcpyAsync(C->d_og, og.data(), sizeof(double) * og.size(), cudaMemcpyHostToDevice,
                       L->stream) != cudaSuccess ||
       (C->d_fsum && cudaMemsetAsync(C->d_fsum, 0, sizeof(double) * 3 * (size_t)n * nc,
                                     L->stream) != cudaSuccess) ||
       cudaStreamSynchronize(L->stream) != cudaSuccess)) {  // pageable host arrays
    cudaGetLastError();
    coulps_charges_destroy(C);
    return COULPS_ECUDA;
  }
  *out = C;
  return COULPS_OK;
}

int coulps_charges_near(coulps_charges_t C, double rc, int64_t *n_pairs, double *e_direct,
                        double *f_direct) {
  if (!C || !std::isfinite(rc) || rc < 0.0) return COULPS_EINVAL;
  if (!C->off) return COULPS_EUNSUPPORTED;
  coulps_lattice *L = C->lat;
  const int64_t n = C->n;
  const double *p = C->pos.data();
  std::vector<int64_t> ptr;
  std::vector<uint32_t> nbr;
  near_csr(p, n, rc, ptr, nbr);
  const int64_t pairs = (int64_t)nbr.size() / 2;
  // the direct part with the continuum kernel of Eq. (s1), in FP64
  double E = 0.0;
  if (f_direct)
    for (int64_t k = 0; k < 3 * n; ++k) f_direct[k] = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) {
      const int64_t j = nbr[k];
      const double d[3] = {p[3 * i] - p[3 * j], p[3 * i + 1] - p[3 * j + 1],
                           p[3 * i + 2] - p[3 * j + 2]};
      const double r = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      const double qq = C->qv[i] * C->qv[j];
      if (j > i) E += 2.0 * qq / r;
      if (f_direct)
        for (int mu = 0; mu < 3; ++mu) f_direct[3 * i + mu] += 2.0 * qq * d[mu] / (r * r * r);
    }
  const double inv4pi = 1.0 / (4.0 * M_PI);
  E *= inv4pi;
  if (f_direct)
    for (int64_t k = 0; k < 3 * n; ++k) f_direct[k] *= inv4pi;
  if (n_pairs) *n_pairs = pairs;
  if (e_direct) *e_direct = E;
  // device side: the graphs that measure this set are rebuilt, the samples
  // taken under the previous list are dropped
  if (L->graph_key == C ||
      std::find(L->mgraph_key.begin(), L->mgraph_key.end(), (const void *)C) != L->mgraph_key.end())
    drop_graph(L);
  CK(cudaStreamSynchronize(L->stream));
  const int nc = L->g.n_chains;
  const int row = C->nblk_g + (pairs > 0 ? near_blocks(n) : 0);
  // the new device buffers first: if one cannot be had, the set keeps its
  // previous near list and buffers unchanged
  double *part = nullptr, *t = nullptr, *u = nullptr;
  int64_t *dptr = nullptr;
  uint32_t *dnbr = nullptr;
  auto release = [&]() {
    for (void *q : {(void *)part, (void *)t, (void *)u, (void *)dptr, (void *)dnbr})
      dev_free(L->alloc, q, L->stream);
  };
  bool ok = true;
  if (row != C->nblk) {
    part = (double *)dev_alloc(L->alloc, sizeof(double) * 2 * (size_t)row * nc, L->stream);
    ok = part != nullptr;
  }
  if (ok && pairs > 0) {
    dptr = (int64_t *)dev_alloc(L->alloc, sizeof(int64_t) * ptr.size(), L->stream);
    dnbr = (uint32_t *)dev_alloc(L->alloc, sizeof(uint32_t) * nbr.size(), L->stream);
    t = (double *)dev_alloc(L->alloc, sizeof(double) * (size_t)n * nc, L->stream);
    u = (double *)dev_alloc(L->alloc, sizeof(double) * (size_t)n * nc, L->stream);
    ok = dptr && dnbr && t && u;
    if (ok && (cudaMemcpyAsync(dptr, ptr.data(), sizeof(int64_t) * ptr.size(),
                               cudaMemcpyHostToDevice, L->stream) != cudaSuccess ||
               cudaMemcpyAsync(dnbr, nbr.data(), sizeof(uint32_t) * nbr.size(),
                               cudaMemcpyHostToDevice, L->stream) != cudaSuccess)) {
      cudaGetLastError();
      release();
      return COULPS_ECUDA;
    }
  }
  if (!ok) {
    release();
    return COULPS_ENOMEM;
  }
  // swap in the new list
  for (void **q : {(void **)&C->d_nptr, (void **)&C->d_nbr, (void **)&C->d_t, (void **)&C->d_u}) {
    dev_free(L->alloc, *q, L->stream);
    *q = nullptr;
  }
  if (row != C->nblk) {
    dev_free(L->alloc, C->d_partials, L->stream);
    C->d_partials = part;
    C->nblk = row;
  }
  C->d_nptr = dptr;
  C->d_nbr = dnbr;
  C->d_t = t;
  C->d_u = u;
  C->n_pairs = pairs;
  int st = coulps_reset_stats(C);
  if (st) return st;
  CK(launch_reset_stats(C->d_cvstats, nc, L->stream));
  CK(cudaStreamSynchronize(L->stream));  // pageable host arrays
  return COULPS_OK;
}

int coulps_near_pairs(int64_t n, const double *pos, double rc, int64_t *ptr, uint32_t *nbr,
                      int64_t cap, int64_t *n_entries) {
  if (n < 0 || (n > 0 && (!pos || !ptr)) || !n_entries || !std::isfinite(rc) || rc < 0.0 ||
      cap < 0 || n > ((int64_t)1 << 31))
    return COULPS_EINVAL;
  for (int64_t k = 0; k < 3 * n; ++k)
    if (!std::isfinite(pos[k])) return COULPS_EINVAL;
  std::vector<int64_t> p;
  std::vector<uint32_t> b;
  try {
    near_csr(pos, n, rc, p, b);
  } catch (...) {
    return COULPS_ENOMEM;
  }
  *n_entries = (int64_t)b.size();
  if ((int64_t)b.size() > cap || (!b.empty() && !nbr)) return COULPS_EINVAL;
  std::copy(p.begin(), p.end(), ptr);
  std::copy(b.begin(), b.end(), nbr);
  return COULPS_OK;
}

int coulps_offlattice_corners(int Lx, int Ly, int Lz, int precision, int64_t n, const double *pos,
                              uint32_t *offset, double *weight, double *grad) {
  if (n < 0 || (n > 0 && (!pos || !offset || !weight || !grad))) return COULPS_EINVAL;
  if (precision != COULPS_F32 && precision != COULPS_F64) return COULPS_EINVAL;
  if (Lx < 2 || Ly < 2 || Lz < 2 || Lx > 512 || Ly > 65535 || Lz > 65535) return COULPS_EINVAL;
  // the row stride and colour size of a lattice of this shape and precision
  const int es = precision == COULPS_F32 ? 4 : 8;
  const int Wq = (Lx + 7) / 8, align_elems = 32 / es;
  const int W = ((4 * Wq + align_elems - 1) / align_elems) * align_elems;
  const size_t colour_elems = (size_t)Lz * Ly * W;
  return offlattice_corners(Lx, Ly, Lz, W, colour_elems, n, pos, offset, weight, grad)
             ? COULPS_OK
             : COULPS_EINVAL;
}

int coulps_forces(coulps_charges_t C, double *mean, double *stderr_chains) {
  if (!C || !mean) return COULPS_EINVAL;
  if (!C->off || !C->d_fsum) return COULPS_EUNSUPPORTED;
  coulps_lattice *L = C->lat;
  const int nc = L->g.n_chains;
  const size_t n = (size_t)C->n;
  std::vector<double> fs(3 * n * nc), st((size_t)kStatStride * nc);
  CK(cudaMemcpyAsync(fs.data(), C->d_fsum, sizeof(double) * fs.size(), cudaMemcpyDeviceToHost,
                     L->stream));
  CK(cudaMemcpyAsync(st.data(), C->d_stats, sizeof(double) * st.size(), cudaMemcpyDeviceToHost,
                     L->stream));
  int s = check_device_error(L);
  if (s) return s;
  double N = 0.0;
  for (int b = 0; b < nc; ++b) N += st[(size_t)b * kStatStride + kStatN];
  for (size_t k = 0; k < 3 * n; ++k) {
    double sum = 0.0;
    for (int b = 0; b < nc; ++b) sum += fs[(size_t)b * 3 * n + k];
    mean[k] = N > 0 ? sum / N : NAN;
    if (stderr_chains) {
      // spread of the chains' own means (independent chains)
      double m1 = 0.0, m2 = 0.0;
      int used = 0;
      for (int b = 0; b < nc; ++b) {
        const double nb = st[(size_t)b * kStatStride + kStatN];
        if (nb <= 0) continue;
        const double m = fs[(size_t)b * 3 * n + k] / nb;
        m1 += m;
        m2 += m * m;
        ++used;
      }
      if (used >= 2) {
        const double mu = m1 / used;
        const double var = (m2 - used * mu * mu) / (used - 1);
        stderr_chains[k] = std::sqrt(var > 0 ? var / used : 0.0);
      } else {
        stderr_chains[k] = NAN;
      }
    }
  }
  return COULPS_OK;
}

int coulps_cv_record(coulps_charges_t C, const double *tg, double c) {
  if (!C || !tg || !std::isfinite(c)) return COULPS_EINVAL;
  coulps_lattice *L = C->lat;
  CK(launch_cv_record(C->d_stats, tg, c, C->d_cvstats, L->g.n_chains, L->d_err, L->stream));
  return COULPS_OK;
}

int coulps_cv_chain_stats(coulps_charges_t C, double *out, int64_t cap) {
  if (!C || !out) return COULPS_EINVAL;
  coulps_lattice *L = C->lat;
  const int64_t need = (int64_t)L->g.n_chains * kStatStride;
  if (cap < need) return COULPS_EINVAL;
  CK(cudaMemcpyAsync(out, C->d_cvstats, need * sizeof(double), cudaMemcpyDeviceToHost,
                     L->stream));
  return check_device_error(L);
}

int coulps_cv_estimate(coulps_charges_t C, double *mean, double *stderr_bm, double *tau_int,
                       int64_t *n) {
  if (!C) return COULPS_EINVAL;
  coulps_lattice *L = C->lat;
  std::vector<double> st((size_t)L->g.n_chains * kStatStride);
  int s = coulps_cv_chain_stats(C, st.data(), (int64_t)st.size());
  if (s) return s;
  return coulps_pool_stats(st.data(), L->g.n_chains, mean, stderr_bm, tau_int, n);
}

int coulps_cv_reset(coulps_charges_t C) {
  if (!C) return COULPS_EINVAL;
  CK(launch_reset_stats(C->d_cvstats, C->lat->g.n_chains, C->lat->stream));
  return COULPS_OK;
}

// ---- global control variate (gcv.cu) ---------------------------------------
struct coulps_gcv {
  coulps_charges *ch = nullptr;
  double *d_rho = nullptr, *d_u = nullptr, *d_scratch = nullptr;
  double *d_c0res = nullptr, *d_partials = nullptr, *d_tg = nullptr;
  float *d_h32 = nullptr, *d_v = nullptr;
  int nblk_red = 64, nblk = 1;
  size_t bytes = 0;
  // local term of P: kernel of radius R, its centre value times sum q^2
  int R = 0;
  float *d_k = nullptr;
  double cP = 0.0;
  double *d_ppart = nullptr;
  // the local term runs on a side stream beside the v . phi sums
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

}  // extern "C"

// Dirichlet Green function of the (2R+1)^3 cube at its centre: A k = e_centre
// by Gaussian elimination (at most 729 unknowns), in FP64, rounded to FP32.
std::vector<float> coulps::cube_green(int R) {
  const int m = 2 * R + 1, n = m * m * m;
  std::vector<double> A((size_t)n * n, 0.0), b(n, 0.0);
  auto id = [&](int x, int y, int z) { return (z * m + y) * m + x; };
  for (int z = 0; z < m; ++z)
    for (int y = 0; y < m; ++y)
      for (int x = 0; x < m; ++x) {
        const int i = id(x, y, z);
        A[(size_t)i * n + i] = 6.0;
        const int nb[6][3] = {{x - 1, y, z}, {x + 1, y, z}, {x, y - 1, z},
                              {x, y + 1, z}, {x, y, z - 1}, {x, y, z + 1}};
        for (auto &p : nb)
          if (p[0] >= 0 && p[1] >= 0 && p[2] >= 0 && p[0] < m && p[1] < m && p[2] < m)
            A[(size_t)i * n + id(p[0], p[1], p[2])] = -1.0;
      }
  b[id(R, R, R)] = 1.0;
  for (int c = 0; c < n; ++c) {  // SPD: no pivoting needed
    const double d = A[(size_t)c * n + c];
    for (int r = c + 1; r < n; ++r) {
      const double f = A[(size_t)r * n + c] / d;
      if (f == 0.0) continue;
      for (int k = c; k < n; ++k) A[(size_t)r * n + k] -= f * A[(size_t)c * n + k];
      b[r] -= f * b[c];
    }
  }
  std::vector<double> x(n, 0.0);
  for (int r = n - 1; r >= 0; --r) {
    double s = b[r];
    for (int k = r + 1; k < n; ++k) s -= A[(size_t)r * n + k] * x[k];
    x[r] = s / A[(size_t)r * n + r];
  }
  std::vector<float> out(n);
  for (int i = 0; i < n; ++i) out[i] = (float)x[i];
  return out;
}

extern "C" {

void coulps_gcv_destroy(coulps_gcv_t G) {
  if (!G) return;
  coulps_lattice *L = G->ch->lat;
  if (L->stream) cudaStreamSynchronize(L->stream);
  if (G->side) cudaStreamSynchronize(G->side);
  if (G->ev_fork) cudaEventDestroy(G->ev_fork);
  if (G->ev_join) cudaEventDestroy(G->ev_join);
  if (G->side) cudaStreamDestroy(G->side);
  for (void *p : {(void *)G->d_rho, (void *)G->d_u, (void *)G->d_v, (void *)G->d_scratch,
                  (void *)G->d_c0res, (void *)G->d_partials, (void *)G->d_tg, (void *)G->d_h32,
                  (void *)G->d_k, (void *)G->d_ppart})
    dev_free(L->alloc, p, L->stream);
  delete G;
}

int coulps_gcv_create(coulps_charges_t C, int n_iter, int R, coulps_gcv_t *out) {
  if (!C || !out || n_iter < 0 || R < 0 || R > 4) return COULPS_EINVAL;
  if (C->off) return COULPS_EUNSUPPORTED;
  *out = nullptr;
  coulps_lattice *L = C->lat;
  const Geometry &g = L->g;
  coulps_gcv *G = new (std::nothrow) coulps_gcv();
  if (!G) return COULPS_ENOMEM;
  G->ch = C;
  G->nblk = gcv_blocks(g);
  if (cudaStreamCreateWithFlags(&G->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&G->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&G->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    coulps_gcv_destroy(G);
    return COULPS_ECUDA;
  }
  const size_t n = (size_t)g.Lx * g.Ly * g.Lz;
  G->d_rho = (double *)dev_alloc(L->alloc, n * sizeof(double), L->stream);
  G->d_u = (double *)dev_alloc(L->alloc, n * sizeof(double), L->stream);
  G->d_h32 = (float *)dev_alloc(L->alloc, n * sizeof(float), L->stream);
  G->d_v = (float *)dev_alloc(L->alloc, g.chain_elems * sizeof(float), L->stream);
  G->d_scratch = (double *)dev_alloc(L->alloc, 4 * G->nblk_red * sizeof(double), L->stream);
  G->d_c0res = (double *)dev_alloc(L->alloc, 4 * sizeof(double), L->stream);
  G->d_partials =
      (double *)dev_alloc(L->alloc, 2 * (size_t)G->nblk * g.n_chains * sizeof(double), L->stream);
  G->d_tg = (double *)dev_alloc(L->alloc, (size_t)g.n_chains * sizeof(double), L->stream);
  G->R = C->n > 0 ? R : 0;
  std::vector<float> kt;
  if (G->R > 0) {
    kt = cube_green(G->R);
    const int m = 2 * G->R + 1;
    double q2 = 0.0;
    for (double v : C->qv) q2 += v * v;
    G->cP = (double)kt[(G->R * m + G->R) * m + G->R] * q2;
    G->d_k = (float *)dev_alloc(L->alloc, kt.size() * sizeof(float), L->stream);
    G->d_ppart = (double *)dev_alloc(
        L->alloc, (size_t)((C->n + 7) / 8) * g.n_chains * sizeof(double), L->stream);
    if (!G->d_k || !G->d_ppart) {
      coulps_gcv_destroy(G);
      return COULPS_ENOMEM;
    }
  }
  G->bytes = n * (2 * sizeof(double) + sizeof(float)) + g.chain_elems * sizeof(float);
  if (!G->d_rho || !G->d_u || !G->d_h32 || !G->d_v || !G->d_scratch || !G->d_c0res ||
      !G->d_partials || !G->d_tg) {
    coulps_gcv_destroy(G);
    return COULPS_ENOMEM;
  }
  // the charge density from the set's host copy (natural order)
  std::vector<double> rho;
  try {
    rho.assign(n, 0.0);
  } catch (...) {
    coulps_gcv_destroy(G);
    return COULPS_ENOMEM;
  }
  for (size_t i = 0; i < C->qv.size(); ++i) {
    const int32_t *s = &C->sites[3 * i];
    rho[((size_t)s[2] * g.Ly + s[1]) * g.Lx + s[0]] += C->qv[i];
  }
  if (cudaMemcpyAsync(G->d_rho, rho.data(), n * sizeof(double), cudaMemcpyHostToDevice,
                      L->stream) != cudaSuccess ||
      (G->R > 0 && cudaMemcpyAsync(G->d_k, kt.data(), kt.size() * sizeof(float),
                                   cudaMemcpyHostToDevice, L->stream) != cudaSuccess) ||
      gcv_solve(g, G->d_rho, G->d_u, G->d_h32, G->d_v, G->d_scratch, G->nblk_red, n_iter,
                G->d_c0res, L->stream) != cudaSuccess ||
      cudaStreamSynchronize(L->stream) != cudaSuccess) {  // rho is pageable host memory
    cudaGetLastError();
    coulps_gcv_destroy(G);
    return COULPS_ECUDA;
  }
  *out = G;
  return COULPS_OK;
}

int coulps_gcv_info(coulps_gcv_t G, double out[2]) {
  if (!G || !out) return COULPS_EINVAL;
  coulps_lattice *L = G->ch->lat;
  CK(cudaMemcpyAsync(out, G->d_c0res, 2 * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
  CK(cudaStreamSynchronize(L->stream));
  return COULPS_OK;
}

int coulps_gcv_h(coulps_gcv_t G, float *host_xyz) {
  if (!G || !host_xyz) return COULPS_EINVAL;
  coulps_lattice *L = G->ch->lat;
  const size_t n = (size_t)L->g.Lx * L->g.Ly * L->g.Lz;
  CK(cudaMemcpyAsync(host_xyz, G->d_h32, n * sizeof(float), cudaMemcpyDeviceToHost, L->stream));
  CK(cudaStreamSynchronize(L->stream));
  return COULPS_OK;
}

int coulps_gcv_eval(coulps_gcv_t G, double *tg) {
  if (!G) return COULPS_EINVAL;
  coulps_charges *C = G->ch;
  coulps_lattice *L = C->lat;
  CK(gcv_eval(L->g, L->field, G->d_v, C->d_idx, C->d_q, C->n, G->d_partials, G->nblk,
              G->d_c0res, G->d_k, G->R, G->cP, G->d_ppart, tg ? tg : G->d_tg, L->stream,
              G->side, G->ev_fork, G->ev_join));
  return COULPS_OK;
}

int coulps_gcv_run(coulps_gcv_t G, int n_meas, int n_hb, int n_or, double c) {
  if (!G || n_meas < 0 || n_hb < 0 || n_or < 0 || !std::isfinite(c)) return COULPS_EINVAL;
  coulps_charges *C = G->ch;
  coulps_lattice *L = C->lat;
  if (n_meas == 0) return COULPS_OK;
  const bool fused = n_hb + n_or > 0;
  if (fused) {
    int st = stage_gather(L, C, fused_gather_tile(L, n_hb, n_or));
    if (st) return st;
  }
  auto one = [&]() -> int {
    int st = enqueue_compound(L, n_hb, n_or, fused ? C : nullptr);
    if (!st && !fused) st = enqueue_measure(L, C);
    if (st) return st;
    CK(gcv_eval(L->g, L->field, G->d_v, C->d_idx, C->d_q, C->n, G->d_partials, G->nblk,
                G->d_c0res, G->d_k, G->R, G->cP, G->d_ppart, G->d_tg, L->stream, G->side,
                G->ev_fork, G->ev_join));
    CK(launch_cv_record(C->d_stats, G->d_tg, c, C->d_cvstats, L->g.n_chains, L->d_err,
                        L->stream));
    return COULPS_OK;
  };
  cudaGraphExec_t exec = nullptr;
  if (L->stream != nullptr && !L->profiling && n_meas >= 8) {
    cudaGraph_t gr = nullptr;
    CK(cudaStreamBeginCapture(L->stream, cudaStreamCaptureModeThreadLocal));
    const int s1 = one();
    cudaError_t e = cudaStreamEndCapture(L->stream, &gr);
    if (s1 || e != cudaSuccess) {
      cudaGetLastError();
      if (gr) cudaGraphDestroy(gr);
      return s1 ? s1 : COULPS_ECUDA;
    }
    e = cudaGraphInstantiate(&exec, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return COULPS_ECUDA;
    }
  }
  int st = COULPS_OK;
  for (int k = 0; k < n_meas && !st; ++k) {
    if (exec) {
      if (cudaGraphLaunch(exec, L->stream) != cudaSuccess) {
        cudaGetLastError();
        st = COULPS_ECUDA;
      }
    } else {
      st = one();
    }
    if (!st) L->pass += (uint64_t)(n_hb + n_or);
  }
  if (exec) {
    cudaStreamSynchronize(L->stream);  // the replays are done before the graph goes
    cudaGraphExecDestroy(exec);
  }
  return st;
}

int coulps_charges_update(coulps_charges_t C, const int32_t *site, const double *q) {
  if (!C) return COULPS_EINVAL;
  if (C->off) return COULPS_EUNSUPPORTED;
  if (C->n == 0) return COULPS_OK;
  if (!site || !q) return COULPS_EINVAL;
  coulps_lattice *L = C->lat;
  const Geometry &g = L->g;
  const int64_t n = C->n;
  if (!C->h_idx) {
    // all three or none: a failure leaves the set as it was
    uint32_t *hi = nullptr;
    double *hq = nullptr;
    cudaEvent_t ev = nullptr;
    if (cudaMallocHost((void **)&hi, sizeof(uint32_t) * (size_t)n) != cudaSuccess ||
        cudaMallocHost((void **)&hq, sizeof(double) * (size_t)n) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      if (hi) cudaFreeHost(hi);
      if (hq) cudaFreeHost(hq);
      return COULPS_ENOMEM;
    }
    C->h_idx = hi;
    C->h_q = hq;
    C->staged = ev;
  } else {
    // the previous upload must have left the staging buffers
    CK(cudaEventSynchronize(C->staged));
  }
  for (int64_t i = 0; i < n; ++i) {
    const int x = site[3 * i], y = site[3 * i + 1], z = site[3 * i + 2];
    if (x < 0 || x >= g.Lx || y < 0 || y >= g.Ly || z < 0 || z >= g.Lz || !std::isfinite(q[i]))
      return COULPS_EINVAL;
    const int c = (x + y + z) & 1;
    C->h_idx[i] = (uint32_t)((size_t)c * g.colour_elems + ((size_t)z * g.Ly + y) * g.W + (x >> 1));
    C->h_q[i] = q[i];
  }
  for (int64_t i = 0; i < 3 * n; ++i) C->sites[i] = site[i];
  for (int64_t i = 0; i < n; ++i) C->qv[i] = q[i];
  C->gather_dirty = true;
  CK(cudaMemcpyAsync(C->d_idx, C->h_idx, sizeof(uint32_t) * (size_t)n, cudaMemcpyHostToDevice,
                     L->stream));
  CK(cudaMemcpyAsync(C->d_q, C->h_q, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice,
                     L->stream));
  CK(cudaEventRecord(C->staged, L->stream));
  return COULPS_OK;
}

int coulps_set_streams(coulps_lattice_t L, int n) {
  if (!L || n < 1 || n > 4) return COULPS_EINVAL;
  if (n == L->split) return COULPS_OK;
  drop_graph(L);
  if (n > 1 && !L->ev_fork &&
      cudaEventCreateWithFlags(&L->ev_fork, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return COULPS_ECUDA;
  }
  for (int j = 0; j < n - 1; ++j) {
    if (!L->xstream[j] &&
        (cudaStreamCreateWithFlags(&L->xstream[j], cudaStreamNonBlocking) != cudaSuccess ||
         cudaEventCreateWithFlags(&L->ev_join[j], cudaEventDisableTiming) != cudaSuccess)) {
      cudaGetLastError();
      return COULPS_ECUDA;
    }
  }
  L->split = n;
  return COULPS_OK;
}

int coulps_set_schedule(coulps_lattice_t L, int schedule) {
  if (!L || (schedule != COULPS_SCHEDULE_ALIGNED && schedule != COULPS_SCHEDULE_PHASED &&
             schedule != COULPS_SCHEDULE_SHIFTED))
    return COULPS_EINVAL;
  if (schedule != L->schedule) drop_graph(L);
  L->schedule = schedule;
  return COULPS_OK;
}

int coulps_set_profiling(coulps_lattice_t L, int enable) {
  if (!L) return COULPS_EINVAL;
  L->profiling = enable != 0;
  if (L->profiling) drop_graph(L);
  return COULPS_OK;
}

int coulps_kernel_times_n(coulps_lattice_t L, double *out, int n) {
  if (!L || !out || n < 0) return COULPS_EINVAL;
  CK(cudaStreamSynchronize(L->stream));
  for (auto &t : L->pending) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, t.a, t.b));
    L->times[2 * t.kind] += ms;
    L->times[2 * t.kind + 1] += 1;
    L->spare_events.push_back(t.a);
    L->spare_events.push_back(t.b);
  }
  L->pending.clear();
  for (int i = 0; i < coulps_lattice::kTimeSlots; ++i) {
    if (i < n) out[i] = L->times[i];
    L->times[i] = 0;
  }
  for (int i = coulps_lattice::kTimeSlots; i < n; ++i) out[i] = 0.0;
  return COULPS_OK;
}

int coulps_kernel_times(coulps_lattice_t L, double out[10]) {
  return coulps_kernel_times_n(L, out, 10);
}

int coulps_cv_pack_field(coulps_lattice_t L, const float *rho, void *act_bf16, float *Aphi) {
  if (!L) return COULPS_EINVAL;
  const int32_t origin[3] = {0, 0, 0}, dims[3] = {L->g.Lx, L->g.Ly, L->g.Lz};
  return coulps_cv_pack_region(L, rho, origin, dims, 0, act_bf16, Aphi);
}

int coulps_cv_pack_region(coulps_lattice_t L, const float *rho, const int32_t *origin,
                          const int32_t *dims, int interleave, void *act_bf16, float *Aphi) {
  if (!L || !rho || !origin || !dims || !act_bf16 || !Aphi) return COULPS_EINVAL;
  if (L->g.precision != COULPS_F32) return COULPS_EUNSUPPORTED;
  if (reinterpret_cast<uintptr_t>(act_bf16) & 15) return COULPS_EINVAL;
  const int Ls[3] = {L->g.Lx, L->g.Ly, L->g.Lz};
  int o[3], d[3];
  for (int k = 0; k < 3; ++k) {
    if (origin[k] < 0 || dims[k] < 1 || origin[k] + dims[k] > Ls[k]) return COULPS_EINVAL;
    o[k] = origin[k];
    d[k] = dims[k];
  }
  return coulps_cv_pack_field_impl(L->field, L->g, rho, act_bf16, Aphi, o, d, interleave != 0,
                                   L->stream);
}

// ---- checkpoint ------------------------------------------------------------
namespace {
struct CkptHeader {
  char magic[8];
  int64_t version;
  int64_t Lx, Ly, Lz, n_chains, precision, W;
  uint64_t seed, pass;
  int64_t has_charges, n_charges, stat_stride, log_cap;
};
}  // namespace

int coulps_checkpoint_save(coulps_lattice_t L, coulps_charges_t C, const char *path) {
  if (!L || !path || (C && C->lat != L)) return COULPS_EINVAL;
  const Geometry &g = L->g;
  CkptHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, "COULPS1", 8);
  h.version = 2;
  h.Lx = g.Lx; h.Ly = g.Ly; h.Lz = g.Lz; h.n_chains = g.n_chains;
  h.precision = g.precision; h.W = g.W;
  h.seed = L->seed;
  h.pass = L->pass;
  h.has_charges = C ? 1 : 0;
  h.n_charges = C ? C->n : 0;
  h.stat_stride = kStatStride;
  h.log_cap = C ? C->log_cap : 0;
  std::vector<unsigned char> field(g.chain_elems * g.es * (size_t)g.n_chains);
  std::vector<double> stats, log, cvstats, fsum;
  // version 2: after the log, {has control-variate state, has force sums}
  // and those blocks
  int64_t ex[2] = {C ? 1 : 0, (C && C->d_fsum) ? 1 : 0};
  CK(cudaMemcpyAsync(field.data(), L->field, field.size(), cudaMemcpyDeviceToHost, L->stream));
  if (C) {
    stats.resize((size_t)kStatStride * g.n_chains);
    log.resize((size_t)3 * C->log_cap * g.n_chains);
    CK(cudaMemcpyAsync(stats.data(), C->d_stats, stats.size() * sizeof(double),
                       cudaMemcpyDeviceToHost, L->stream));
    if (!log.empty())
      CK(cudaMemcpyAsync(log.data(), C->d_log, log.size() * sizeof(double),
                         cudaMemcpyDeviceToHost, L->stream));
    cvstats.resize(stats.size());
    CK(cudaMemcpyAsync(cvstats.data(), C->d_cvstats, cvstats.size() * sizeof(double),
                       cudaMemcpyDeviceToHost, L->stream));
    if (ex[1]) {
      fsum.resize((size_t)3 * C->n * g.n_chains);
      CK(cudaMemcpyAsync(fsum.data(), C->d_fsum, fsum.size() * sizeof(double),
                         cudaMemcpyDeviceToHost, L->stream));
    }
  }
  uint32_t dpass = 0;
  CK(cudaMemcpyAsync(&dpass, L->d_pass, sizeof(dpass), cudaMemcpyDeviceToHost, L->stream));
  int s = check_device_error(L);
  if (s) return s;
  h.pass = dpass;  // the device counter is authoritative
  uint64_t sum = 1469598103934665603ull;
  sum = fnv1a(sum, &h, sizeof(h));
  sum = fnv1a(sum, field.data(), field.size());
  sum = fnv1a(sum, stats.data(), stats.size() * sizeof(double));
  sum = fnv1a(sum, log.data(), log.size() * sizeof(double));
  sum = fnv1a(sum, ex, sizeof(ex));
  sum = fnv1a(sum, cvstats.data(), cvstats.size() * sizeof(double));
  sum = fnv1a(sum, fsum.data(), fsum.size() * sizeof(double));
  FILE *f = std::fopen(path, "wb");
  if (!f) return COULPS_EIO;
  bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1 &&
            std::fwrite(field.data(), 1, field.size(), f) == field.size() &&
            std::fwrite(stats.data(), sizeof(double), stats.size(), f) == stats.size() &&
            std::fwrite(log.data(), sizeof(double), log.size(), f) == log.size() &&
            std::fwrite(ex, sizeof(ex), 1, f) == 1 &&
            std::fwrite(cvstats.data(), sizeof(double), cvstats.size(), f) == cvstats.size() &&
            std::fwrite(fsum.data(), sizeof(double), fsum.size(), f) == fsum.size() &&
            std::fwrite(&sum, sizeof(sum), 1, f) == 1;
  ok = (std::fclose(f) == 0) && ok;
  return ok ? COULPS_OK : COULPS_EIO;
}

int coulps_checkpoint_load(coulps_lattice_t L, coulps_charges_t C, const char *path) {
  if (!L || !path || (C && C->lat != L)) return COULPS_EINVAL;
  const Geometry &g = L->g;
  FILE *f = std::fopen(path, "rb");
  if (!f) return COULPS_EIO;
  CkptHeader h;
  if (std::fread(&h, sizeof(h), 1, f) != 1) {
    std::fclose(f);
    return COULPS_ECORRUPT;
  }
  if (std::memcmp(h.magic, "COULPS1", 8) != 0 || (h.version != 1 && h.version != 2) ||
      h.Lx != g.Lx ||
      h.Ly != g.Ly || h.Lz != g.Lz || h.n_chains != g.n_chains || h.precision != g.precision ||
      h.W != g.W || h.seed != L->seed || h.stat_stride != kStatStride ||
      (C && (!h.has_charges || h.n_charges != C->n || h.log_cap != C->log_cap))) {
    std::fclose(f);
    return COULPS_ECORRUPT;
  }
  std::vector<unsigned char> field(g.chain_elems * g.es * (size_t)g.n_chains);
  std::vector<double> stats(h.has_charges ? (size_t)kStatStride * g.n_chains : 0);
  std::vector<double> log(h.has_charges ? (size_t)3 * h.log_cap * g.n_chains : 0);
  uint64_t sum_file = 0;
  bool ok = std::fread(field.data(), 1, field.size(), f) == field.size() &&
            std::fread(stats.data(), sizeof(double), stats.size(), f) == stats.size() &&
            std::fread(log.data(), sizeof(double), log.size(), f) == log.size();
  // version 2 extras: control-variate state and force sums (version 1: none)
  int64_t ex[2] = {0, 0};
  std::vector<double> cvstats, fsum;
  if (ok && h.version == 2) {
    ok = std::fread(ex, sizeof(ex), 1, f) == 1 && ex[0] == h.has_charges &&
         (ex[1] == 0 || ex[1] == 1) && (!ex[1] || h.has_charges);
    if (ok) {
      cvstats.resize(ex[0] ? stats.size() : 0);
      fsum.resize(ex[1] ? (size_t)3 * h.n_charges * g.n_chains : 0);
      ok = std::fread(cvstats.data(), sizeof(double), cvstats.size(), f) == cvstats.size() &&
           std::fread(fsum.data(), sizeof(double), fsum.size(), f) == fsum.size();
    }
  }
  ok = ok && std::fread(&sum_file, sizeof(sum_file), 1, f) == 1;
  std::fclose(f);
  if (!ok) return COULPS_ECORRUPT;
  uint64_t sum = 1469598103934665603ull;
  sum = fnv1a(sum, &h, sizeof(h));
  sum = fnv1a(sum, field.data(), field.size());
  sum = fnv1a(sum, stats.data(), stats.size() * sizeof(double));
  sum = fnv1a(sum, log.data(), log.size() * sizeof(double));
  if (h.version == 2) {
    sum = fnv1a(sum, ex, sizeof(ex));
    sum = fnv1a(sum, cvstats.data(), cvstats.size() * sizeof(double));
    sum = fnv1a(sum, fsum.data(), fsum.size() * sizeof(double));
  }
  if (sum != sum_file) return COULPS_ECORRUPT;
  // a set that keeps force sums needs them from the file, and only such a set takes them
  if (C && ((C->d_fsum != nullptr) != (ex[1] != 0))) return COULPS_ECORRUPT;
  const uint32_t dpass = (uint32_t)h.pass;
  CK(cudaMemcpyAsync(L->field, field.data(), field.size(), cudaMemcpyHostToDevice, L->stream));
  CK(cudaMemcpyAsync(L->d_pass, &dpass, sizeof(dpass), cudaMemcpyHostToDevice, L->stream));
  if (C) {
    CK(cudaMemcpyAsync(C->d_stats, stats.data(), stats.size() * sizeof(double),
                       cudaMemcpyHostToDevice, L->stream));
    if (!log.empty())
      CK(cudaMemcpyAsync(C->d_log, log.data(), log.size() * sizeof(double),
                         cudaMemcpyHostToDevice, L->stream));
    if (!cvstats.empty())
      CK(cudaMemcpyAsync(C->d_cvstats, cvstats.data(), cvstats.size() * sizeof(double),
                         cudaMemcpyHostToDevice, L->stream));
    else
      CK(launch_reset_stats(C->d_cvstats, g.n_chains, L->stream));
    if (!fsum.empty())
      CK(cudaMemcpyAsync(C->d_fsum, fsum.data(), fsum.size() * sizeof(double),
                         cudaMemcpyHostToDevice, L->stream));
  }
  CK(cudaStreamSynchronize(L->stream));
  L->pass = h.pass;
  return COULPS_OK;
}

}  // extern "C"
