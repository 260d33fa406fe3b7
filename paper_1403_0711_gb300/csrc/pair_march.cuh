// One tile of a pass pair (two passes in one z-march from a source copy of
// the field to a destination copy, four stages one plane apart; see
// pass_pair.cu for the design), shared by the single-lattice pair kernel and
// the many-system kernel.  A CTA may march several tiles of different
// systems in a row: the ring's mbarrier phases run on from tile to tile
// (`gbase`).
#pragma once

#include "device_common.cuh"
#include "internal.h"
#include "tile_march.cuh"

namespace coulps {
namespace tile {

// Ring depth: one CTA per SM streams the pair, so several planes (tens of KB)
// must be in flight to cover DRAM latency (measured at 128^3 x 64 chains,
// over-relaxation pairs: 0.373 ms per launch with 4 slots, 0.292 with 8).
constexpr int kPairStages = 8;
// header: kPairStages (<= 12) mbarriers at 0, abort flag at 96, block reduction at 128
constexpr int kPairAbort = 96;
static_assert(kPairStages <= 12, "mbarriers must end before the abort flag");

struct PairLayout {
  int c1_bytes;   // colour-1 box: (TY + 8) rows x W
  int c0_bytes;   // colour-0 box: (TY + 6) rows x W (pass A over-relaxation only)
  int slot_bytes;
  int buf_bytes;  // one plane of one stage's rows: (TY + 6) x W
  int total;      // header + ring slots + 3 stages x 2 planes
};

__host__ __device__ inline PairLayout pair_layout(int TY, int W, int es, bool a_or) {
  PairLayout L;
  L.c1_bytes = (TY + 8) * W * es;
  L.c0_bytes = a_or ? (TY + 6) * W * es : 0;
  L.slot_bytes = round_up_int(L.c1_bytes, 128) + round_up_int(L.c0_bytes, 128);
  L.buf_bytes = round_up_int((TY + 6) * W * es, 128);
  L.total = kHeaderBytes + kPairStages * L.slot_bytes + 6 * L.buf_bytes;
  return L;
}

template <typename T>
__device__ __forceinline__ Quad<T> qzero() {
  Quad<T> q;
  q.a = pset(T(0));
  q.b = pset(T(0));
  return q;
}

template <typename T>
__device__ __forceinline__ Quad<T> qload(const T *p);
template <>
__device__ __forceinline__ Quad<float> qload<float>(const float *p) {
  const float4 f = *reinterpret_cast<const float4 *>(p);
  Quad<float> q;
  q.a = make_float2(f.x, f.y);
  q.b = make_float2(f.z, f.w);
  return q;
}
template <>
__device__ __forceinline__ Quad<double> qload<double>(const double *p) {
  Quad<double> q;
  q.a = reinterpret_cast<const double2 *>(p)[0];
  q.b = reinterpret_cast<const double2 *>(p)[1];
  return q;
}

template <typename T>
__device__ __forceinline__ void qstore(T *p, const Quad<T> &q);
template <>
__device__ __forceinline__ void qstore<float>(float *p, const Quad<float> &q) {
  *reinterpret_cast<float4 *>(p) = make_float4(q.a.x, q.a.y, q.b.x, q.b.y);
}
template <>
__device__ __forceinline__ void qstore<double>(double *p, const Quad<double> &q) {
  reinterpret_cast<double2 *>(p)[0] = q.a;
  reinterpret_cast<double2 *>(p)[1] = q.b;
}

// The heatbath deviates of two quads (two stages' Philox words): FP32 as
// four packed pairs under one warp vote (every lane of the warp must call
// it); FP64 word by word.
template <typename T> struct StageNoise;
template <> struct StageNoise<float> {
  __device__ __forceinline__ static void of(uint4 wa, uint4 wb, Quad<float> &na,
                                            Quad<float> &nb) {
    const uint32_t w[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
    float2 o[4];
    hb_noise_pairs_f32<4>(w, o);
    na.a = o[0];
    na.b = o[1];
    nb.a = o[2];
    nb.b = o[3];
  }
};
template <> struct StageNoise<double> {
  __device__ __forceinline__ static void of(uint4 wa, uint4 wb, Quad<double> &na,
                                            Quad<double> &nb) {
    na.a = make_double2(hb_noise_f64(wa.x), hb_noise_f64(wa.y));
    na.b = make_double2(hb_noise_f64(wa.z), hb_noise_f64(wa.w));
    nb.a = make_double2(hb_noise_f64(wb.x), hb_noise_f64(wb.y));
    nb.b = make_double2(hb_noise_f64(wb.z), hb_noise_f64(wb.w));
  }
};

// The new values of a quad.  zm, zp: the other colour's quad on planes
// z -+ 1; ym, yp: rows y -+ 1; c: same row and plane; e: the x neighbour
// outside c (the previous quad's last site for an even row, the next quad's
// first for an odd row; 0 beyond the box); r: the site's value before the
// pass (over-relaxation) or the heatbath deviates.  Sums in the order of the
// half-sweep kernel: S = ((zm + zp) + (ym + yp)) + (c + xs), then
// S/3 - old or S/6 + deviate by one fma.
template <typename T, bool OR>
__device__ __forceinline__ Quad<T> update(const Quad<T> &zm, const Quad<T> &zp, const Quad<T> &ym,
                                          const Quad<T> &yp, const Quad<T> &c, bool odd, T e,
                                          const Quad<T> &r) {
  using P2 = typename Pair2<T>::type;
  P2 xa, xb;
  xa.x = odd ? c.a.y : e;
  xa.y = odd ? c.b.x : c.a.x;
  xb.x = odd ? c.b.y : c.a.y;
  xb.y = odd ? e : c.b.x;
  Quad<T> S, v;
  S.a = padd(padd(padd(zm.a, zp.a), padd(ym.a, yp.a)), padd(c.a, xa));
  S.b = padd(padd(padd(zm.b, zp.b), padd(ym.b, yp.b)), padd(c.b, xb));
  if (OR) {
    const P2 third = pset(Coef<T>::third);
    v.a = pfma(S.a, third, pneg(r.a));
    v.b = pfma(S.b, third, pneg(r.b));
  } else {
    const P2 sixth = pset(Coef<T>::sixth);
    v.a = pfma(S.a, sixth, r.a);
    v.b = pfma(S.b, sixth, r.b);
  }
  return v;
}

// Zero what is not a site of the box: the whole quad when `valid` is false
// (a ghost row or plane), else the lanes past x = Lx - 1 (bit i of pm: site i
// of the quad).  `fast` (warp-uniform): nothing to zero.
template <typename T>
__device__ __forceinline__ Quad<T> mask(Quad<T> v, bool fast, bool valid, uint32_t pm) {
  if (fast) return v;
  if (!valid) return qzero<T>();
  if (pm) {
    if (pm & 1u) v.a.x = T(0);
    if (pm & 2u) v.a.y = T(0);
    if (pm & 4u) v.b.x = T(0);
    if (pm & 8u) v.b.y = T(0);
  }
  return v;
}

// The tile: TY rows from y0 and planes [z0, z0 + nz) of one chain (or
// system), read through tm_c1 (TY + 8 rows) / tm_c0 (TY + 6 rows) with 4th
// coordinates map_c1 / map_c0, written to dst (colour 0) and dst +
// colour_elems (colour 1), element (z Ly + y) W + h.  Philox counter words:
// quad, pass (pass A; B is pass + 1), rng_id, colour.  With GATHER, g_off
// points at the tile column's plane offsets (entries of plane z:
// [g_off[z], g_off[z + 1])).  march_pair reads a tile through accessors of
// these names, as march_pass does (pass_march.cuh): PairTile stores them for
// the many-system kernel, the one-tile-per-CTA kernel reads its parameters.
template <typename T>
struct PairTile {
  // the CTA may have whole warps past the tile's rows (one block size for
  // tiles of every system): they skip the stages
  static constexpr bool kIdleWarps = true;
  const CUtensorMap *tm_c1_, *tm_c0_;
  int map_c1_, map_c0_;
  T *dst_;
  size_t colour_elems_;
  int Lx_, Ly_, Lz_, W_, Wq_, QW_, TY_;
  int y0_, z0_, nz_;
  uint32_t rng_id_, pass_;
  const uint32_t *g_off_, *g_ent_;
  const double *g_q_;
  COULPS_FIELD(const CUtensorMap *, tm_c1) COULPS_FIELD(const CUtensorMap *, tm_c0)
  COULPS_FIELD(int, map_c1) COULPS_FIELD(int, map_c0)
  COULPS_FIELD(T *, dst) COULPS_FIELD(size_t, colour_elems)
  COULPS_FIELD(int, Lx) COULPS_FIELD(int, Ly) COULPS_FIELD(int, Lz) COULPS_FIELD(int, W)
  COULPS_FIELD(int, Wq) COULPS_FIELD(int, QW) COULPS_FIELD(int, TY)
  COULPS_FIELD(int, y0) COULPS_FIELD(int, z0) COULPS_FIELD(int, nz)
  COULPS_FIELD(uint32_t, rng_id) COULPS_FIELD(uint32_t, pass)
  COULPS_FIELD(const uint32_t *, g_off) COULPS_FIELD(const uint32_t *, g_ent)
  COULPS_FIELD(const double *, g_q)
};

// Shared-memory header of a pair CTA: kPairStages mbarriers and the abort
// flag; done once per CTA.
__device__ __forceinline__ void pair_ring_init(unsigned char *smem) {
  if (threadIdx.x == 0) {
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    for (int k = 0; k < kPairStages; ++k) mbar_init(smem_addr(&bars[k]), 1);
    *reinterpret_cast<volatile int *>(smem + kPairAbort) = 0;
    fence_mbar_init();
  }
  __syncthreads();
}

// Runs the tile; with GATHER adds this thread's share of Q and P over the
// tile's charges to (sq, sp).  `gbase` counts the ring planes this CTA has
// streamed before and is advanced past this tile's.  Returns false if a
// bounded wait gave up (the error word is set and no copy is left in flight).
// With Job::kIdleWarps, warps with no row of the tile only take part in the
// barriers.
template <typename T, bool A_OR, bool B_OR, bool GATHER, typename Job>
__device__ bool march_pair(const Job &a, const PhiloxKeys &K, unsigned char *smem, int *err,
                           int &gbase, double &sq, double &sp) {
  const PairLayout lay = pair_layout(a.TY(), a.W(), (int)sizeof(T), A_OR);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + kPairAbort);
  unsigned char *ring = smem + kHeaderBytes;
  unsigned char *bufs = ring + kPairStages * lay.slot_bytes;
  const int gb = gbase;
  auto c1_slot = [&](int j) {
    return reinterpret_cast<const T *>(ring + ((gb + j) % kPairStages) * lay.slot_bytes);
  };
  auto c0_slot = [&](int j) {
    return reinterpret_cast<const T *>(ring + ((gb + j) % kPairStages) * lay.slot_bytes +
                                       round_up_int(lay.c1_bytes, 128));
  };
  auto buf = [&](int k, int par) {
    return reinterpret_cast<T *>(bufs + (2 * k + (par & 1)) * lay.buf_bytes);
  };

  const int W = a.W(), TY = a.TY(), QW = a.QW(), Ly = a.Ly(), Lz = a.Lz();
  const int y0 = a.y0(), z0 = a.z0(), nz = a.nz();
  const int tid = threadIdx.x;
  const int rows = TY + 6;
  // this thread: quad qx of row r (y = y0 - 3 + r); lanes past the last row
  // (block rounded up to whole warps) alias the last row's addresses for
  // their loads and store nothing (their stores would race with that row's)
  const int qx = tid % QW;
  const bool lane_ok = tid < rows * QW;
  const int r = lane_ok ? tid / QW : rows - 1;
  const int y = y0 - 3 + r;
  const bool live = lane_ok && y >= 0 && y < Ly && qx < a.Wq();
  const bool own_row = live && r >= 3 && r < TY + 3;  // a row of this tile: written out
  // rows of this warp, for skipping a stage that has none of them
  const int wr_lo = (tid & ~31) / QW, wr_hi = (tid | 31) / QW;
  bool warp_in[4];  // warp_in[0]: the warp has a row of the tile at all
#pragma unroll
  for (int k = 0; k < 4; ++k) warp_in[k] = wr_hi >= k && wr_lo <= rows - 1 - k;

  // offsets: row r in a buffer / colour-0 box, row r + 1 in the colour-1 box
  const int o_r = r * W + 4 * qx;
  const int o_m = max(r - 1, 0) * W + 4 * qx;         // clamped for rows no stage reads
  const int o_p = min(r + 1, rows - 1) * W + 4 * qx;
  const bool lo_ok = qx > 0, hi_ok = 4 * qx + 4 < W;
  uint32_t pad0 = 0u, pad1 = 0u;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (2 * (4 * qx + i) >= a.Lx()) pad0 |= 1u << i;
    if (2 * (4 * qx + i) + 1 >= a.Lx()) pad1 |= 1u << i;
  }
  // the whole warp is inside the box and has no padding lanes
  const bool warp_full = __all_sync(0xffffffffu, live && pad0 == 0u && pad1 == 0u);
  T *dst0 = a.dst();
  T *dst1 = dst0 + a.colour_elems();
  const size_t plane_elems = (size_t)Ly * W;
  const size_t row_off = (size_t)(y < 0 ? 0 : y) * W + 4 * qx;
  const uint32_t pass_a = a.pass();
  const uint32_t pass_b = pass_a + 1u;
  const uint32_t rng = a.rng_id();
  // Philox counter word 0 of the quad at plane p: (p Ly + y) Wq + qx
  const uint32_t qrow = (uint32_t)y * (uint32_t)a.Wq() + (uint32_t)qx;
  const uint32_t qplane = (uint32_t)Ly * (uint32_t)a.Wq();

  const int n_ring = nz + 8;  // colour-1 planes z0 - 4 .. z0 + nz + 3
  if (tid == 0) {
    prefetch_tensormap(a.tm_c1());
    if (A_OR) prefetch_tensormap(a.tm_c0());
  }
  // ring plane j: colour 1 at z0 - 4 + j, with it (j >= 2) colour 0 at z0 - 5 + j
  auto issue = [&](int j) {
    const uint32_t bar = smem_addr(&bars[(gb + j) % kPairStages]);
    const bool own = A_OR && j >= 2;
    mbar_arrive_expect_tx(bar, lay.c1_bytes + (own ? lay.c0_bytes : 0));
    tma_load_4d(smem_addr(c1_slot(j)), a.tm_c1(), 0, y0 - 4, z0 - 4 + j, a.map_c1(), bar);
    if (own) tma_load_4d(smem_addr(c0_slot(j)), a.tm_c0(), 0, y0 - 3, z0 - 5 + j, a.map_c0(), bar);
  };
  auto wait_plane = [&](int j) -> bool {
    return mbar_wait_bounded(smem_addr(&bars[(gb + j) % kPairStages]),
                             (uint32_t)(((gb + j) / kPairStages) & 1));
  };
  int issued = 0;
  if (tid == 0)
    for (; issued < min(kPairStages, n_ring); ++issued) issue(issued);
  // fused gather: this CTA's charge range, and this thread's first entry,
  // loaded while the first planes arrive (used once the tile is written)
  uint32_t g_e = 0u, g_e1 = 0u, g_ent0 = 0u;
  double g_q0 = 0.0;
  if (GATHER) {
    const uint32_t *g_off = a.g_off();
    g_e = g_off[z0] + (uint32_t)tid;
    g_e1 = g_off[z0 + nz];
    if (g_e < g_e1) {
      g_ent0 = a.g_ent()[g_e];
      g_q0 = a.g_q()[g_e];
    }
  }
  {
    const bool ok = wait_plane(0) && wait_plane(1);
    if (!ok) {
      atomicOr(err, kErrTimeout);
      *abort_flag = 1;
    }
  }
  __syncthreads();
  bool aborted = *abort_flag != 0;
  int done = 1;  // ring planes 0 .. done completed for every thread

  // windows, per stage, of the quad's three planes (see the step): old colour
  // 1 (P), colour 0 after A (Q), colour 1 after A (R), colour 0 after B (U)
  Quad<T> P0 = qzero<T>(), P1 = qzero<T>(), P2 = qzero<T>();
  Quad<T> Q0 = qzero<T>(), Q1 = qzero<T>(), Q2 = qzero<T>();
  Quad<T> R0 = qzero<T>(), R1 = qzero<T>(), R2 = qzero<T>();
  Quad<T> U0 = qzero<T>(), U1 = qzero<T>(), U2 = qzero<T>();
  if (!aborted) {
    P0 = qload(c1_slot(0) + o_r + W);
    P1 = qload(c1_slot(1) + o_r + W);
  }

  // Step s with the windows' names rotated by the caller.  At entry:
  // P0, P1 = old colour 1 at f - 1, f (P2 loaded here: f + 1); Q0, Q1 =
  // colour 0 after A at f - 2, f - 1 (Q2 made here: f); R0, R1 = colour 1
  // after A at f - 3, f - 2 (R2: f - 1); U0, U1 = colour 0 after B at f - 4,
  // f - 3 (U2: f - 2).  Ring planes s, s + 1 have arrived; s + 2 is waited
  // for here.
  //
  // What needs no other warp's rows of this step -- the heatbath deviates
  // (Philox words and erfc^-1) of every stage and the whole of stage 0,
  // which reads only the ring -- comes before the step's one barrier, so a
  // warp that finished the previous step early goes on with it while the
  // others finish.  After the barrier (all warps are through the previous
  // step: its buffer writes are visible and the buffers it read are free)
  // stages 1 .. 3 read the previous step's buffers and write this step's.
  auto step = [&](int s, Quad<T> &P0, Quad<T> &P1, Quad<T> &P2, Quad<T> &Q0, Quad<T> &Q1,
                  Quad<T> &Q2, Quad<T> &R0, Quad<T> &R1, Quad<T> &R2, Quad<T> &U0, Quad<T> &U1,
                  Quad<T> &U2) -> bool {
    const int f = z0 - 3 + s;
    const bool odd = ((y + f) & 1) != 0;  // the same row parity for all four stages
    const uint32_t pm = odd ? pad1 : pad0;
    const int eo = odd ? 4 : -1;
    const bool e_ok = odd ? hi_ok : lo_ok;
    bool plane_ok[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) plane_ok[k] = f - k >= 0 && f - k < Lz;
    // the whole warp agrees on the outcome, so it never splits around the
    // heatbath deviates' warp vote
    const bool got = __all_sync(0xffffffffu, wait_plane(s + 2));
    if (!got) {
      atomicOr(err, kErrTimeout);
      *abort_flag = 1;
    }
    Quad<T> nA0 = qzero<T>(), nA1 = qzero<T>(), nB0 = qzero<T>(), nB1 = qzero<T>();
    if (got && (!Job::kIdleWarps || warp_in[0])) {
      if (!A_OR) {
        const uint4 w0 = philox4x32_10(
            make_uint4((uint32_t)f * qplane + qrow, pass_a, rng, 0u), K);
        const uint4 w1 = philox4x32_10(
            make_uint4((uint32_t)(f - 1) * qplane + qrow, pass_a, rng, 1u), K);
        StageNoise<T>::of(w0, w1, nA0, nA1);
      }
      if (!B_OR && s >= 4) {
        const uint4 w2 = philox4x32_10(
            make_uint4((uint32_t)(f - 2) * qplane + qrow, pass_b, rng, 0u), K);
        const uint4 w3 = philox4x32_10(
            make_uint4((uint32_t)(f - 3) * qplane + qrow, pass_b, rng, 1u), K);
        StageNoise<T>::of(w2, w3, nB0, nB1);
      }
      // ---- stage 0: colour 0 of pass A at plane f (ring only)
      const T *C = c1_slot(s + 1);  // old colour 1, plane f (box row r + 1)
      P2 = qload(c1_slot(s + 2) + o_r + W);
      const Quad<T> ym = qload(C + o_r), yp = qload(C + o_r + 2 * W);
      const T e = e_ok ? C[o_r + W + eo] : T(0);
      Quad<T> r0 = nA0;
      if (A_OR) r0 = qload(c0_slot(s + 2) + o_r);
      const Quad<T> v = update<T, A_OR>(P0, P2, ym, yp, P1, odd, e, r0);
      Q2 = mask(v, warp_full && plane_ok[0], live && plane_ok[0], pm);
    }
    __syncthreads();
    if (*abort_flag) return false;
    done = s + 2;
    // ring plane s was last read in the previous step: refill its slot
    if (tid == 0 && issued < n_ring) issue(issued++);
    if (lane_ok) qstore(buf(0, s) + o_r, Q2);
    // ---- stage 1: colour 1 of pass A at plane f - 1 (old value: P0)
    if (s >= 2 && warp_in[1]) {
      const T *B = buf(0, s - 1);  // colour 0 after A, plane f - 1
      const Quad<T> ym = qload(B + o_m), yp = qload(B + o_p);
      const T e = e_ok ? B[o_r + eo] : T(0);
      const Quad<T> v = update<T, A_OR>(Q0, Q2, ym, yp, Q1, odd, e, A_OR ? P0 : nA1);
      R2 = mask(v, warp_full && plane_ok[1], live && plane_ok[1], pm);
      if (lane_ok) qstore(buf(1, s) + o_r, R2);
    }
    // ---- stage 2: colour 0 of pass B at plane f - 2 (old value: Q0)
    if (s >= 4 && warp_in[2]) {
      const T *B = buf(1, s - 1);  // colour 1 after A, plane f - 2
      const Quad<T> ym = qload(B + o_m), yp = qload(B + o_p);
      const T e = e_ok ? B[o_r + eo] : T(0);
      const Quad<T> v = update<T, B_OR>(R0, R2, ym, yp, R1, odd, e, B_OR ? Q0 : nB0);
      const int p = f - 2;
      U2 = mask(v, warp_full && plane_ok[2], live && plane_ok[2], pm);
      if (lane_ok) qstore(buf(2, s) + o_r, U2);
      if (own_row && p >= z0 && p < z0 + nz) qstore(dst0 + (size_t)p * plane_elems + row_off, U2);
    }
    // ---- stage 3: colour 1 of pass B at plane f - 3 (old value: R0)
    if (s >= 6 && warp_in[3]) {
      const T *B = buf(2, s - 1);  // colour 0 after B, plane f - 3
      const Quad<T> ym = qload(B + o_m), yp = qload(B + o_p);
      const T e = e_ok ? B[o_r + eo] : T(0);
      const Quad<T> v = update<T, B_OR>(U0, U2, ym, yp, U1, odd, e, B_OR ? R0 : nB1);
      const int p = f - 3;
      if (own_row && p >= z0 && p < z0 + nz)
        qstore(dst1 + (size_t)p * plane_elems + row_off, mask(v, warp_full, true, pm));
    }
    return true;
  };

  const int n_steps = nz + 6;
  for (int s = 0; s < n_steps && !aborted; s += 3) {
    if (!step(s, P0, P1, P2, Q0, Q1, Q2, R0, R1, R2, U0, U1, U2)) { aborted = true; break; }
    if (s + 1 >= n_steps) break;
    if (!step(s + 1, P1, P2, P0, Q1, Q2, Q0, R1, R2, R0, U1, U2, U0)) { aborted = true; break; }
    if (s + 2 >= n_steps) break;
    if (!step(s + 2, P2, P0, P1, Q2, Q0, Q1, R2, R0, R1, U2, U0, U1)) { aborted = true; break; }
  }
  if (aborted && tid == 0) {
    // leave no copy in flight into this CTA's shared memory
    for (int k = done + 1; k < issued; ++k)
      if (!wait_plane(k)) break;
  }
  gbase = gb + n_ring;
  if (GATHER) {
    __syncthreads();  // this CTA's stores of the last step are visible to all its threads
    if (!aborted) {
      // both colours of the tile are still in L2; an entry holds its site's
      // colour and offset within the colour's array
      for (uint32_t e = g_e; e < g_e1; e += blockDim.x) {
        const uint32_t ent = e == g_e ? g_ent0 : a.g_ent()[e];
        const double qe = e == g_e ? g_q0 : a.g_q()[e];
        const uint32_t at = ent & ~kGatherColourBit;
        const T val = (ent & kGatherColourBit) ? dst1[at] : dst0[at];
        const double t = qe * (double)val;
        sq += t;
        sp += t * t;
      }
    }
  }
  return !aborted;
}


}  // namespace tile
}  // namespace coulps
