// Per-tile z-march shared by the single-lattice and the many-system
// half-sweep kernels (see sweep.cu for the design).
#pragma once

#include "device_common.cuh"
#include "internal.h"

namespace coulps {
namespace tile {

// Ring depth (slots of other-colour planes) and barrier group of a march:
// the CTA synchronises once every GROUP planes and then refills the slots of
// the planes it has finished, so copies run GROUP .. STAGES - GROUP planes
// ahead.  A barrier per plane (GROUP = 1) was the heatbath half-sweep's second
// stall; the single-lattice kernels use 8 slots in groups of 4, the
// many-system kernel (whose largest systems' slots would cut its occupancy)
// 4 slots in groups of 1.  At most 8 slots: 8 mbarriers fill the header's
// first 64 bytes.
constexpr int kStages = 4;
constexpr int kLatticeStages = 8, kLatticeGroup = 4;

__host__ __device__ inline int round_up_int(int v, int m) { return (v + m - 1) / m * m; }

struct SmemLayout {
  int halo_bytes;  // exact TMA box bytes of the other colour: (TY + 2) * W * es
  int own_bytes;   // exact TMA box bytes of the own colour: TY * W * es (OR only)
  int slot_bytes;  // one ring slot, both boxes, each rounded to 128 bytes
  int total;       // header (barriers, flags, reduction) + ring, no alignment slack
};

// barriers at 0, abort flag at 64, block reduction (2 x 32 doubles) at 128
constexpr int kHeaderBytes = 1024;

__host__ __device__ inline SmemLayout smem_layout(int TY, int W, int es, bool orx,
                                                  int stages = kStages) {
  SmemLayout L;
  L.halo_bytes = (TY + 2) * W * es;
  L.own_bytes = orx ? TY * W * es : 0;
  L.slot_bytes = round_up_int(L.halo_bytes, 128) + round_up_int(L.own_bytes, 128);
  L.total = kHeaderBytes + stages * L.slot_bytes;
  return L;
}

template <typename T>
__device__ __forceinline__ void ld_quad(const T *p, T (&v)[4]);
template <>
__device__ __forceinline__ void ld_quad<float>(const float *p, float (&v)[4]) {
  const float4 f = *reinterpret_cast<const float4 *>(p);
  v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
}
template <>
__device__ __forceinline__ void ld_quad<double>(const double *p, double (&v)[4]) {
  const double2 a = reinterpret_cast<const double2 *>(p)[0];
  const double2 b = reinterpret_cast<const double2 *>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

template <typename T>
__device__ __forceinline__ void st_quad(T *p, const T (&v)[4]);
template <>
__device__ __forceinline__ void st_quad<float>(float *p, const float (&v)[4]) {
  *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void st_quad<double>(double *p, const double (&v)[4]) {
  reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}

// The x neighbours of a quad's 4 same-colour sites h .. h + 3 of a row: for
// row parity 0 the x - 1 neighbour of h is the other colour's h - 1 and x + 1
// is h; for parity 1 they are h and h + 1.  So S takes C[i] + xs[i], with
// xs[i] = C[i - 1] (even) or C[i + 1] (odd); the one value outside C is e
// (from shared memory, or 0 beyond the box).  Selects rather than a branch:
// the two rows one warp covers have opposite parity.
template <typename T>
__device__ __forceinline__ void x_neighbours(bool odd, T e, const T (&C)[4], T (&xs)[4]) {
  xs[0] = odd ? C[1] : e;
  xs[1] = odd ? C[2] : C[0];
  xs[2] = odd ? C[3] : C[1];
  xs[3] = odd ? e : C[2];
}

// A quad (four same-colour sites of a row) as two pairs: sites 0, 1 and 2, 3.
template <typename T> struct Pair2;
template <> struct Pair2<float> { using type = float2; };
template <> struct Pair2<double> { using type = double2; };

template <typename T>
struct Quad {
  typename Pair2<T>::type a, b;
};

__device__ __forceinline__ float2 padd(float2 p, float2 q) { return __fadd2_rn(p, q); }
__device__ __forceinline__ double2 padd(double2 p, double2 q) {
  return make_double2(p.x + q.x, p.y + q.y);
}
__device__ __forceinline__ float2 pfma(float2 p, float2 q, float2 r) { return __ffma2_rn(p, q, r); }
__device__ __forceinline__ double2 pfma(double2 p, double2 q, double2 r) {
  return make_double2(fma(p.x, q.x, r.x), fma(p.y, q.y, r.y));
}
__device__ __forceinline__ float2 pneg(float2 p) { return make_float2(-p.x, -p.y); }
__device__ __forceinline__ double2 pneg(double2 p) { return make_double2(-p.x, -p.y); }
__device__ __forceinline__ float2 pset(float c) { return make_float2(c, c); }
__device__ __forceinline__ double2 pset(double c) { return make_double2(c, c); }

// The heatbath deviates of one quad's four Philox words as two pairs (sites
// 0, 1 and 2, 3): FP32 as packed pairs, each under its own tail vote of the
// active lanes (no divergent branch per site), FP64 word by word.  Bitwise
// those of Noise<T>::of per word.  A warp's vote over 64 words finds a tail
// word (v >= 7, probability 0.0039 per word) 22% of the time, one over the
// quad's 128 words 39%: measured at 128^3 x 64 chains, 0.1498 against 0.1538
// ms per heatbath half-sweep with neighbour sums on packed pairs (before
// those, the vote per quad measured faster than a vote per site: 0.156
// against 0.159 ms).
template <typename T> struct QuadNoise2;
template <> struct QuadNoise2<float> {
  __device__ __forceinline__ static void of(uint4 w, float2 (&n)[2]) {
    const uint32_t u0[2] = {w.x, w.y}, u1[2] = {w.z, w.w};
    float2 a[1], b[1];
    hb_noise_pairs_f32<1>(u0, a);
    hb_noise_pairs_f32<1>(u1, b);
    n[0] = a[0];
    n[1] = b[0];
  }
};
template <> struct QuadNoise2<double> {
  __device__ __forceinline__ static void of(uint4 w, double2 (&n)[2]) {
    n[0] = make_double2(hb_noise_f64(w.x), hb_noise_f64(w.y));
    n[1] = make_double2(hb_noise_f64(w.z), hb_noise_f64(w.w));
  }
};

__device__ __forceinline__ float2 pair_of(const float (&a)[4], int h) {
  return make_float2(a[2 * h], a[2 * h + 1]);
}
__device__ __forceinline__ double2 pair_of(const double (&a)[4], int h) {
  return make_double2(a[2 * h], a[2 * h + 1]);
}

template <typename T> struct Coef;
template <> struct Coef<float> {
  static constexpr float sixth = 0.166666666666666666667f;
  static constexpr float third = 0.333333333333333333333f;
};
template <> struct Coef<double> {
  static constexpr double sixth = 0.166666666666666666667;
  static constexpr double third = 0.333333333333333333333;
};

// Accessors of a stored tile job: `name()` returns field `name_`.  The
// marches read their tile through such accessors, so that a kernel with one
// tile per CTA can instead answer each from its own parameters and block
// index at the point of use (see GridPass in pass_fused.cu).
#define COULPS_FIELD(type, name) \
  __device__ __forceinline__ type name() const { return name##_; }

// One tile of one half-sweep: TY rows (all of x) of one chain, planes
// z0 .. z0+nz-1, streamed as described at the top of this file: read through
// tm_halo / tm_own (4th coordinates map_other / map_own), the own colour
// written to out (element (z*Ly + y)*W + h), the other colour at `other`
// (GATHER only); Philox counter words quad, pass, rng_id (chain), colour;
// the fused gather of the tile column at g_off (GATHER only).  march_tile
// reads a tile through accessors of these names; TileJob stores them.  (For
// this march a stored job measured as fast as reading the kernel's
// parameters at each use, unlike the fused pass and the pair.)
template <typename T>
struct TileJob {
  const CUtensorMap *tm_halo_, *tm_own_;
  int map_other_, map_own_;
  T *out_;
  const T *other_;
  int Lx_, Ly_, Lz_, W_, Wq_, QW_, TY_;
  int y0_, z0_, nz_;
  int colour_;
  uint32_t rng_id_, pass_;
  const uint32_t *g_off_, *g_ent_;
  const double *g_q_;
  COULPS_FIELD(const CUtensorMap *, tm_halo) COULPS_FIELD(const CUtensorMap *, tm_own)
  COULPS_FIELD(int, map_other) COULPS_FIELD(int, map_own)
  COULPS_FIELD(T *, out) COULPS_FIELD(const T *, other)
  COULPS_FIELD(int, Lx) COULPS_FIELD(int, Ly) COULPS_FIELD(int, Lz) COULPS_FIELD(int, W)
  COULPS_FIELD(int, Wq) COULPS_FIELD(int, QW) COULPS_FIELD(int, TY)
  COULPS_FIELD(int, y0) COULPS_FIELD(int, z0) COULPS_FIELD(int, nz)
  COULPS_FIELD(int, colour)
  COULPS_FIELD(uint32_t, rng_id) COULPS_FIELD(uint32_t, pass)
  COULPS_FIELD(const uint32_t *, g_off) COULPS_FIELD(const uint32_t *, g_ent)
  COULPS_FIELD(const double *, g_q)
};

// Shared-memory ring header: STAGES mbarriers and the abort flag.  Done
// once per CTA; the barriers' phases then run on across every tile the CTA
// streams (see `gbase` below).
template <int STAGES = kStages>
__device__ __forceinline__ void ring_init(unsigned char *smem) {
  static_assert(STAGES <= 8 && (STAGES & (STAGES - 1)) == 0, "ring of at most 8, a power of 2");
  if (threadIdx.x == 0) {
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    for (int s = 0; s < STAGES; ++s) mbar_init(smem_addr(&bars[s]), 1);
    *reinterpret_cast<volatile int *>(smem + 64) = 0;
    fence_mbar_init();
  }
  __syncthreads();
}

// Runs the tile; with GATHER also accumulates this thread's share of
// Q = sum q phi and P = sum (q phi)^2 over the tile's charges into (sq, sp).
// `gbase` counts the planes this CTA has already streamed through its ring
// (the ring position and barrier phases continue from there) and is advanced
// past this tile's planes.  Returns false if a bounded wait gave up (the error
// word is set and no copy is left in flight).
//
// V quads per thread (V consecutive quads of a row, 4 V same-colour sites):
// V = 2 halves the per-site share of the loop's fixed work (waits, barrier,
// addresses, predicates) at the cost of registers; the sites' arithmetic is
// unchanged, so the results are bitwise those of V = 1.  The block has
// ceil(QW / V) threads per row.
template <typename T, bool OR, bool GATHER, int V = 1, int STAGES = kStages, int GROUP = 1,
          typename Job>
__device__ bool march_tile(const Job &j, const PhiloxKeys &K, unsigned char *smem,
                           int *err, int &gbase, double &sq, double &sp) {
  static_assert(GROUP >= 1 && GROUP < STAGES, "copies must run ahead of the group");
  const SmemLayout lay = smem_layout(j.TY(), j.W(), (int)sizeof(T), OR, STAGES);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem);  // STAGES barriers
  volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 64);
  unsigned char *ring = smem + kHeaderBytes;
  auto halo_slot = [&](int s) -> T * {
    return reinterpret_cast<T *>(ring + s * lay.slot_bytes);
  };
  auto own_slot = [&](int s) -> T * {
    return reinterpret_cast<T *>(ring + s * lay.slot_bytes + round_up_int(lay.halo_bytes, 128));
  };

  const int tid = threadIdx.x;
  const int W = j.W();
  const int qwv = (j.QW() + V - 1) / V;  // threads per row
  const int qx = (tid % qwv) * V, ty = tid / qwv;  // this thread's first quad
  const int n_planes = j.nz() + 2;  // other-colour planes z0-1 .. z0+nz
  const int c = j.colour();
  const int y = j.y0() + ty;
  // A CTA may have more threads than the tile has quads (the many-system
  // kernel runs tiles of different shapes with one block size): threads past
  // row TY - 1 touch no shared or global memory of the tile.
  const bool in_tile = ty < j.TY();
  const bool live = in_tile && (y < j.Ly()) && (qx < j.Wq());
  // quad v of this thread: inside the row's storage (loads), holds sites (updates)
  bool qmem[V], qlive[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    qmem[v] = in_tile && qx + v < j.QW();
    qlive[v] = live && qx + v < j.Wq();
  }

  const int gb = gbase;
  if (tid == 0) {
    prefetch_tensormap(j.tm_halo());
    if (OR) prefetch_tensormap(j.tm_own());
  }

  // Plane k of this tile is other-colour plane z0 - 1 + k; it is ring plane
  // gb + k, in slot (gb + k) % STAGES, completed in that slot's phase
  // (gb + k) / STAGES.
  auto slot_of = [&](int k) { return (gb + k) & (STAGES - 1); };
  auto issue = [&](int k) {
    const int s = slot_of(k);
    const uint32_t bar = smem_addr(&bars[s]);
    const bool own = OR && k >= 1 && k <= j.nz();
    mbar_arrive_expect_tx(bar, lay.halo_bytes + (own ? lay.own_bytes : 0));
    tma_load_4d(smem_addr(halo_slot(s)), j.tm_halo(), 0, j.y0() - 1, j.z0() - 1 + k, j.map_other(), bar);
    if (own) tma_load_4d(smem_addr(own_slot(s)), j.tm_own(), 0, j.y0(), j.z0() - 1 + k, j.map_own(), bar);
  };
  auto wait_plane = [&](int k) -> bool {
    return mbar_wait_bounded(smem_addr(&bars[slot_of(k)]), (uint32_t)(((gb + k) / STAGES) & 1));
  };

  int issued = 0;  // meaningful in thread 0 only
  int t0_waited = -1;  // thread 0: planes 0 .. t0_waited waited for (drained on abort)
  if (tid == 0)
    for (; issued < min(STAGES, n_planes); ++issued) issue(issued);
  // thread 0 refills every slot whose plane every thread has finished
  // (planes 0 .. last_free), in order
  auto refill = [&](int last_free) {
    if (tid == 0)
      while (issued < n_planes && issued - STAGES <= last_free) issue(issued++);
  };

  T cm[V][4], c0[V][4], cp[V][4];
#pragma unroll
  for (int v = 0; v < V; ++v)
#pragma unroll
    for (int i = 0; i < 4; ++i) cm[v][i] = c0[v][i] = cp[v][i] = T(0);
  bool ok = wait_plane(0);
  if (ok)
#pragma unroll
    for (int v = 0; v < V; ++v)
      if (qmem[v]) ld_quad(halo_slot(slot_of(0)) + (ty + 1) * W + 4 * (qx + v), cm[v]);
  ok = ok && wait_plane(1);
  if (ok)
#pragma unroll
    for (int v = 0; v < V; ++v)
      if (qmem[v]) ld_quad(halo_slot(slot_of(1)) + (ty + 1) * W + 4 * (qx + v), c0[v]);
  if (ok) t0_waited = 1;
  if (!ok) {
    atomicOr(err, kErrTimeout);
    *abort_flag = 1;
  }
  __syncthreads();
  bool aborted = *abort_flag != 0;

  // per-thread constants of the plane loop
  // quad lanes past x = Lx - 1 (kept at 0), row parity 0 / 1, per quad
  uint32_t pad0[V], pad1[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    pad0[v] = pad1[v] = 0u;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (2 * (4 * (qx + v) + i) >= j.Lx()) pad0[v] |= 1u << i;
      if (2 * (4 * (qx + v) + i) + 1 >= j.Lx()) pad1[v] |= 1u << i;
    }
  }
  const bool lo_ok = qx > 0, hi_ok = 4 * qx + 4 * V < W;
  const int hrow = (ty + 1) * W + 4 * qx;  // this quad in a halo box (first row y0 - 1)
  const int orow = ty * W + 4 * qx;        // this quad in an own box (first row y0)
  T *outp = j.out() + ((size_t)j.z0() * j.Ly() + y) * W + 4 * qx;  // plane z0; one plane per step
  const size_t pstride = (size_t)j.Ly() * W;
  int par = (c + y + j.z0()) & 1;  // the row (y, z) holds x = 2h + par; flips with z

  // Plane k (z = z0 + k - 1): M, C, P are the other colour's quads of planes
  // z - 1, z, z + 1 (P loaded here).  The loop calls it with the names
  // rotated, so no register is copied from plane to plane.
  //
  // Between barriers a thread that finds the abort flag set only skips its
  // work: whether the CTA stops is decided right after a barrier, where
  // every thread reads the same flag (a thread leaving early would miss the
  // barriers the others still reach).
  auto step = [&](int k, T(&M)[V][4], T(&C)[V][4], T(&P)[V][4]) -> bool {
    const bool got = *abort_flag == 0 && wait_plane(k + 1);
    if (got) t0_waited = k + 1;
    const T *Pz = halo_slot(slot_of(k)) + hrow;  // row y of plane z
    if (got) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        if (qmem[v]) {
          ld_quad(halo_slot(slot_of(k + 1)) + hrow + 4 * v, P[v]);
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i) P[v][i] = T(0);
        }
      }
      if (live) {
        const bool odd = par != 0;
        // the x neighbour beyond this thread's quads (left end when even,
        // right end when odd); between its own quads it is in registers
        const T edge = (odd ? hi_ok : lo_ok) ? Pz[odd ? 4 * V : -1] : T(0);
#pragma unroll
        for (int v = 0; v < V; ++v) {
          if (!qlive[v]) continue;
          T ym[4], yp[4], xs[4], u[4];
          ld_quad(Pz + 4 * v - W, ym);
          ld_quad(Pz + 4 * v + W, yp);
          const T e = odd ? (v + 1 < V ? C[v + 1 < V ? v + 1 : v][0] : edge)
                          : (v > 0 ? C[v > 0 ? v - 1 : v][3] : edge);
          x_neighbours(odd, e, C[v], xs);
          // the sums and the update on packed pairs of sites (FP32: one
          // instruction per pair, each lane rounded as the scalar form)
          using P2 = typename Pair2<T>::type;
          P2 S2[2], u2[2];
#pragma unroll
          for (int h = 0; h < 2; ++h)
            S2[h] = padd(padd(padd(pair_of(M[v], h), pair_of(P[v], h)),
                              padd(pair_of(ym, h), pair_of(yp, h))),
                         padd(pair_of(C[v], h), pair_of(xs, h)));
          if (!OR) {
            const uint32_t z = (uint32_t)(j.z0() + k - 1);
            const uint32_t quad =
                (z * (uint32_t)j.Ly() + (uint32_t)y) * (uint32_t)j.Wq() + (uint32_t)(qx + v);
            const uint4 w = philox4x32_10(make_uint4(quad, j.pass(), j.rng_id(), (uint32_t)c), K);
            P2 n2[2];
            QuadNoise2<T>::of(w, n2);
            u2[0] = pfma(S2[0], pset(Coef<T>::sixth), n2[0]);
            u2[1] = pfma(S2[1], pset(Coef<T>::sixth), n2[1]);
          } else {
            T old[4];
            ld_quad(own_slot(slot_of(k)) + orow + 4 * v, old);
#pragma unroll
            for (int h = 0; h < 2; ++h)
              u2[h] = pfma(S2[h], pset(Coef<T>::third), pneg(pair_of(old, h)));
          }
          u[0] = u2[0].x;
          u[1] = u2[0].y;
          u[2] = u2[1].x;
          u[3] = u2[1].y;
          const uint32_t pm = par ? pad1[v] : pad0[v];
          if (pm) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
              if ((pm >> i) & 1u) u[i] = T(0);  // keep the row padding at 0
          }
          st_quad(outp + 4 * v, u);
        }
      }
    } else {
      atomicOr(err, kErrTimeout);
      *abort_flag = 1;
    }
    outp += pstride;
    par ^= 1;
    if (k % GROUP == 0 || k == j.nz()) {
      __syncthreads();
      if (*abort_flag) return false;
      // planes 0 .. k are no longer read: refill their slots
      refill(k);
    }
    return true;
  };

  if (!aborted) {
    refill(0);  // plane 0 was read only above
    for (int k = 1; k <= j.nz(); k += 3) {
      if (!step(k, cm, c0, cp)) { aborted = true; break; }
      if (k + 1 > j.nz()) break;
      if (!step(k + 1, c0, cp, cm)) { aborted = true; break; }
      if (k + 2 > j.nz()) break;
      if (!step(k + 2, cp, cm, c0)) { aborted = true; break; }
    }
  }
  if (aborted && tid == 0) {
    // Leave no copy in flight into this CTA's shared memory.
    for (int k = t0_waited + 1; k < issued; ++k)
      if (!wait_plane(k)) break;
  }
  gbase = gb + n_planes;
  if (GATHER && !aborted) {
    // Q and P over the tile's charges, once the whole tile is written: the
    // barrier makes this CTA's global stores visible to all its threads, and
    // both colours of the tile are still in L2.  An entry holds its site's
    // colour and offset within the colour's array.
    __syncthreads();
    const uint32_t e0 = j.g_off()[j.z0()], e1 = j.g_off()[j.z0() + j.nz()];
    for (uint32_t e = e0 + tid; e < e1; e += blockDim.x) {
      const uint32_t ent = j.g_ent()[e];
      const size_t at = ent & ~kGatherColourBit;
      const bool own = ((ent >> 31) & 1u) == (uint32_t)c;
      const T val = own ? j.out()[at] : j.other()[at];
      const double t = j.g_q()[e] * (double)val;
      sq += t;
      sp += t * t;
    }
  }
  return !aborted;
}

// Block reduction of (sq, sp) into one partial per CTA (fixed order).
__device__ __forceinline__ void block_partials(double sq, double sp, unsigned char *smem,
                                               double *out) {
  double *red = reinterpret_cast<double *>(smem + 128);  // 2 x 32 doubles
  sq = warp_sum(sq);
  sp = warp_sum(sp);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) {
    red[wid] = sq;
    red[32 + wid] = sp;
  }
  __syncthreads();
  if (wid == 0) {
    sq = lane < nw ? red[lane] : 0.0;
    sp = lane < nw ? red[32 + lane] : 0.0;
    sq = warp_sum(sq);
    sp = warp_sum(sp);
    if (lane == 0) {
      out[0] = sq;
      out[1] = sp;
    }
  }
  __syncthreads();  // red[] is free again
}

}  // namespace tile
}  // namespace coulps
