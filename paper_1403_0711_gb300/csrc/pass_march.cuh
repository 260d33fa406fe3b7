// One tile of a fused pass (both half-sweeps of one pass in a single z-march
// from a source copy of the field to a destination copy; see pass_fused.cu for
// the design), shared by the single-lattice pass kernel and the many-system
// kernel.  A CTA may march several tiles of different systems in a row: the
// ring's mbarrier phases run on from tile to tile (`gbase`).
#pragma once

#include "device_common.cuh"
#include "internal.h"
#include "tile_march.cuh"

namespace coulps {
namespace tile {

// Ring depth of the fused pass (slots of one colour-1 box and one colour-0
// box); at most 8 (mbarriers at 0 .. 63 of the header, abort flag at 64).
// Measured at 128^3 x 64 chains: 0.203 ms per over-relaxation pass with 4
// slots, 0.194 with 6, 0.196 with 8.
constexpr int kPassStages = 6;
static_assert(kPassStages <= 8, "mbarriers must end before the abort flag");

struct PassLayout {
  int c1_bytes;    // colour-1 box: (TY + 4) rows x W
  int c0_bytes;    // colour-0 box: (TY + 2) rows x W (over-relaxation only)
  int slot_bytes;  // both, each rounded to 128 bytes
  int new_bytes;   // one plane of new colour-0 rows: (TY + 2) x W
  int total;       // header + 4 slots + 2 new planes
};

__host__ __device__ inline PassLayout pass_layout(int TY, int W, int es, bool orx) {
  PassLayout L;
  L.c1_bytes = (TY + 4) * W * es;
  L.c0_bytes = orx ? (TY + 2) * W * es : 0;
  L.slot_bytes = round_up_int(L.c1_bytes, 128) + round_up_int(L.c0_bytes, 128);
  L.new_bytes = round_up_int((TY + 2) * W * es, 128);
  L.total = kHeaderBytes + kPassStages * L.slot_bytes + 2 * L.new_bytes;
  return L;
}

// The tile: TY rows from y0 and planes [z0, z0 + nz) of one chain (or
// system), read through tm_c1 / tm_c0 (4th coordinates map_c1 / map_c0) and
// written to dst (colour 0) and dst + colour_elems (colour 1), element
// (z Ly + y) W + h.  Philox counter words: quad, pass, rng_id, colour.  With
// GATHER, g_off points at the tile column's plane offsets (entries of plane
// z: [g_off[z], g_off[z + 1])).
//
// march_pass reads a tile through accessors of these names.  PassTile
// stores them (the many-system kernel fills one per tile of its work list);
// the one-tile-per-CTA kernel answers from its parameters and block index at
// the point of use, which measured 8% fewer instructions than a stored job
// (the compiler then shares the address arithmetic of the two colours and
// keeps the origin out of registers).
template <typename T>
struct PassTile {
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

// Shared-memory header of a pass CTA: kPassStages mbarriers and the abort
// flag; done once per CTA.
__device__ __forceinline__ void pass_ring_init(unsigned char *smem) {
  if (threadIdx.x == 0) {
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    for (int k = 0; k < kPassStages; ++k) mbar_init(smem_addr(&bars[k]), 1);
    *reinterpret_cast<volatile int *>(smem + 64) = 0;
    fence_mbar_init();
  }
  __syncthreads();
}

// Runs the tile; with GATHER adds this thread's share of Q and P over the
// tile's charges to (sq, sp).  `gbase` counts the ring planes this CTA has
// streamed before (phases continue from there) and is advanced past this
// tile's.  Returns false if a bounded wait gave up (the error word is set and
// no copy is left in flight).  Threads past the tile's (TY + 2) x QW quads
// only take part in the barriers.
template <typename T, bool OR, bool GATHER, typename Job>
__device__ bool march_pass(const Job &a, const PhiloxKeys &K, unsigned char *smem, int *err,
                           int &gbase, double &sq, double &sp) {
  constexpr int R = 1;  // rows per thread
  const PassLayout lay = pass_layout(a.TY(), a.W(), (int)sizeof(T), OR);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 64);
  unsigned char *ring = smem + kHeaderBytes;
  T *newbuf = reinterpret_cast<T *>(ring + kPassStages * lay.slot_bytes);
  const int gb = gbase;
  auto c1_slot = [&](int j) {
    return reinterpret_cast<T *>(ring + ((gb + j) % kPassStages) * lay.slot_bytes);
  };
  auto c0_slot = [&](int j) {
    return reinterpret_cast<T *>(ring + ((gb + j) % kPassStages) * lay.slot_bytes +
                                 round_up_int(lay.c1_bytes, 128));
  };
  auto new_plane = [&](int s) {
    return reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(newbuf) + (s & 1) * lay.new_bytes);
  };

  const int W = a.W(), TY = a.TY();
  const int y0 = a.y0(), z0 = a.z0(), nz = a.nz();
  const int tid = threadIdx.x;
  // this thread: quad qx of row r0 (y = y0 - 1 + r0; rows 0 and TY + 1 are
  // the halo of stage 0)
  const int qx = tid % a.QW(), r0 = R * (tid / a.QW());
  const bool in_tile = r0 < TY + 2;
  bool live0[R], live1[R];
  int yk[R];
#pragma unroll
  for (int k = 0; k < R; ++k) {
    yk[k] = y0 - 1 + r0 + k;
    live0[k] = in_tile && yk[k] >= 0 && yk[k] < a.Ly() && qx < a.Wq();
    live1[k] = live0[k] && r0 + k >= 1 && r0 + k <= TY;
  }
  const int n_ring = nz + 4;  // colour-1 planes z0 - 2 .. z0 + nz + 1
  T *dst0 = a.dst();
  T *dst1 = dst0 + a.colour_elems();
  const uint32_t pass = a.pass();

  if (tid == 0) {
    prefetch_tensormap(a.tm_c1());
    if (OR) prefetch_tensormap(a.tm_c0());
  }
  // ring plane j: colour 1 at z0 - 2 + j; with it (j >= 2) colour 0 at z0 - 3 + j
  auto issue = [&](int j) {
    const uint32_t bar = smem_addr(&bars[(gb + j) % kPassStages]);
    const bool own = OR && j >= 2;
    mbar_arrive_expect_tx(bar, lay.c1_bytes + (own ? lay.c0_bytes : 0));
    tma_load_4d(smem_addr(c1_slot(j)), a.tm_c1(), 0, y0 - 2, z0 - 2 + j, a.map_c1(), bar);
    if (own) tma_load_4d(smem_addr(c0_slot(j)), a.tm_c0(), 0, y0 - 1, z0 - 3 + j, a.map_c0(), bar);
  };
  auto wait_plane = [&](int j) -> bool {
    return mbar_wait_bounded(smem_addr(&bars[(gb + j) % kPassStages]),
                             (uint32_t)(((gb + j) / kPassStages) & 1));
  };
  int issued = 0;
  if (tid == 0)
    for (; issued < min(kPassStages, n_ring); ++issued) issue(issued);
  // fused gather: this tile's charge range, and this thread's first entry,
  // loaded while the first planes arrive (used once the tile is written)
  uint32_t g_e = 0u, g_e1 = 0u, g_ent0 = 0u;
  double g_q0 = 0.0;
  if (GATHER) {
    g_e = a.g_off()[z0] + (uint32_t)tid;
    g_e1 = a.g_off()[z0 + nz];
    if (g_e < g_e1) {
      g_ent0 = a.g_ent()[g_e];
      g_q0 = a.g_q()[g_e];
    }
  }
  // lanes of the quad past x = Lx - 1 (kept at 0), for row parity 0 and 1
  uint32_t pad0 = 0u, pad1 = 0u;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (2 * (4 * qx + i) >= a.Lx()) pad0 |= 1u << i;
    if (2 * (4 * qx + i) + 1 >= a.Lx()) pad1 |= 1u << i;
  }
  const bool lo_ok = qx > 0, hi_ok = 4 * qx + 4 < W;
  const int row = r0 * W + 4 * qx;  // first row of this thread in a box starting at y0 - 1
  T *out0 = dst0 + (size_t)yk[0] * W + 4 * qx;
  T *out1 = dst1 + (size_t)yk[0] * W + 4 * qx;
  const size_t plane = (size_t)a.Ly() * W;

  // registers along z, per row: colour 1 old at p0 - 1, p0, p0 + 1; colour 0
  // new at p1 - 1, p1, p1 + 1 (p1 = p0 - 1)
  T am[R][4], ac[R][4], ap[R][4], nm[R][4], nc[R][4], np[R][4];
#pragma unroll
  for (int k = 0; k < R; ++k)
#pragma unroll
    for (int i = 0; i < 4; ++i) am[k][i] = ac[k][i] = ap[k][i] = nm[k][i] = nc[k][i] = np[k][i] = T(0);
  bool ok = wait_plane(0);
  if (ok && in_tile)
#pragma unroll
    for (int k = 0; k < R; ++k) ld_quad(c1_slot(0) + row + (k + 1) * W, am[k]);
  ok = ok && wait_plane(1);
  if (ok && in_tile)
#pragma unroll
    for (int k = 0; k < R; ++k) ld_quad(c1_slot(1) + row + (k + 1) * W, ac[k]);
  if (!ok) {
    atomicOr(err, kErrTimeout);
    *abort_flag = 1;
  }
  __syncthreads();
  bool aborted = *abort_flag != 0;
  int done = 1;  // ring planes 0 .. done waited for by every thread

  // One step s: stage 0 at p0 = z0 - 1 + s, then stage 1 at p0 - 1.  The
  // register triples rotate from step to step (A0 = plane - 1, A1 = plane,
  // A2 = plane + 1; A2 and N2 written here); the loop below calls it with the
  // names rotated, so no values are moved.  The y neighbours inside the
  // thread's rows come from its own registers, the outer two from shared
  // memory.
  auto step = [&](int s, T(&A0)[R][4], T(&A1)[R][4], T(&A2)[R][4], T(&N0)[R][4],
                  T(&N1)[R][4], T(&N2)[R][4]) -> bool {
    const int j = s + 2;
    const int p0 = z0 - 1 + s;
    const bool got = wait_plane(j);
    T v0[R][4];
#pragma unroll
    for (int k = 0; k < R; ++k)
#pragma unroll
      for (int i = 0; i < 4; ++i) v0[k][i] = T(0);
    if (got) {
      const T *C1 = c1_slot(j) + row;
#pragma unroll
      for (int k = 0; k < R; ++k) {
        if (in_tile) {
          ld_quad(C1 + (k + 1) * W, A2[k]);
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i) A2[k][i] = T(0);
        }
      }
      if (in_tile && p0 >= 0 && p0 < a.Lz()) {
        const T *Pz = c1_slot(j - 1) + row;  // colour 1 old, plane p0; row r0 + k at + (k + 1) W
        T lo[4], hi[4];
        ld_quad(Pz, lo);                // row r0 - 1
        ld_quad(Pz + (R + 1) * W, hi);  // row r0 + R
#pragma unroll
        for (int k = 0; k < R; ++k) {
          if (!live0[k]) continue;
          const T *ym = k == 0 ? lo : A1[k - 1];
          const T *yp = k == R - 1 ? hi : A1[k + 1];
          T xs[4], S[4];
          const int par = (yk[k] + p0) & 1;
          const bool odd = par != 0;
          const T e = (odd ? hi_ok : lo_ok) ? Pz[(k + 1) * W + (odd ? 4 : -1)] : T(0);
          x_neighbours(odd, e, A1[k], xs);
#pragma unroll
          for (int i = 0; i < 4; ++i)
            S[i] = ((A0[k][i] + A2[k][i]) + (ym[i] + yp[i])) + (A1[k][i] + xs[i]);
          if (!OR) {
            const uint32_t quad = ((uint32_t)p0 * (uint32_t)a.Ly() + (uint32_t)yk[k]) *
                                      (uint32_t)a.Wq() + (uint32_t)qx;
            const uint4 w = philox4x32_10(make_uint4(quad, pass, a.rng_id(), 0u), K);
            v0[k][0] = fma(S[0], Coef<T>::sixth, Noise<T>::of(w.x));
            v0[k][1] = fma(S[1], Coef<T>::sixth, Noise<T>::of(w.y));
            v0[k][2] = fma(S[2], Coef<T>::sixth, Noise<T>::of(w.z));
            v0[k][3] = fma(S[3], Coef<T>::sixth, Noise<T>::of(w.w));
          } else {
            T old[4];
            ld_quad(c0_slot(j) + row + k * W, old);
#pragma unroll
            for (int i = 0; i < 4; ++i) v0[k][i] = fma(S[i], Coef<T>::third, -old[i]);
          }
          const uint32_t pm = par ? pad1 : pad0;
          if (pm) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
              if ((pm >> i) & 1u) v0[k][i] = T(0);
          }
          if (live1[k] && p0 >= z0 && p0 < z0 + nz)
            st_quad(out0 + (size_t)p0 * plane + (size_t)k * W, v0[k]);
        }
      }
      if (in_tile)
#pragma unroll
        for (int k = 0; k < R; ++k) st_quad(new_plane(s) + row + k * W, v0[k]);
    } else {
      atomicOr(err, kErrTimeout);
      *abort_flag = 1;
    }
#pragma unroll
    for (int k = 0; k < R; ++k)
#pragma unroll
      for (int i = 0; i < 4; ++i) N2[k][i] = v0[k][i];
    // ---- stage 1: colour 1 at plane p1 = p0 - 1 on this tile's rows.  It
    // reads the new colour-0 rows of plane p1 (written in the previous step,
    // before the barrier that ends it) and this thread's own registers, none
    // of what stage 0 of this step wrote to shared memory, so no barrier
    // between the stages.
    const int p1 = p0 - 1;
    if (s >= 2 && (live1[0] || live1[R - 1])) {
      const T *N = new_plane(s - 1) + row;  // colour 0 new, plane p1
      T lo[4], hi[4];
      if (live1[0]) ld_quad(N - W, lo);      // row r0 - 1 (r0 >= 1 here)
      if (live1[R - 1]) ld_quad(N + R * W, hi);  // row r0 + R (<= TY + 1 here)
#pragma unroll
      for (int k = 0; k < R; ++k) {
        if (!live1[k]) continue;
        const T *ym = k == 0 ? lo : N1[k - 1];
        const T *yp = k == R - 1 ? hi : N1[k + 1];
        T xs[4], S[4], v[4];
        const int par = (1 + yk[k] + p1) & 1;
        const bool odd = par != 0;
        const T e = (odd ? hi_ok : lo_ok) ? N[k * W + (odd ? 4 : -1)] : T(0);
        x_neighbours(odd, e, N1[k], xs);
#pragma unroll
        for (int i = 0; i < 4; ++i)
          S[i] = ((N0[k][i] + N2[k][i]) + (ym[i] + yp[i])) + (N1[k][i] + xs[i]);
        if (!OR) {
          const uint32_t quad = ((uint32_t)p1 * (uint32_t)a.Ly() + (uint32_t)yk[k]) *
                                    (uint32_t)a.Wq() + (uint32_t)qx;
          const uint4 w = philox4x32_10(make_uint4(quad, pass, a.rng_id(), 1u), K);
          v[0] = fma(S[0], Coef<T>::sixth, Noise<T>::of(w.x));
          v[1] = fma(S[1], Coef<T>::sixth, Noise<T>::of(w.y));
          v[2] = fma(S[2], Coef<T>::sixth, Noise<T>::of(w.z));
          v[3] = fma(S[3], Coef<T>::sixth, Noise<T>::of(w.w));
        } else {
          // colour 1's own old value at plane p1 = p0 - 1 is A0
#pragma unroll
          for (int i = 0; i < 4; ++i) v[i] = fma(S[i], Coef<T>::third, -A0[k][i]);
        }
        const uint32_t pm = par ? pad1 : pad0;
        if (pm) {
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if ((pm >> i) & 1u) v[i] = T(0);
        }
        st_quad(out1 + (size_t)p1 * plane + (size_t)k * W, v);
      }
    }
    // new plane s visible to the next step's stage 1; new plane s - 1 and
    // ring plane s free for reuse
    __syncthreads();
    if (*abort_flag) return false;
    done = j;
    if (tid == 0 && issued < n_ring) issue(issued++);
    return true;
  };

  const int n_steps = nz + 2;
  for (int s = 0; s < n_steps && !aborted; s += 3) {
    if (!step(s, am, ac, ap, nm, nc, np)) { aborted = true; break; }
    if (s + 1 >= n_steps) break;
    if (!step(s + 1, ac, ap, am, nc, np, nm)) { aborted = true; break; }
    if (s + 2 >= n_steps) break;
    if (!step(s + 2, ap, am, ac, np, nm, nc)) { aborted = true; break; }
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
      double tq = 0.0, tp = 0.0;
      for (uint32_t e = g_e; e < g_e1; e += blockDim.x) {
        const uint32_t ent = e == g_e ? g_ent0 : a.g_ent()[e];
        const double qe = e == g_e ? g_q0 : a.g_q()[e];
        const uint32_t at = ent & ~kGatherColourBit;
        const T val = (ent & kGatherColourBit) ? dst1[at] : dst0[at];
        const double t = qe * (double)val;
        tq += t;
        tp += t * t;
      }
      sq += tq;
      sp += tp;
    }
  }
  return !aborted;
}

}  // namespace tile
}  // namespace coulps
