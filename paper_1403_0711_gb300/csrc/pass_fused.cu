// Fused pass: both half-sweeps of one pass (colour 0, then colour 1 with the
// new colour-0 values) in a single z-march, from a source copy of the field
// to a destination copy.  Per pass each site is read once and written once
// (8 bytes per site in FP32) instead of 12: the colour-0 half-sweep reads
// colour 1 and its own old values, the colour-1 half-sweep would read the new
// colour 0 and its own old values again.
//
// Order of work inside one CTA (TY rows of y, slab [z0, z0 + nz) of z, one
// chain), step s = 0 .. nz + 1:
//   stage 0: colour 0 at plane p0 = z0 - 1 + s on rows y0 - 1 .. y0 + TY
//            (one halo row each side, recomputed by both neighbouring CTAs:
//            same inputs, same Philox counters, same values);
//   stage 1: colour 1 at plane p1 = p0 - 1 on rows y0 .. y0 + TY - 1.
// Colour 1's old planes p0 - 1 .. p0 + 1 (rows y0 - 2 .. y0 + TY + 1) and
// colour 0's old plane p0 (rows y0 - 1 .. y0 + TY) arrive by TMA in a
// kPassStages-slot ring.  Each thread owns one quad of one row for both
// stages and carries in registers the three planes of colour 1 (old) and of
// colour 0 (new) that its quad needs along z; the y +- 1 rows and the x
// neighbour come from shared memory (the ring, and a 2-plane buffer of the
// new colour-0 rows).  The march of one tile is march_pass (pass_march.cuh),
// which the many-system kernel (batch.cu) runs tile after tile.
// Ghost rows and planes (outside the box) hold 0 in both.
//
// Reading the source and writing a separate destination is what makes the
// halo rows safe: a neighbouring CTA still reads old colour-1 rows that this
// CTA has already updated.  The arithmetic per site is exactly that of the
// half-sweep kernel (same sums in the same order, same fma), so a pass gives
// bitwise the same field as its two half-sweeps.
//
// With a gather (the last kernel of a measured compound sweep) each CTA then
// adds up Q = sum q phi and P = sum (q phi)^2 (Eq. (nsum2)) over the charges
// of its own rows and planes, read back from dst, into one FP64 partial.
#include "device_common.cuh"
#include "internal.h"
#include "pass_march.cuh"
#include "tile_march.cuh"

namespace coulps {
namespace {

using namespace tile;

template <typename T, bool OR, bool GATHER>
__global__ void __launch_bounds__(512)
    pass_kernel(const __grid_constant__ CUtensorMap tm_c1, const __grid_constant__ CUtensorMap tm_c0,
                const PassArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = align_smem128(smem_raw);
  const int chain = a.chain0 + (int)blockIdx.z * a.chain_stride;
  PassJob<T> j;
  j.tm_c1 = &tm_c1;
  j.tm_c0 = &tm_c0;
  j.map_c1 = 2 * chain + 1;
  j.map_c0 = 2 * chain;
  j.dst0 = reinterpret_cast<T *>(a.dst) + (size_t)chain * a.chain_elems;
  j.dst1 = j.dst0 + a.colour_elems;
  j.Lx = a.Lx; j.Ly = a.Ly; j.Lz = a.Lz; j.W = a.W; j.Wq = a.Wq; j.QW = a.QW; j.TY = a.TY;
  j.y0 = blockIdx.x * a.TY;
  j.z0 = blockIdx.y * a.DZ;
  j.nz = min(a.DZ, a.Lz - j.z0);
  j.rng_id = (uint32_t)chain;
  j.pass = OR ? 0u : (*a.pass_ptr + a.pass_off);
  j.g_off = GATHER ? a.g_off + (size_t)blockIdx.x * a.Lz : nullptr;
  j.g_ent = a.g_ent;
  j.g_q = a.g_q;
  double sq = 0.0, sp = 0.0;
  int gbase = 0;
  pass_ring_init(smem);
  march_pass<T, OR, GATHER>(j, *reinterpret_cast<const PhiloxKeys *>(a.round_keys), smem, a.err,
                            gbase, sq, sp);
  if (GATHER) {
    const size_t cta = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    block_partials(sq, sp, smem, a.g_partials + 2 * ((size_t)chain * gridDim.x * gridDim.y + cta));
  }
}

template <typename T, bool OR, bool GATHER>
cudaError_t launch_pt(const Geometry &g, const Tile &t, const CUtensorMap &tm_c1,
                      const CUtensorMap &tm_c0, const PassArgs &a, cudaStream_t s) {
  const PassLayout lay = pass_layout(t.ty, g.W, (int)sizeof(T), OR);
  const size_t smem = (size_t)lay.total + 128;
  auto kfn = pass_kernel<T, OR, GATHER>;
  static int configured_bytes = 0;  // per instantiation
  if ((int)smem > configured_bytes) {
    cudaError_t e =
        cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured_bytes = (int)smem;
  }
  dim3 grid((g.Ly + t.ty - 1) / t.ty, (g.Lz + t.dz - 1) / t.dz,
            launch_chains(g.n_chains, a.chain0, a.chain_stride));
  dim3 block(pass_threads(g, t));
  kfn<<<grid, block, smem, s>>>(tm_c1, tm_c0, a);
  return cudaGetLastError();
}

}  // namespace

int pass_threads(const Geometry &g, const Tile &t) {
  const int n = (g.W / 4) * (t.ty + 2);
  return (n + 31) / 32 * 32;
}

size_t pass_smem_bytes(const Geometry &g, const Tile &t, bool overrelax) {
  return (size_t)pass_layout(t.ty, g.W, g.es, overrelax).total + 128;
}

cudaError_t launch_pass(const Geometry &g, const Tile &t, const CUtensorMap &tm_c1,
                        const CUtensorMap &tm_c0, const PassArgs &a, bool overrelax,
                        cudaStream_t s) {
  const bool gather = a.g_partials != nullptr;
  if (g.precision == COULPS_F32) {
    if (overrelax)
      return gather ? launch_pt<float, true, true>(g, t, tm_c1, tm_c0, a, s)
                    : launch_pt<float, true, false>(g, t, tm_c1, tm_c0, a, s);
    return gather ? launch_pt<float, false, true>(g, t, tm_c1, tm_c0, a, s)
                  : launch_pt<float, false, false>(g, t, tm_c1, tm_c0, a, s);
  }
  if (overrelax)
    return gather ? launch_pt<double, true, true>(g, t, tm_c1, tm_c0, a, s)
                  : launch_pt<double, true, false>(g, t, tm_c1, tm_c0, a, s);
  return gather ? launch_pt<double, false, true>(g, t, tm_c1, tm_c0, a, s)
                : launch_pt<double, false, false>(g, t, tm_c1, tm_c0, a, s);
}

}  // namespace coulps
