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

// The tile of one CTA: y tile blockIdx.x, z slab blockIdx.y, chain chain0 +
// blockIdx.z * chain_stride; every quantity read from the kernel's
// parameters where the march uses it.
template <typename T, bool OR>
struct GridPass {
  const CUtensorMap &m1, &m0;
  const PassArgs &p;
  __device__ __forceinline__ int chain() const { return p.chain0 + (int)blockIdx.z * p.chain_stride; }
  __device__ __forceinline__ const CUtensorMap *tm_c1() const { return &m1; }
  __device__ __forceinline__ const CUtensorMap *tm_c0() const { return &m0; }
  __device__ __forceinline__ int map_c1() const { return 2 * chain() + 1; }
  __device__ __forceinline__ int map_c0() const { return 2 * chain(); }
  __device__ __forceinline__ T *dst() const {
    return reinterpret_cast<T *>(p.dst) + (size_t)chain() * p.chain_elems;
  }
  __device__ __forceinline__ size_t colour_elems() const { return p.colour_elems; }
  __device__ __forceinline__ int Lx() const { return p.Lx; }
  __device__ __forceinline__ int Ly() const { return p.Ly; }
  __device__ __forceinline__ int Lz() const { return p.Lz; }
  __device__ __forceinline__ int W() const { return p.W; }
  __device__ __forceinline__ int Wq() const { return p.Wq; }
  __device__ __forceinline__ int QW() const { return p.QW; }
  __device__ __forceinline__ int TY() const { return p.TY; }
  __device__ __forceinline__ int y0() const { return (int)blockIdx.x * p.TY; }
  __device__ __forceinline__ int z0() const { return (int)blockIdx.y * p.DZ; }
  __device__ __forceinline__ int nz() const { return min(p.DZ, p.Lz - z0()); }
  __device__ __forceinline__ uint32_t rng_id() const { return (uint32_t)chain(); }
  __device__ __forceinline__ uint32_t pass() const { return OR ? 0u : (*p.pass_ptr + p.pass_off); }
  __device__ __forceinline__ const uint32_t *g_off() const {
    return p.g_off + (size_t)blockIdx.x * p.Lz;
  }
  __device__ __forceinline__ const uint32_t *g_ent() const { return p.g_ent; }
  __device__ __forceinline__ const double *g_q() const { return p.g_q; }
};

template <typename T, bool OR, bool GATHER>
__global__ void __launch_bounds__(512)
    pass_kernel(const __grid_constant__ CUtensorMap tm_c1, const __grid_constant__ CUtensorMap tm_c0,
                const PassArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = align_smem128(smem_raw);
  const GridPass<T, OR> j{tm_c1, tm_c0, a};
  double sq = 0.0, sp = 0.0;
  int gbase = 0;
  pass_ring_init(smem);
  march_pass<T, OR, GATHER>(j, *reinterpret_cast<const PhiloxKeys *>(a.round_keys), smem, a.err,
                            gbase, sq, sp);
  if (GATHER) {
    const size_t cta = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    block_partials(sq, sp, smem,
                   a.g_partials + 2 * ((size_t)j.chain() * gridDim.x * gridDim.y + cta));
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
