// Pass pair: two consecutive passes A and B (each a red then a black
// half-sweep, heatbath Eq. (phi) or over-relaxation) in one z-march from a
// source copy of the field to a destination copy.  Each site is read once
// and written once for both passes: 4 bytes per site and pass in FP32,
// against 8 for a fused single pass (pass_fused.cu) and 12 / 8 for the
// half-sweeps.
//
// Four stages run one plane apart inside one CTA (TY rows of y, slab
// [z0, z0 + nz) of z, one chain).  At step s the front plane is
// f = z0 - 3 + s and
//   stage 0: colour 0 of pass A at plane f,     rows y0 - 3 .. y0 + TY + 2
//   stage 1: colour 1 of pass A at plane f - 1, rows y0 - 2 .. y0 + TY + 1
//   stage 2: colour 0 of pass B at plane f - 2, rows y0 - 1 .. y0 + TY
//   stage 3: colour 1 of pass B at plane f - 3, rows y0     .. y0 + TY - 1
// Stage k + 1 needs stage k's values on planes q - 1 .. q + 1 of its own
// quad (registers; plane q + 1 was made earlier in the same step) and on rows
// y +- 1 and the x neighbour of plane q (made in the previous step, read from
// a 2-plane shared buffer per stage).  An over-relaxation stage also needs
// the site's value before its pass: stage k - 2's value of the same plane
// (registers) or, for pass A, the source copy.  The halo rows of stages 0..2
// (3, 2, 1 rows each side) and the halo planes at the slab ends are computed
// by both neighbouring CTAs from identical inputs with identical Philox
// counters, so they agree bit for bit; only the tile's own rows and planes of
// pass B are written.  Stage k works at plane f - k, so its first needed
// plane z0 - 3 + k is reached at step 2k; earlier steps skip it.
//
// Inputs: colour 1 of the source at planes f - 1 .. f + 1 (rows y0 - 4 ..
// y0 + TY + 3) and, when pass A is over-relaxation, colour 0 at plane f
// (rows y0 - 3 .. y0 + TY + 2), by TMA through an 8-slot ring, zero-filled
// outside the box (the phi = 0 ghosts).  Each thread owns one quad of one
// row for all four stages and keeps, per stage, the quad's three planes in
// registers (rotated by unrolling the step three times).  One CTA barrier
// per step.
//
// The per-site arithmetic is that of the half-sweep kernels (same sums in
// the same order, same fma, the same deviate per Philox word, two sites per
// packed FP32 instruction with per-lane round-to-nearest), so a pass pair
// gives bitwise the field of its four half-sweeps.
//
// With a gather (the last kernel of a measured compound sweep) every CTA
// adds up Q = sum q phi and P = sum (q phi)^2 (Eq. (nsum2)) over the charges
// of its own rows and planes once they are written, and leaves one FP64
// (Q, P) partial.
#include "device_common.cuh"
#include "internal.h"
#include "pair_march.cuh"
#include "tile_march.cuh"

namespace coulps {
namespace {

using namespace tile;

// The tile of one CTA: y tile blockIdx.x, z slab blockIdx.y, chain chain0 +
// blockIdx.z * chain_stride; every quantity read from the kernel's
// parameters where the march uses it (as GridPass in pass_fused.cu).
template <typename T, bool A_OR, bool B_OR>
struct GridPair {
  static constexpr bool kIdleWarps = false;  // the block is the tile's rows, rounded to warps
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
  __device__ __forceinline__ uint32_t pass() const {
    return (A_OR && B_OR) ? 0u : (*p.pass_ptr + p.pass_off);
  }
  __device__ __forceinline__ const uint32_t *g_off() const {
    return p.g_off + (size_t)blockIdx.x * p.Lz;
  }
  __device__ __forceinline__ const uint32_t *g_ent() const { return p.g_ent; }
  __device__ __forceinline__ const double *g_q() const { return p.g_q; }
};

template <typename T, bool A_OR, bool B_OR, bool GATHER>
__global__ void __launch_bounds__(sizeof(T) == 4 ? kPairMaxThreads32 : kPairMaxThreads64, 1)
    pair_kernel(const __grid_constant__ CUtensorMap tm_c1, const __grid_constant__ CUtensorMap tm_c0,
                const PassArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = align_smem128(smem_raw);
  const GridPair<T, A_OR, B_OR> j{tm_c1, tm_c0, a};
  double sq = 0.0, sp = 0.0;
  int gbase = 0;
  pair_ring_init(smem);
  march_pair<T, A_OR, B_OR, GATHER>(j, *reinterpret_cast<const PhiloxKeys *>(a.round_keys), smem,
                                    a.err, gbase, sq, sp);
  if (GATHER) {
    const size_t cta = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    block_partials(sq, sp, smem,
                   a.g_partials + 2 * ((size_t)j.chain() * gridDim.x * gridDim.y + cta));
  }
}

template <typename T, bool A_OR, bool B_OR, bool GATHER>
cudaError_t launch_pt(const Geometry &g, const Tile &t, const CUtensorMap &tm_c1,
                      const CUtensorMap &tm_c0, const PassArgs &a, cudaStream_t s) {
  const PairLayout lay = pair_layout(t.ty, g.W, (int)sizeof(T), A_OR);
  const size_t smem = (size_t)lay.total + 128;
  auto kfn = pair_kernel<T, A_OR, B_OR, GATHER>;
  static int configured_bytes = 0;  // per instantiation
  if ((int)smem > configured_bytes) {
    cudaError_t e =
        cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured_bytes = (int)smem;
  }
  dim3 grid((g.Ly + t.ty - 1) / t.ty, (g.Lz + t.dz - 1) / t.dz,
            launch_chains(g.n_chains, a.chain0, a.chain_stride));
  kfn<<<grid, dim3(pair_threads(g, t)), smem, s>>>(tm_c1, tm_c0, a);
  return cudaGetLastError();
}

template <typename T, bool GATHER>
cudaError_t launch_kinds(const Geometry &g, const Tile &t, const CUtensorMap &tm_c1,
                         const CUtensorMap &tm_c0, const PassArgs &a, bool a_or, bool b_or,
                         cudaStream_t s) {
  if (a_or)
    return b_or ? launch_pt<T, true, true, GATHER>(g, t, tm_c1, tm_c0, a, s)
                : launch_pt<T, true, false, GATHER>(g, t, tm_c1, tm_c0, a, s);
  return b_or ? launch_pt<T, false, true, GATHER>(g, t, tm_c1, tm_c0, a, s)
              : launch_pt<T, false, false, GATHER>(g, t, tm_c1, tm_c0, a, s);
}

}  // namespace

int pair_threads(const Geometry &g, const Tile &t) {
  const int n = (g.W / 4) * (t.ty + 6);
  return (n + 31) / 32 * 32;
}

size_t pair_smem_bytes(const Geometry &g, const Tile &t, bool a_or) {
  return (size_t)pair_layout(t.ty, g.W, g.es, a_or).total + 128;
}

cudaError_t launch_pair(const Geometry &g, const Tile &t, const CUtensorMap &tm_c1,
                        const CUtensorMap &tm_c0, const PassArgs &a, bool a_or, bool b_or,
                        cudaStream_t s) {
  const bool gather = a.g_partials != nullptr;
  if (g.precision == COULPS_F32)
    return gather ? launch_kinds<float, true>(g, t, tm_c1, tm_c0, a, a_or, b_or, s)
                  : launch_kinds<float, false>(g, t, tm_c1, tm_c0, a, a_or, b_or, s);
  return gather ? launch_kinds<double, true>(g, t, tm_c1, tm_c0, a, a_or, b_or, s)
                : launch_kinds<double, false>(g, t, tm_c1, tm_c0, a, a_or, b_or, s);
}

}  // namespace coulps
