// Checkerboard half-sweep kernels: heatbath Eq. (phi) and over-relaxation.
//
// A half-sweep of colour c rewrites every site of colour c from the six
// neighbours, which all have the other colour, so all sites of one colour are
// independent (the red/black reading of the paper's sequential update).
//
//   heatbath:         phi_x = S_x / 6 - erfc^-1(2 r_x) / sqrt(3)
//   over-relaxation:  phi_x = S_x / 3 - phi_x
//
// S_x is the sum of the six neighbours with phi = 0 outside the box (the
// paper's open-boundary modification of Eq. (phi)).
//
// Work decomposition.  One CTA owns a tile of TY rows (all of x) of one
// chain and marches through DZ consecutive z planes.  For each plane it needs
// the other colour's planes z-1, z, z+1; these are streamed through a
// shared-memory ring by TMA (one 4D box = TY+2 rows x W elements, the rows
// y0-1 .. y0+TY of one plane; 8 slots, the CTA synchronising once every 4
// planes and then refilling the slots it has finished), each slot guarded
// by an mbarrier.  Out-of-range rows and planes (y = -1, y = Ly, z = -1,
// z = Lz) arrive zero-filled from the TMA unit, which is exactly the
// Dirichlet ghost layer.  Each thread owns one quad of four same-colour sites
// of one row and keeps the quad's values of planes z-1 and z in registers, so
// per plane it reads from shared memory the quad of plane z+1, the quads of
// rows y-1 and y+1 and one scalar for the x neighbour that lies in the next
// or previous quad (FP32 heatbath: two quads per thread).  Over-relaxation
// also streams its own colour's plane (TY rows) through the same ring.
// Results go straight to global memory as 16-byte (FP32) or 2 x 16-byte
// (FP64) stores.
//
// Fused gather.  On the last half-sweep of a measured compound sweep the
// kernel also forms the tile's share of Q = sum q_i phi(r_i) and
// P = sum (q_i phi(r_i))^2 (Eq. (nsum2)): once the tile is written it reads
// the values at the tile's charges back from L2 (one barrier per tile, none
// per plane), and each CTA writes one FP64 (Q, P) partial; finalize adds them
// in a fixed order.
//
// DRAM traffic per updated site: one read of the other colour, one write
// (heatbath, 8 B in FP32) plus one read of the old value (over-relaxation,
// 12 B).  The halo rows/planes shared with neighbouring tiles are re-read
// from L2.
#include "device_common.cuh"
#include "internal.h"
#include "tile_march.cuh"

namespace coulps {
namespace {

using namespace tile;

template <typename T, bool OR, bool GATHER, int V>
__global__ void __launch_bounds__(256)
    halfsweep_kernel(const __grid_constant__ CUtensorMap tm_halo,
                     const __grid_constant__ CUtensorMap tm_own, const SweepArgs a) {
  extern __shared__ unsigned char smem_raw[];
  // 128-byte aligned base (the launch reserves 128 bytes of slack).
  unsigned char *smem = align_smem128(smem_raw);
  const int chain = a.chain0 + (int)blockIdx.z * a.chain_stride;
  TileJob<T> j;
  j.tm_halo_ = &tm_halo;
  j.tm_own_ = &tm_own;
  j.colour_ = a.colour;
  j.map_other_ = 2 * chain + (a.colour ^ 1);
  j.map_own_ = 2 * chain + a.colour;
  j.out_ = reinterpret_cast<T *>(a.field) + (size_t)chain * a.chain_elems +
          (size_t)a.colour * a.colour_elems;
  j.Lx_ = a.Lx; j.Ly_ = a.Ly; j.Lz_ = a.Lz; j.W_ = a.W; j.Wq_ = a.Wq; j.QW_ = a.QW; j.TY_ = a.TY;
  j.y0_ = blockIdx.x * a.TY;
  j.z0_ = blockIdx.y * a.DZ;
  j.nz_ = min(a.DZ, a.Lz - j.z0_);
  j.rng_id_ = (uint32_t)chain;
  j.pass_ = OR ? 0u : (*a.pass_ptr + a.pass_off);
  if (GATHER) {
    j.g_off_ = a.g_off + (size_t)blockIdx.x * a.Lz;
    j.g_ent_ = a.g_ent;
    j.other_ = reinterpret_cast<const T *>(a.field) + (size_t)chain * a.chain_elems +
              (size_t)(a.colour ^ 1) * a.colour_elems;
    j.g_q_ = a.g_q;
  }
  double sq = 0.0, sp = 0.0;
  int gbase = 0;
  ring_init<kLatticeStages>(smem);
  march_tile<T, OR, GATHER, V, kLatticeStages, kLatticeGroup>(
      j, *reinterpret_cast<const PhiloxKeys *>(a.round_keys), smem,
                               a.err, gbase, sq, sp);
  if (GATHER) {
    const size_t cta = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    block_partials(sq, sp, smem,
                   a.g_partials + 2 * ((size_t)chain * gridDim.x * gridDim.y + cta));
  }
}

// Phase-shifted schedule: every CTA looks up its chain's group and runs that
// group's half-sweep kind; idle groups' CTAs return before touching anything.
template <typename T>
__global__ void __launch_bounds__(256)
    halfsweep_mixed_kernel(const __grid_constant__ CUtensorMap tm_halo,
                           const __grid_constant__ CUtensorMap tm_own, const MixedArgs m) {
  const SweepArgs &a = m.base;
  const int chain = a.chain0 + (int)blockIdx.z * a.chain_stride;
  const int grp = chain % m.groups;
  const int mode = m.mode[grp];
  if (mode == 0) return;
  const bool gather = m.gather[grp] != 0;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = align_smem128(smem_raw);
  TileJob<T> j;
  j.tm_halo_ = &tm_halo;
  j.tm_own_ = &tm_own;
  j.colour_ = a.colour;
  j.map_other_ = 2 * chain + (a.colour ^ 1);
  j.map_own_ = 2 * chain + a.colour;
  j.out_ = reinterpret_cast<T *>(a.field) + (size_t)chain * a.chain_elems +
          (size_t)a.colour * a.colour_elems;
  j.Lx_ = a.Lx; j.Ly_ = a.Ly; j.Lz_ = a.Lz; j.W_ = a.W; j.Wq_ = a.Wq; j.QW_ = a.QW; j.TY_ = a.TY;
  j.y0_ = blockIdx.x * a.TY;
  j.z0_ = blockIdx.y * a.DZ;
  j.nz_ = min(a.DZ, a.Lz - j.z0_);
  j.rng_id_ = (uint32_t)chain;
  j.pass_ = *a.pass_ptr + m.pass_delta[grp];
  j.g_off_ = a.g_off + (size_t)blockIdx.x * a.Lz;
  j.g_ent_ = a.g_ent;
  j.other_ = reinterpret_cast<const T *>(a.field) + (size_t)chain * a.chain_elems +
            (size_t)(a.colour ^ 1) * a.colour_elems;
  j.g_q_ = a.g_q;
  const PhiloxKeys &K = *reinterpret_cast<const PhiloxKeys *>(a.round_keys);
  double sq = 0.0, sp = 0.0;
  int gbase = 0;
  ring_init<kLatticeStages>(smem);
  constexpr int S = kLatticeStages, G = kLatticeGroup;
  if (mode == 1) {
    if (gather) march_tile<T, false, true, 1, S, G>(j, K, smem, a.err, gbase, sq, sp);
    else march_tile<T, false, false, 1, S, G>(j, K, smem, a.err, gbase, sq, sp);
  } else {
    if (gather) march_tile<T, true, true, 1, S, G>(j, K, smem, a.err, gbase, sq, sp);
    else march_tile<T, true, false, 1, S, G>(j, K, smem, a.err, gbase, sq, sp);
  }
  if (gather) {
    const size_t cta = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    block_partials(sq, sp, smem,
                   a.g_partials + 2 * ((size_t)chain * gridDim.x * gridDim.y + cta));
  }
}

template <typename T>
cudaError_t launch_mixed_t(const Geometry &g, const Tile &t, const CUtensorMap &tm_halo,
                           const CUtensorMap &tm_own, const MixedArgs &m, cudaStream_t s) {
  const SmemLayout lay = smem_layout(t.ty, g.W, (int)sizeof(T), true, kLatticeStages);
  const size_t smem = (size_t)lay.total + 128;
  auto kfn = halfsweep_mixed_kernel<T>;
  static int configured_bytes = 0;
  if ((int)smem > configured_bytes) {
    cudaError_t e =
        cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured_bytes = (int)smem;
  }
  dim3 grid((g.Ly + t.ty - 1) / t.ty, (g.Lz + t.dz - 1) / t.dz,
            launch_chains(g.n_chains, m.base.chain0, m.base.chain_stride));
  kfn<<<grid, dim3((g.W / 4) * t.ty), smem, s>>>(tm_halo, tm_own, m);
  return cudaGetLastError();
}

__global__ void advance_pass_kernel(uint32_t *pass, uint32_t n) { *pass += n; }

// The heatbath half-sweep in FP32 (issue-bound: Philox and the deviate) runs
// two quads per thread; the others one.
template <typename T, bool OR, bool GATHER>
constexpr int quads_per_thread() {
  return (sizeof(T) == 4 && !OR && !GATHER) ? 2 : 1;
}

template <typename T, bool OR, bool GATHER>
cudaError_t launch_t(const Geometry &g, const Tile &t, const CUtensorMap &tm_halo,
                     const CUtensorMap &tm_own, const SweepArgs &a, cudaStream_t s) {
  const SmemLayout lay = smem_layout(t.ty, g.W, (int)sizeof(T), OR, kLatticeStages);
  const size_t smem = (size_t)lay.total + 128;
  constexpr int V = quads_per_thread<T, OR, GATHER>();
  auto kfn = halfsweep_kernel<T, OR, GATHER, V>;
  static int configured_bytes = 0;  // per instantiation
  if ((int)smem > configured_bytes) {
    cudaError_t e =
        cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured_bytes = (int)smem;
  }
  dim3 grid((g.Ly + t.ty - 1) / t.ty, (g.Lz + t.dz - 1) / t.dz,
            launch_chains(g.n_chains, a.chain0, a.chain_stride));
  dim3 block((g.W / 4 + V - 1) / V * t.ty);
  kfn<<<grid, block, smem, s>>>(tm_halo, tm_own, a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_p(const Geometry &g, const Tile &t, const CUtensorMap &tm_halo,
                     const CUtensorMap &tm_own, const SweepArgs &a, bool overrelax,
                     cudaStream_t s) {
  const bool gather = a.g_partials != nullptr;
  if (overrelax)
    return gather ? launch_t<T, true, true>(g, t, tm_halo, tm_own, a, s)
                  : launch_t<T, true, false>(g, t, tm_halo, tm_own, a, s);
  return gather ? launch_t<T, false, true>(g, t, tm_halo, tm_own, a, s)
                : launch_t<T, false, false>(g, t, tm_halo, tm_own, a, s);
}

}  // namespace

size_t halfsweep_smem_bytes(const Geometry &g, const Tile &t, bool overrelax) {
  return (size_t)smem_layout(t.ty, g.W, g.es, overrelax, kLatticeStages).total + 128;
}

cudaError_t launch_halfsweep(const Geometry &g, const Tile &t, const CUtensorMap &tm_halo,
                             const CUtensorMap &tm_own, const SweepArgs &a, bool overrelax,
                             cudaStream_t s) {
  if (g.precision == COULPS_F32) return launch_p<float>(g, t, tm_halo, tm_own, a, overrelax, s);
  return launch_p<double>(g, t, tm_halo, tm_own, a, overrelax, s);
}

cudaError_t launch_halfsweep_mixed(const Geometry &g, const Tile &t, const CUtensorMap &tm_halo,
                                   const CUtensorMap &tm_own, const MixedArgs &m, cudaStream_t s) {
  if (m.groups < 1 || m.groups > kMaxGroups) return cudaErrorInvalidValue;
  if (g.precision == COULPS_F32) return launch_mixed_t<float>(g, t, tm_halo, tm_own, m, s);
  return launch_mixed_t<double>(g, t, tm_halo, tm_own, m, s);
}

cudaError_t launch_advance_pass(uint32_t *pass, uint32_t n, cudaStream_t s) {
  advance_pass_kernel<<<1, 1, 0, s>>>(pass, n);
  return cudaGetLastError();
}

namespace {
template <typename T>
__global__ void noise_kernel(const uint32_t *__restrict__ w, T *__restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = Noise<T>::of(w[i]);
}
}  // namespace

}  // namespace coulps

extern "C" int coulps_heatbath_noise(int precision, const uint32_t *w, void *out, int64_t n,
                                     void *stream) {
  using namespace coulps;
  if (n < 0 || (n > 0 && (!w || !out))) return COULPS_EINVAL;
  if (precision != COULPS_F32 && precision != COULPS_F64) return COULPS_EINVAL;
  if (n == 0) return COULPS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t want = (n + 255) / 256;
  const unsigned blocks = (unsigned)(want < 4096 ? want : 4096);
  if (precision == COULPS_F32)
    noise_kernel<float><<<blocks, 256, 0, s>>>(w, (float *)out, n);
  else
    noise_kernel<double><<<blocks, 256, 0, s>>>(w, (double *)out, n);
  return cudaGetLastError() == cudaSuccess ? COULPS_OK : COULPS_ECUDA;
}
