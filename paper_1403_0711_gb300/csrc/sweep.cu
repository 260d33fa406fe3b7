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
// the other colour's planes z-1, z, z+1; these are streamed through a 4-slot
// shared-memory ring by TMA (one 4D box = TY+2 rows x W elements, the rows
// y0-1 .. y0+TY of one plane), three planes ahead of use, each slot guarded
// by an mbarrier.  Out-of-range rows and planes (y = -1, y = Ly, z = -1,
// z = Lz) arrive zero-filled from the TMA unit, which is exactly the
// Dirichlet ghost layer.  Each thread owns one quad of four same-colour sites
// of one row and keeps the quad's values of planes z-1 and z in registers, so
// per plane it reads from shared memory the quad of plane z+1, the quads of
// rows y-1 and y+1 and one scalar for the x neighbour that lies in the next
// or previous quad.  Over-relaxation also streams its own colour's plane
// (TY rows) through the same ring.  Results go straight to global memory as
// 16-byte (FP32) or 2 x 16-byte (FP64) stores.
//
// DRAM traffic per updated site: one read of the other colour, one write
// (heatbath, 8 B in FP32) plus one read of the old value (over-relaxation,
// 12 B).  The halo rows/planes shared with neighbouring tiles are re-read
// from L2.
#include "device_common.cuh"
#include "internal.h"

namespace coulps {
namespace {

constexpr int kStages = 4;

__host__ __device__ inline int round_up_int(int v, int m) { return (v + m - 1) / m * m; }

struct SmemLayout {
  int halo_bytes;  // exact TMA box bytes of the other colour: (TY + 2) * W * es
  int own_bytes;   // exact TMA box bytes of the own colour: TY * W * es (OR only)
  int slot_bytes;  // one ring slot, both boxes, each rounded to 128 bytes
  int total;       // header (barriers, flags) + ring, without alignment slack
};

__host__ __device__ inline SmemLayout smem_layout(int TY, int W, int es, bool orx) {
  SmemLayout L;
  L.halo_bytes = (TY + 2) * W * es;
  L.own_bytes = orx ? TY * W * es : 0;
  L.slot_bytes = round_up_int(L.halo_bytes, 128) + round_up_int(L.own_bytes, 128);
  L.total = 128 + kStages * L.slot_bytes;
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

template <typename T> struct Coef;
template <> struct Coef<float> {
  static constexpr float sixth = 0.166666666666666666667f;
  static constexpr float third = 0.333333333333333333333f;
};
template <> struct Coef<double> {
  static constexpr double sixth = 0.166666666666666666667;
  static constexpr double third = 0.333333333333333333333;
};

template <typename T, bool OR>
__global__ void __launch_bounds__(1024)
    halfsweep_kernel(const __grid_constant__ CUtensorMap tm_halo,
                     const __grid_constant__ CUtensorMap tm_own, const SweepArgs a) {
  extern __shared__ unsigned char smem_raw[];
  // 128-byte aligned base (the launch reserves 128 bytes of slack).
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  const SmemLayout lay = smem_layout(a.TY, a.W, (int)sizeof(T), OR);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem);        // kStages barriers
  volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 64);
  unsigned char *ring = smem + 128;
  auto halo_slot = [&](int s) -> T * {
    return reinterpret_cast<T *>(ring + s * lay.slot_bytes);
  };
  auto own_slot = [&](int s) -> T * {
    return reinterpret_cast<T *>(ring + s * lay.slot_bytes + round_up_int(lay.halo_bytes, 128));
  };

  const int tid = threadIdx.x;
  const int W = a.W, TY = a.TY;
  const int qx = tid % a.QW, ty = tid / a.QW;
  const int y0 = blockIdx.x * TY, z0 = blockIdx.y * a.DZ, chain = blockIdx.z;
  const int nz = min(a.DZ, a.Lz - z0);
  const int n_planes = nz + 2;  // other-colour planes z0-1 .. z0+nz
  const int c = a.colour, oc = c ^ 1;
  const int y = y0 + ty;
  const bool live = (y < a.Ly) && (qx < a.Wq);

  if (tid == 0) {
    prefetch_tensormap(&tm_halo);
    if (OR) prefetch_tensormap(&tm_own);
    for (int s = 0; s < kStages; ++s) mbar_init(smem_addr(&bars[s]), 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();

  // Plane k of the ring is other-colour plane z0 - 1 + k, in slot k % kStages,
  // completed in that slot's phase k / kStages.
  auto issue = [&](int k) {
    const int s = k % kStages;
    const uint32_t bar = smem_addr(&bars[s]);
    const bool own = OR && k >= 1 && k <= nz;
    mbar_arrive_expect_tx(bar, lay.halo_bytes + (own ? lay.own_bytes : 0));
    tma_load_4d(smem_addr(halo_slot(s)), &tm_halo, 0, y0 - 1, z0 - 1 + k, 2 * chain + oc, bar);
    if (own) tma_load_4d(smem_addr(own_slot(s)), &tm_own, 0, y0, z0 - 1 + k, 2 * chain + c, bar);
  };
  auto wait_plane = [&](int k) -> bool {
    return mbar_wait_bounded(smem_addr(&bars[k % kStages]), (uint32_t)((k / kStages) & 1));
  };

  int issued = 0;  // meaningful in thread 0 only
  if (tid == 0)
    for (; issued < min(kStages, n_planes); ++issued) issue(issued);

  const uint32_t pass = OR ? 0u : (*a.pass_ptr + a.pass_off);
  T *out_base = reinterpret_cast<T *>(a.field) + (size_t)chain * a.chain_elems +
                (size_t)c * a.colour_elems;

  T cm[4], c0[4], cp[4];
  bool ok = wait_plane(0);
  if (ok) ld_quad(halo_slot(0) + (ty + 1) * W + 4 * qx, cm);
  ok = ok && wait_plane(1);
  if (ok) ld_quad(halo_slot(1) + (ty + 1) * W + 4 * qx, c0);
  if (!ok) {
    atomicOr(a.err, kErrTimeout);
    *abort_flag = 1;
  }
  __syncthreads();
  bool aborted = *abort_flag != 0;
  int done = 1;  // planes 0..done completed for every thread
  if (!aborted) {
    if (tid == 0 && issued < n_planes) issue(issued++);
    for (int k = 1; k <= nz; ++k) {
      if (wait_plane(k + 1)) {
        const int z = z0 + k - 1;
        const T *Pz = halo_slot(k % kStages);
        ld_quad(halo_slot((k + 1) % kStages) + (ty + 1) * W + 4 * qx, cp);
        if (live) {
          T ym[4], yp[4], xs[4], S[4], v[4];
          ld_quad(Pz + ty * W + 4 * qx, ym);
          ld_quad(Pz + (ty + 2) * W + 4 * qx, yp);
          const int par = (c + y + z) & 1;  // row holds x = 2h + par
          if (par == 0) {
            // x - 1 of h lies at h - 1 in the other colour, x + 1 at h
            xs[0] = qx > 0 ? Pz[(ty + 1) * W + 4 * qx - 1] : T(0);
            xs[1] = c0[0]; xs[2] = c0[1]; xs[3] = c0[2];
          } else {
            // x - 1 of h lies at h, x + 1 at h + 1
            xs[0] = c0[1]; xs[1] = c0[2]; xs[2] = c0[3];
            xs[3] = (4 * qx + 4 < W) ? Pz[(ty + 1) * W + 4 * qx + 4] : T(0);
          }
#pragma unroll
          for (int i = 0; i < 4; ++i) S[i] = ((cm[i] + cp[i]) + (ym[i] + yp[i])) + (c0[i] + xs[i]);
          if (!OR) {
            const uint32_t quad = ((uint32_t)z * (uint32_t)a.Ly + (uint32_t)y) * (uint32_t)a.Wq +
                                  (uint32_t)qx;
            const uint4 w = philox4x32_10(make_uint4(quad, pass, (uint32_t)chain, (uint32_t)c),
                                          a.seed_lo, a.seed_hi);
            v[0] = fma(S[0], Coef<T>::sixth, Noise<T>::of(w.x));
            v[1] = fma(S[1], Coef<T>::sixth, Noise<T>::of(w.y));
            v[2] = fma(S[2], Coef<T>::sixth, Noise<T>::of(w.z));
            v[3] = fma(S[3], Coef<T>::sixth, Noise<T>::of(w.w));
          } else {
            T old[4];
            ld_quad(own_slot(k % kStages) + ty * W + 4 * qx, old);
#pragma unroll
            for (int i = 0; i < 4; ++i) v[i] = fma(S[i], Coef<T>::third, -old[i]);
          }
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (2 * (4 * qx + i) + par >= a.Lx) v[i] = T(0);  // keep the row padding at 0
          st_quad(out_base + ((size_t)z * a.Ly + y) * W + 4 * qx, v);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          cm[i] = c0[i];
          c0[i] = cp[i];
        }
      } else {
        atomicOr(a.err, kErrTimeout);
        *abort_flag = 1;
      }
      __syncthreads();
      if (*abort_flag) {
        aborted = true;
        break;
      }
      done = k + 1;
      // plane k is no longer read: refill its slot with plane k + kStages
      if (tid == 0 && issued < n_planes) issue(issued++);
    }
  }
  if (aborted && tid == 0) {
    // Leave no copy in flight into this CTA's shared memory.
    for (int k = done + 1; k < issued; ++k)
      if (!wait_plane(k)) break;
  }
}

__global__ void advance_pass_kernel(uint32_t *pass, uint32_t n) { *pass += n; }

template <typename T, bool OR>
cudaError_t launch_t(const Geometry &g, const Tile &t, const CUtensorMap &tm_halo,
                     const CUtensorMap &tm_own, const SweepArgs &a, cudaStream_t s) {
  const SmemLayout lay = smem_layout(t.ty, g.W, (int)sizeof(T), OR);
  const size_t smem = (size_t)lay.total + 128;
  auto kfn = halfsweep_kernel<T, OR>;
  static int configured_bytes = 0;  // per instantiation
  if ((int)smem > configured_bytes) {
    cudaError_t e =
        cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured_bytes = (int)smem;
  }
  dim3 grid((g.Ly + t.ty - 1) / t.ty, (g.Lz + t.dz - 1) / t.dz, g.n_chains);
  dim3 block((g.W / 4) * t.ty);
  kfn<<<grid, block, smem, s>>>(tm_halo, tm_own, a);
  return cudaGetLastError();
}

}  // namespace

size_t halfsweep_smem_bytes(const Geometry &g, const Tile &t, bool overrelax) {
  return (size_t)smem_layout(t.ty, g.W, g.es, overrelax).total + 128;
}

cudaError_t launch_halfsweep(const Geometry &g, const Tile &t, const CUtensorMap &tm_halo,
                             const CUtensorMap &tm_own, const SweepArgs &a, bool overrelax,
                             cudaStream_t s) {
  if (g.precision == COULPS_F32)
    return overrelax ? launch_t<float, true>(g, t, tm_halo, tm_own, a, s)
                     : launch_t<float, false>(g, t, tm_halo, tm_own, a, s);
  return overrelax ? launch_t<double, true>(g, t, tm_halo, tm_own, a, s)
                   : launch_t<double, false>(g, t, tm_halo, tm_own, a, s);
}

cudaError_t launch_advance_pass(uint32_t *pass, uint32_t n, cudaStream_t s) {
  advance_pass_kernel<<<1, 1, 0, s>>>(pass, n);
  return cudaGetLastError();
}

}  // namespace coulps
