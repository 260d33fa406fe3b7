// Elementwise, reduction and weight-gradient kernels of the Stein control
// variate (the convolutions themselves are in cv_conv.cu).
//
//   pack:      lattice field (split colours, FP32) -> channels-last BF16 input
//              (phi, rho, 0 ...) and A phi (FP32), A = -Delta_lat with phi = 0
//              outside the box (A phi = dH_L/dphi).
//   activate:  a = tanh(h), s = tanh'(h) = 1 - a^2, both BF16.
//   stein_sum: per chain, sum_q sum_c s2[c, q] D[c, q] - sum_x g_x (A phi)_x,
//              D = conv(s1, K) over all sites (the divergence of g for every
//              site not on a face of the box, see below), g = channel 0 of the
//              last conv.
//   boundary:  per chain, the divergence correction of the face sites:
//              sum_q s2[c2, q] sum_{c1, e} dK_b(q)[c2, c1, e] s1[c1, q + e],
//              dK_b = K_b - K for the face class b(q) of q.
//   wgrad:     dW[co, ci, o] = sum_{b, p} dh[b, p, co] a[b, p + o, ci]
//              (zero outside), per-CTA partials then a fixed-order sum.
//
// Divergence of the net g (three 3x3x3 convs, tanh between them): with
// s1 = tanh'(h1), s2 = tanh'(h2),
//   sum_x dg_x/dphi_x = sum_q sum_c2 s2[c2, q] sum_{c1, e} K_b(q)[c2, c1, e] s1[c1, q+e],
//   K_b[c2, c1, e] = W2[c2, c1, e] sum_{f in F_b} W3[c2, f] W1[c1, phi, -(e + f)],
// where F_b holds the offsets f whose x = q - f lies inside the box; for q
// off the faces F_b is all 27 offsets and K_b = K.
#include <cstdint>

#include <cuda_bf16.h>

#include "device_common.cuh"
#include "internal.h"

namespace coulps {
namespace {

__device__ __forceinline__ float ld_field(const float *f, const Geometry &g, int chain, int x,
                                          int y, int z) {
  if (x < 0 || y < 0 || z < 0 || x >= g.Lx || y >= g.Ly || z >= g.Lz) return 0.f;
  const int c = (x + y + z) & 1;
  return f[(size_t)chain * g.chain_elems + (size_t)c * g.colour_elems +
           ((size_t)z * g.Ly + y) * g.W + (x >> 1)];
}

// Packs the sub-box [o, o + e) of every chain (the whole box when o = 0,
// e = L): rho is the full box's density.
__global__ void cv_pack_kernel(const float *__restrict__ field, Geometry g,
                               const float *__restrict__ rho, __nv_bfloat16 *__restrict__ act,
                               float *__restrict__ Aphi, int ox, int oy, int oz, int ex, int ey,
                               int ez) {
  const int64_t sites = (int64_t)ex * ey * ez;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int chain = blockIdx.y;
  if (i >= sites) return;
  const int x = ox + (int)(i % ex), y = oy + (int)((i / ex) % ey), z = oz + (int)(i / ((int64_t)ex * ey));
  const float p = ld_field(field, g, chain, x, y, z);
  const float S = ld_field(field, g, chain, x - 1, y, z) + ld_field(field, g, chain, x + 1, y, z) +
                  ld_field(field, g, chain, x, y - 1, z) + ld_field(field, g, chain, x, y + 1, z) +
                  ld_field(field, g, chain, x, y, z - 1) + ld_field(field, g, chain, x, y, z + 1);
  const int64_t o = (int64_t)chain * sites + i;
  Aphi[o] = 6.f * p - S;
  __align__(16) __nv_bfloat16 v[16];
  v[0] = __float2bfloat16_rn(p);
  v[1] = __float2bfloat16_rn(rho[((int64_t)z * g.Ly + y) * g.Lx + x]);
#pragma unroll
  for (int k = 2; k < 16; ++k) v[k] = __float2bfloat16_rn(0.f);
  uint4 *dst = reinterpret_cast<uint4 *>(act + o * 16);
  dst[0] = reinterpret_cast<const uint4 *>(v)[0];
  dst[1] = reinterpret_cast<const uint4 *>(v)[1];
}

__global__ void cv_activate_kernel(const float *__restrict__ h, __nv_bfloat16 *__restrict__ a,
                                   __nv_bfloat16 *__restrict__ s, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float t = tanhf(h[i]);
  a[i] = __float2bfloat16_rn(t);
  s[i] = __float2bfloat16_rn(1.f - t * t);
}

constexpr int kRedThreads = 256;

__device__ __forceinline__ void block_sum_to(double v, double *out) {
  __shared__ double red[kRedThreads / 32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = lane < kRedThreads / 32 ? red[lane] : 0.0;
    v = warp_sum(v);
    if (lane == 0) *out = v;
  }
}

// per (chain, block) partial of sum_q s2 . D - sum_x g_x (A phi)_x
__global__ void __launch_bounds__(kRedThreads)
    cv_stein_partial_kernel(const float *__restrict__ g16, const float *__restrict__ D,
                            const __nv_bfloat16 *__restrict__ s2, const float *__restrict__ Aphi,
                            int64_t sites, double *__restrict__ partials) {
  const int chain = blockIdx.y;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; i < sites;
       i += (int64_t)gridDim.x * kRedThreads) {
    const int64_t o = (int64_t)chain * sites + i;
    float d = 0.f;
#pragma unroll
    for (int c = 0; c < 16; ++c) d = fmaf(__bfloat162float(s2[o * 16 + c]), D[o * 16 + c], d);
    acc += (double)d - (double)g16[o * 16] * (double)Aphi[o];
  }
  block_sum_to(acc, partials + (size_t)chain * gridDim.x + blockIdx.x);
}

// face class of coordinate v in [0, n): 0 low face, 1 inside, 2 high face, 3 both (n == 1)
__device__ __forceinline__ int face_class(int v, int n) {
  return n == 1 ? 3 : (v == 0 ? 0 : (v == n - 1 ? 2 : 1));
}

// per (chain, block) partial of the face-site divergence correction
__global__ void __launch_bounds__(kRedThreads)
    cv_boundary_partial_kernel(const __nv_bfloat16 *__restrict__ s1,
                               const __nv_bfloat16 *__restrict__ s2, const float *__restrict__ dK,
                               int Lx, int Ly, int Lz, int64_t nface, double *__restrict__ partials) {
  // one thread per (face site, c2); face sites enumerated as all sites with
  // some coordinate on a face
  const int chain = blockIdx.y;
  const int64_t sites = (int64_t)Lx * Ly * Lz;
  double acc = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; t < nface * 16;
       t += (int64_t)gridDim.x * kRedThreads) {
    const int c2 = (int)(t & 15);
    int64_t k = t >> 4;  // k-th face site in (z, y, x) order
    // decode: walk planes z = 0 and z = Lz-1 fully, the other planes only on their rim
    int x, y, z;
    {
      const int64_t plane = (int64_t)Lx * Ly;
      const int64_t rim = (Ly <= 2 || Lx <= 2) ? plane : 2LL * Lx + 2LL * (Ly - 2);
      const int nfull = Lz == 1 ? 1 : 2;
      if (k < plane) {
        z = 0;
        x = (int)(k % Lx);
        y = (int)(k / Lx);
      } else if (nfull == 2 && k < 2 * plane) {
        z = Lz - 1;
        k -= plane;
        x = (int)(k % Lx);
        y = (int)(k / Lx);
      } else {
        k -= (int64_t)nfull * plane;
        z = 1 + (int)(k / rim);
        int64_t r = k % rim;
        if (rim == plane) {
          x = (int)(r % Lx);
          y = (int)(r / Lx);
        } else if (r < Lx) {
          y = 0;
          x = (int)r;
        } else if (r < 2LL * Lx) {
          y = Ly - 1;
          x = (int)(r - Lx);
        } else {
          r -= 2LL * Lx;
          y = 1 + (int)(r / 2);
          x = (r & 1) ? Lx - 1 : 0;
        }
      }
    }
    const int b = face_class(x, Lx) + 4 * face_class(y, Ly) + 16 * face_class(z, Lz);
    const float *dk = dK + ((size_t)b * 16 + c2) * 16 * 27;
    const int64_t q = ((int64_t)z * Ly + y) * Lx + x;
    float d = 0.f;
    for (int e = 0; e < 27; ++e) {
      const int ez = e / 9 - 1, ey = (e / 3) % 3 - 1, ex = e % 3 - 1;
      const int xx = x + ex, yy = y + ey, zz = z + ez;
      if (xx < 0 || yy < 0 || zz < 0 || xx >= Lx || yy >= Ly || zz >= Lz) continue;
      const __nv_bfloat16 *sp = s1 + ((int64_t)chain * sites + ((int64_t)zz * Ly + yy) * Lx + xx) * 16;
#pragma unroll
      for (int c1 = 0; c1 < 16; ++c1) d = fmaf(dk[c1 * 27 + e], __bfloat162float(sp[c1]), d);
    }
    acc += (double)__bfloat162float(s2[((int64_t)chain * sites + q) * 16 + c2]) * (double)d;
  }
  block_sum_to(acc, partials + (size_t)chain * gridDim.x + blockIdx.x);
}

__global__ void cv_sum_partials_kernel(const double *__restrict__ partials, int nblk, int nb,
                                       double *__restrict__ out, int accumulate) {
  const int chain = blockIdx.x * blockDim.x + threadIdx.x;
  if (chain >= nb) return;
  double s = 0.0;
  for (int k = 0; k < nblk; ++k) s += partials[(size_t)chain * nblk + k];
  out[chain] = accumulate ? out[chain] + s : s;
}

// Region Stein term: g is the net inside R = [lo, hi) (in E coordinates) and
// 0 outside.  For q within one site of R the divergence picks the offsets f
// with q - f inside R: per axis a mask over f in {-1, 0, 1} (bit f + 1),
// mapped to an index 0..5, class = ix + 6 iy + 36 iz.  K[class][c2][c1][e].
__device__ __forceinline__ int allowed_index(int q, int lo, int hi) {
  int m = 0;
#pragma unroll
  for (int f = -1; f <= 1; ++f)
    if (q - f >= lo && q - f < hi) m |= 1 << (f + 1);
  // masks 1, 2, 3, 4, 6, 7 -> 0..5; 0 (not next to R) -> -1
  switch (m) {
    case 1: return 0;
    case 2: return 1;
    case 3: return 2;
    case 4: return 3;
    case 6: return 4;
    case 7: return 5;
    default: return -1;
  }
}

__global__ void __launch_bounds__(kRedThreads)
    cv_region_partial_kernel(const float *__restrict__ g16, const __nv_bfloat16 *__restrict__ s1,
                             const __nv_bfloat16 *__restrict__ s2, const float *__restrict__ Aphi,
                             const float *__restrict__ Ktab, int ex, int ey, int ez, int lox,
                             int loy, int loz, int hix, int hiy, int hiz,
                             double *__restrict__ partials) {
  const int chain = blockIdx.y;
  const int64_t sites = (int64_t)ex * ey * ez;
  // divergence over q in (R + 1) within E, one thread per (q, c2)
  const int qx0 = max(lox - 1, 0), qy0 = max(loy - 1, 0), qz0 = max(loz - 1, 0);
  const int qx1 = min(hix + 1, ex), qy1 = min(hiy + 1, ey), qz1 = min(hiz + 1, ez);
  const int nqx = qx1 - qx0, nqy = qy1 - qy0, nqz = qz1 - qz0;
  const int64_t nq = (int64_t)nqx * nqy * nqz;
  double acc = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; t < nq * 16;
       t += (int64_t)gridDim.x * kRedThreads) {
    const int c2 = (int)(t & 15);
    const int64_t k = t >> 4;
    const int x = qx0 + (int)(k % nqx), y = qy0 + (int)((k / nqx) % nqy), z = qz0 + (int)(k / ((int64_t)nqx * nqy));
    const int ix = allowed_index(x, lox, hix), iy = allowed_index(y, loy, hiy),
              iz = allowed_index(z, loz, hiz);
    if (ix < 0 || iy < 0 || iz < 0) continue;
    const float *kk = Ktab + ((size_t)(ix + 6 * iy + 36 * iz) * 16 + c2) * 16 * 27;
    float d = 0.f;
    for (int e = 0; e < 27; ++e) {
      const int xx = x + e % 3 - 1, yy = y + (e / 3) % 3 - 1, zz = z + e / 9 - 1;
      if (xx < 0 || yy < 0 || zz < 0 || xx >= ex || yy >= ey || zz >= ez) continue;
      const __nv_bfloat16 *sp = s1 + ((int64_t)chain * sites + ((int64_t)zz * ey + yy) * ex + xx) * 16;
#pragma unroll
      for (int c1 = 0; c1 < 16; ++c1) d = fmaf(kk[c1 * 27 + e], __bfloat162float(sp[c1]), d);
    }
    acc += (double)__bfloat162float(s2[((int64_t)chain * sites + ((int64_t)z * ey + y) * ex + x) * 16 + c2]) *
           (double)d;
  }
  // minus sum over x in R of g_x (A phi)_x
  const int nrx = hix - lox, nry = hiy - loy, nrz = hiz - loz;
  const int64_t nr = (int64_t)nrx * nry * nrz;
  for (int64_t k = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; k < nr;
       k += (int64_t)gridDim.x * kRedThreads) {
    const int x = lox + (int)(k % nrx), y = loy + (int)((k / nrx) % nry), z = loz + (int)(k / ((int64_t)nrx * nry));
    const int64_t o = (int64_t)chain * sites + ((int64_t)z * ey + y) * ex + x;
    acc -= (double)g16[o * 16] * (double)Aphi[o];
  }
  block_sum_to(acc, partials + (size_t)chain * gridDim.x + blockIdx.x);
}

constexpr int kWgTile = 64;  // sites of one x row per shared-memory tile

// Per-CTA partial of dW[co][ci][o] over a contiguous range of x-row tiles
// (b, z, y, x0 .. x0+63).  Thread t = co * 16 + ci.  The tile of dh is loaded
// once; for each of the 27 offsets the matching tile of a (row (y+dy, z+dz),
// x shifted by dx, zero outside) is loaded and 64 FMAs accumulate per thread.
__global__ void __launch_bounds__(256)
    cv_wgrad_partial_kernel(const __nv_bfloat16 *__restrict__ a,
                            const __nv_bfloat16 *__restrict__ dh, int Lx, int Ly, int Lz,
                            int64_t ntiles, int64_t per_block, float *__restrict__ partials) {
  __shared__ float sd[kWgTile][17];
  __shared__ float sa[kWgTile + 2][17];
  const int t = threadIdx.x, co = t >> 4, ci = t & 15;
  const int xt = (Lx + kWgTile - 1) / kWgTile;
  const int64_t t0 = (int64_t)blockIdx.x * per_block;
  const int64_t t1 = t0 + per_block < ntiles ? t0 + per_block : ntiles;
  float acc[27];
#pragma unroll
  for (int o = 0; o < 27; ++o) acc[o] = 0.f;
  for (int64_t tile = t0; tile < t1; ++tile) {
    int64_t r = tile;
    const int x0 = (int)(r % xt) * kWgTile;
    r /= xt;
    const int y = (int)(r % Ly);
    r /= Ly;
    const int z = (int)(r % Lz);
    const int64_t b = r / Lz;
    __syncthreads();
    for (int k = t; k < kWgTile * 16; k += 256) {
      const int j = k >> 4, c = k & 15;
      const int x = x0 + j;
      sd[j][c] = x < Lx ? __bfloat162float(dh[((((b * Lz) + z) * Ly + y) * (int64_t)Lx + x) * 16 + c])
                        : 0.f;
    }
#pragma unroll
    for (int o9 = 0; o9 < 9; ++o9) {
      const int dz = o9 / 3 - 1, dy = o9 % 3 - 1;
      const int yy = y + dy, zz = z + dz;
      const bool row_in = yy >= 0 && yy < Ly && zz >= 0 && zz < Lz;
      __syncthreads();
      // a of row (yy, zz) at x0-1 .. x0+64, zero outside the box
      for (int k = t; k < (kWgTile + 2) * 16; k += 256) {
        const int j = k >> 4, c = k & 15;
        const int x = x0 - 1 + j;
        sa[j][c] = (row_in && x >= 0 && x < Lx)
                       ? __bfloat162float(a[((((b * Lz) + zz) * Ly + yy) * (int64_t)Lx + x) * 16 + c])
                       : 0.f;
      }
      __syncthreads();
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) {
        float s = 0.f;
#pragma unroll 16
        for (int j = 0; j < kWgTile; ++j) s = fmaf(sd[j][co], sa[j + dx][ci], s);
        acc[o9 * 3 + dx] += s;
      }
    }
  }
#pragma unroll
  for (int o = 0; o < 27; ++o) partials[((size_t)blockIdx.x * 27 + o) * 256 + t] = acc[o];
}

__global__ void cv_wgrad_reduce_kernel(const float *__restrict__ partials, int nblk,
                                       float *__restrict__ dW) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // o * 256 + t
  if (i >= 27 * 256) return;
  const int o = i / 256, t = i % 256;
  float s = 0.f;
  for (int b = 0; b < nblk; ++b) s += partials[((size_t)b * 27 + o) * 256 + t];
  dW[(size_t)t * 27 + o] = s;  // [co][ci][o]
}

}  // namespace
}  // namespace coulps

using namespace coulps;

// Layout and size rules are in include/coulps.h.
extern "C" {

int coulps_cv_activate(const float *h, void *a_bf16, void *s_bf16, int64_t n, void *stream) {
  if (!h || !a_bf16 || !s_bf16 || n < 0) return COULPS_EINVAL;
  if (n == 0) return COULPS_OK;
  cv_activate_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      h, (__nv_bfloat16 *)a_bf16, (__nv_bfloat16 *)s_bf16, n);
  return cudaGetLastError() == cudaSuccess ? COULPS_OK : COULPS_ECUDA;
}

int coulps_cv_stein_sum(const float *g16, const float *D, const void *s2_bf16, const float *Aphi,
                        const void *s1_bf16, const float *dK, int nb, int Lx, int Ly, int Lz,
                        double *scratch, int64_t scratch_doubles, double *out, void *stream) {
  if (!g16 || !D || !s2_bf16 || !Aphi || !s1_bf16 || !dK || !scratch || !out) return COULPS_EINVAL;
  if (nb < 1 || Lx < 1 || Ly < 1 || Lz < 1) return COULPS_EINVAL;
  const int nblk = 128;
  if (scratch_doubles < (int64_t)nb * nblk) return COULPS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t sites = (int64_t)Lx * Ly * Lz;
  cv_stein_partial_kernel<<<dim3(nblk, nb), kRedThreads, 0, s>>>(
      g16, D, (const __nv_bfloat16 *)s2_bf16, Aphi, sites, scratch);
  cv_sum_partials_kernel<<<(nb + 127) / 128, 128, 0, s>>>(scratch, nblk, nb, out, 0);
  const int64_t interior = (int64_t)(Lx > 2 ? Lx - 2 : 0) * (Ly > 2 ? Ly - 2 : 0) * (Lz > 2 ? Lz - 2 : 0);
  const int64_t nface = sites - interior;
  cv_boundary_partial_kernel<<<dim3(nblk, nb), kRedThreads, 0, s>>>(
      (const __nv_bfloat16 *)s1_bf16, (const __nv_bfloat16 *)s2_bf16, dK, Lx, Ly, Lz, nface,
      scratch);
  cv_sum_partials_kernel<<<(nb + 127) / 128, 128, 0, s>>>(scratch, nblk, nb, out, 1);
  return cudaGetLastError() == cudaSuccess ? COULPS_OK : COULPS_ECUDA;
}

int coulps_cv_stein_region(const float *g16, const void *s1_bf16, const void *s2_bf16,
                           const float *Aphi, const float *Ktab, int nb, const int32_t *edims,
                           const int32_t *lo, const int32_t *hi, double *scratch,
                           int64_t scratch_doubles, double *out, void *stream) {
  if (!g16 || !s1_bf16 || !s2_bf16 || !Aphi || !Ktab || !edims || !lo || !hi || !scratch || !out)
    return COULPS_EINVAL;
  if (nb < 1) return COULPS_EINVAL;
  for (int k = 0; k < 3; ++k)
    if (edims[k] < 1 || lo[k] < 0 || hi[k] > edims[k] || lo[k] >= hi[k]) return COULPS_EINVAL;
  const int nblk = 64;
  if (scratch_doubles < (int64_t)nb * nblk) return COULPS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  cv_region_partial_kernel<<<dim3(nblk, nb), kRedThreads, 0, s>>>(
      g16, (const __nv_bfloat16 *)s1_bf16, (const __nv_bfloat16 *)s2_bf16, Aphi, Ktab, edims[0],
      edims[1], edims[2], lo[0], lo[1], lo[2], hi[0], hi[1], hi[2], scratch);
  cv_sum_partials_kernel<<<(nb + 127) / 128, 128, 0, s>>>(scratch, nblk, nb, out, 0);
  return cudaGetLastError() == cudaSuccess ? COULPS_OK : COULPS_ECUDA;
}

int coulps_cv_conv3d_wgrad(const void *a_bf16, const void *dh_bf16, float *dW, int nb, int Lx,
                           int Ly, int Lz, float *scratch, int64_t scratch_floats, void *stream) {
  if (!a_bf16 || !dh_bf16 || !dW || !scratch) return COULPS_EINVAL;
  if (nb < 1 || Lx < 1 || Ly < 1 || Lz < 1) return COULPS_EINVAL;
  const int64_t ntiles = (int64_t)nb * Lz * Ly * ((Lx + kWgTile - 1) / kWgTile);
  int nblk = (int)((ntiles + 31) / 32);
  if (nblk > 1024) nblk = 1024;
  if (scratch_floats < (int64_t)nblk * 27 * 256) return COULPS_EINVAL;
  const int64_t per_block = (ntiles + nblk - 1) / nblk;
  nblk = (int)((ntiles + per_block - 1) / per_block);
  cudaStream_t s = (cudaStream_t)stream;
  cv_wgrad_partial_kernel<<<nblk, 256, 0, s>>>((const __nv_bfloat16 *)a_bf16,
                                               (const __nv_bfloat16 *)dh_bf16, Lx, Ly, Lz, ntiles,
                                               per_block, scratch);
  cv_wgrad_reduce_kernel<<<(27 * 256 + 255) / 256, 256, 0, s>>>(scratch, nblk, dW);
  return cudaGetLastError() == cudaSuccess ? COULPS_OK : COULPS_ECUDA;
}

}  // extern "C"

// coulps_cv_pack_field (api.cu) supplies the lattice's geometry and stream.
int coulps::coulps_cv_pack_field_impl(const void *field, const Geometry &g, const float *rho,
                              void *act_bf16, float *Aphi, const int *origin, const int *dims,
                              cudaStream_t s) {
  const int64_t sites = (int64_t)dims[0] * dims[1] * dims[2];
  dim3 grid((unsigned)((sites + 255) / 256), g.n_chains);
  cv_pack_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<const float *>(field), g, rho,
                                      (__nv_bfloat16 *)act_bf16, Aphi, origin[0], origin[1],
                                      origin[2], dims[0], dims[1], dims[2]);
  return cudaGetLastError() == cudaSuccess ? COULPS_OK : COULPS_ECUDA;
}
