// Global control variate g_x = Q(phi) h_x, Q = sum_i q_i phi(r_i) = rho . phi,
// with h a fixed field of the charge set (no phi dependence).  Its Stein term
//   T g = sum_x (dg_x/dphi_x - g_x (A phi)_x) = h . rho - Q (A h) . phi
// has mean 0 under exp(-H_L) for any h (integration by parts).  With
// h = -G rho it equals Q^2 - rho.G.rho, so e - T g = rho.G.rho - P: the far
// pairs' part of the variance of the Eq. (nsum2) sample is gone and only that
// of P = sum_i (q_i phi_i)^2 is left.  h comes from red/black SOR on
// A h = -rho (once per charge set); the estimator stays unbiased whatever the
// solver's residual, which only sets how much variance is removed.
//
// A second, local term removes most of the variance of P: g^P_x =
// sum_i q_i^2 phi(r_i) k(x - r_i), k a fixed kernel of radius R (the
// Dirichlet Green function of the (2R+1)^3 cube at its centre, restricted to
// the box), has Stein term
//   T g^P = k(0) sum_i q_i^2 - sum_i q_i^2 phi(r_i) w_i,
//   w_i = sum_d k(d) (A phi)(r_i + d)   (d over the cube, r_i + d in the box);
// with k = G(., r_i) it would equal sum q^2 G_ii - P, so e - T g - T g^P would
// be E_lat exactly.  Mean 0 for any k, like T g.
//
// Exactness: h is rounded to the fixed-point grid 2^-k (h~, k as large as lets
// 13 max|h~| 2^k stay below 2^24), so v = A h~ is a multiple of 2^-k below
// 2^24 2^-k in magnitude and exact in FP32; h~ . rho is formed in FP64.  Thus
// E[T g] = 0 holds for the h~ actually used.  The per-sample v . phi adds FP32
// products in FP32 over 16 sites and those partial sums in FP64.
#include <cmath>

#include "device_common.cuh"
#include "internal.h"

namespace coulps {
namespace {

constexpr int kGcvThreads = 256;

__device__ __forceinline__ double nat_at(const double *u, int Lx, int Ly, int Lz, int x, int y,
                                         int z) {
  if (x < 0 || y < 0 || z < 0 || x >= Lx || y >= Ly || z >= Lz) return 0.0;
  return u[((size_t)z * Ly + y) * Lx + x];
}

// one red/black SOR half-sweep of A u = -rho (natural order, FP64)
__global__ void gcv_sor_kernel(double *__restrict__ u, const double *__restrict__ rho, int Lx,
                               int Ly, int Lz, int colour, double omega) {
  const int64_t n = (int64_t)Lx * Ly * Lz;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % Lx), y = (int)((i / Lx) % Ly), z = (int)(i / ((int64_t)Lx * Ly));
    if (((x + y + z) & 1) != colour) continue;
    const double S = nat_at(u, Lx, Ly, Lz, x - 1, y, z) + nat_at(u, Lx, Ly, Lz, x + 1, y, z) +
                     nat_at(u, Lx, Ly, Lz, x, y - 1, z) + nat_at(u, Lx, Ly, Lz, x, y + 1, z) +
                     nat_at(u, Lx, Ly, Lz, x, y, z - 1) + nat_at(u, Lx, Ly, Lz, x, y, z + 1);
    u[i] = (1.0 - omega) * u[i] + omega * (S - rho[i]) / 6.0;
  }
}

__device__ __forceinline__ void block_sum2(double a, double b, double *out) {
  __shared__ double red[2][kGcvThreads / 32];
  a = warp_sum(a);
  b = warp_sum(b);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = a;
    red[1][wid] = b;
  }
  __syncthreads();
  if (wid == 0) {
    a = lane < kGcvThreads / 32 ? red[0][lane] : 0.0;
    b = lane < kGcvThreads / 32 ? red[1][lane] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) {
      out[0] = a;
      out[1] = b;
    }
  }
}

// per block four doubles: sum (A u + rho)^2, sum rho^2, max |u|, 0
__global__ void gcv_check_kernel(const double *__restrict__ u, const double *__restrict__ rho,
                                 int Lx, int Ly, int Lz, double *__restrict__ partials) {
  const int64_t n = (int64_t)Lx * Ly * Lz;
  double r2 = 0.0, b2 = 0.0, mx = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % Lx), y = (int)((i / Lx) % Ly), z = (int)(i / ((int64_t)Lx * Ly));
    const double S = nat_at(u, Lx, Ly, Lz, x - 1, y, z) + nat_at(u, Lx, Ly, Lz, x + 1, y, z) +
                     nat_at(u, Lx, Ly, Lz, x, y - 1, z) + nat_at(u, Lx, Ly, Lz, x, y + 1, z) +
                     nat_at(u, Lx, Ly, Lz, x, y, z - 1) + nat_at(u, Lx, Ly, Lz, x, y, z + 1);
    const double r = 6.0 * u[i] - S + rho[i];
    r2 += r * r;
    b2 += rho[i] * rho[i];
    mx = fmax(mx, fabs(u[i]));
  }
  block_sum2(r2, b2, partials + 4 * blockIdx.x);
  __syncthreads();
  // block max of mx through the same tree (max is order-free)
  __shared__ double m[kGcvThreads / 32];
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) m[wid] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kGcvThreads / 32; ++w) mx = fmax(mx, m[w]);
    partials[4 * blockIdx.x + 2] = mx;
    partials[4 * blockIdx.x + 3] = 0.0;
  }
}

// res[1] = |A u + rho| / |rho|, res[2] = max |u|
__global__ void gcv_check_sums_kernel(const double *__restrict__ partials, int nblk,
                                      double *__restrict__ res) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double r2 = 0.0, b2 = 0.0, mx = 0.0;
  for (int b = 0; b < nblk; ++b) {
    r2 += partials[4 * b + 0];
    b2 += partials[4 * b + 1];
    mx = fmax(mx, partials[4 * b + 2]);
  }
  res[1] = b2 > 0.0 ? sqrt(r2 / b2) : 0.0;
  res[2] = mx;
}

// h~ = round(u 2^k) 2^-k (an FP32 value), per block h~ . rho
__global__ void gcv_quantize_kernel(const double *__restrict__ u, const double *__restrict__ rho,
                                    int64_t n, double scale, double inv_scale,
                                    float *__restrict__ h32, double *__restrict__ partials) {
  double hr = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float h = (float)(rint(u[i] * scale) * inv_scale);
    h32[i] = h;
    hr += (double)h * rho[i];
  }
  block_sum2(hr, 0.0, partials + 2 * blockIdx.x);
}

__global__ void gcv_c0_kernel(const double *__restrict__ partials, int nblk,
                              double *__restrict__ res) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double hr = 0.0;
  for (int b = 0; b < nblk; ++b) hr += partials[2 * b];
  res[0] = hr;
}

// v = A h~ (exact in FP32, see above), written in the field's per-chain
// layout (colour-split, padded rows; padding and the x >= Lx tail stay 0)
__global__ void gcv_v_kernel(const float *__restrict__ h32, Geometry g, float *__restrict__ v) {
  const int64_t n = (int64_t)g.Lx * g.Ly * g.Lz;
  const int Lx = g.Lx, Ly = g.Ly, Lz = g.Lz;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % Lx), y = (int)((i / Lx) % Ly), z = (int)(i / ((int64_t)Lx * Ly));
    auto at = [&](int xx, int yy, int zz) -> double {
      if (xx < 0 || yy < 0 || zz < 0 || xx >= Lx || yy >= Ly || zz >= Lz) return 0.0;
      return (double)h32[((size_t)zz * Ly + yy) * Lx + xx];
    };
    const double val = 6.0 * (double)h32[i] - at(x - 1, y, z) - at(x + 1, y, z) - at(x, y - 1, z) -
                       at(x, y + 1, z) - at(x, y, z - 1) - at(x, y, z + 1);
    const int c = (x + y + z) & 1;
    v[(size_t)c * g.colour_elems + ((size_t)z * Ly + y) * g.W + (x >> 1)] = (float)val;
  }
}

// per (chain, block): s = v . phi over the chain's storage, Q = sum q_i phi(r_i)
template <typename T>
__global__ void __launch_bounds__(kGcvThreads)
    gcv_sample_kernel(const T *__restrict__ field, size_t chain_elems,
                      const float *__restrict__ v, const uint32_t *__restrict__ idx,
                      const double *__restrict__ q, int64_t n_q, double *__restrict__ partials) {
  const int chain = blockIdx.y;
  const T *f = field + (size_t)chain * chain_elems;
  double s = 0.0, Q = 0.0;
  const int64_t stride = (int64_t)gridDim.x * kGcvThreads;
  if (sizeof(T) == 4) {
    // 16 sites per step: four float4 of the field and of v, FP32 partial sum
    const float4 *f4 = reinterpret_cast<const float4 *>(f);
    const float4 *v4 = reinterpret_cast<const float4 *>(v);
    const int64_t n16 = (int64_t)chain_elems / 16;
    for (int64_t k = (int64_t)blockIdx.x * kGcvThreads + threadIdx.x; k < n16; k += stride) {
      float a = 0.f;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float4 x = f4[4 * k + j], w = v4[4 * k + j];
        a = fmaf(w.x, x.x, a);
        a = fmaf(w.y, x.y, a);
        a = fmaf(w.z, x.z, a);
        a = fmaf(w.w, x.w, a);
      }
      s += (double)a;
    }
    for (int64_t e = n16 * 16 + (int64_t)blockIdx.x * kGcvThreads + threadIdx.x;
         e < (int64_t)chain_elems; e += stride)
      s += (double)(v[e] * (float)f[e]);
  } else {
    for (int64_t e = (int64_t)blockIdx.x * kGcvThreads + threadIdx.x; e < (int64_t)chain_elems;
         e += stride)
      s += (double)v[e] * (double)f[e];
  }
  for (int64_t i = (int64_t)blockIdx.x * kGcvThreads + threadIdx.x; i < n_q; i += stride)
    Q += q[i] * (double)f[idx[i]];
  block_sum2(s, Q, partials + 2 * ((size_t)chain * gridDim.x + blockIdx.x));
}

// phi at (x, y, z) of one chain in the field layout (0 outside the box), in
// the field's precision
template <typename T>
__device__ __forceinline__ T phi_at(const T *f, const Geometry &g, int x, int y, int z) {
  if (x < 0 || y < 0 || z < 0 || x >= g.Lx || y >= g.Ly || z >= g.Lz) return T(0);
  const int c = (x + y + z) & 1;
  return f[(size_t)c * g.colour_elems + ((size_t)z * g.Ly + y) * g.W + (x >> 1)];
}

// warp per (charge, chain): q_i^2 phi(r_i) w_i; per block of 8 charges one
// partial per chain.  A phi and each lane's share of w are in the field's
// precision (FP32 fields: GB300's FP64 rate made the FP64 form several times
// slower; any kernel k keeps the Stein term's mean 0 and FP32 rounding of w
// adds a zero-mean error of about 1e-6 relative); lanes are added in FP64.
template <typename T>
__global__ void __launch_bounds__(256)
    gcv_p_kernel(const T *__restrict__ field, const Geometry g, const uint32_t *__restrict__ idx,
                 const double *__restrict__ q, int64_t n_q, const float *__restrict__ kt, int R,
                 double *__restrict__ partials) {
  const int chain = blockIdx.y;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * 8 + wid;
  const T *f = field + (size_t)chain * g.chain_elems;
  double contrib = 0.0;
  if (i < n_q) {
    // site of charge i from its storage offset
    const uint32_t e = idx[i];
    const int c = (int)(e / g.colour_elems);
    const uint32_t r = e - (uint32_t)c * (uint32_t)g.colour_elems;
    const int h = (int)(r % g.W), y = (int)((r / g.W) % g.Ly), z = (int)(r / ((uint32_t)g.W * g.Ly));
    const int x = 2 * h + ((c + y + z) & 1);
    const int m = 2 * R + 1, m3 = m * m * m;
    T wl = T(0);
    for (int t = lane; t < m3; t += 32) {
      const int dx = t % m - R, dy = (t / m) % m - R, dz = t / (m * m) - R;
      const int xx = x + dx, yy = y + dy, zz = z + dz;
      if (xx < 0 || yy < 0 || zz < 0 || xx >= g.Lx || yy >= g.Ly || zz >= g.Lz) continue;
      const T Ap = T(6) * phi_at(f, g, xx, yy, zz) - phi_at(f, g, xx - 1, yy, zz) -
                   phi_at(f, g, xx + 1, yy, zz) - phi_at(f, g, xx, yy - 1, zz) -
                   phi_at(f, g, xx, yy + 1, zz) - phi_at(f, g, xx, yy, zz - 1) -
                   phi_at(f, g, xx, yy, zz + 1);
      wl += (T)kt[t] * Ap;
    }
    const double w = warp_sum((double)wl);
    contrib = q[i] * q[i] * (double)f[e] * w;
  }
  __shared__ double red[8];
  if (lane == 0) red[wid] = contrib;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int k = 0; k < 8; ++k) sum += red[k];
    partials[(size_t)chain * gridDim.x + blockIdx.x] = sum;
  }
}

// warp per chain: fixed-order sums, then
// T g + T g^P = h~ . rho - Q s + cP - sum_i q_i^2 phi_i w_i
__global__ void gcv_finish_kernel(const double *__restrict__ partials, int nblk,
                                  const double *__restrict__ ppart, int nblk_p, int n_chains,
                                  const double *__restrict__ c0, double cP,
                                  double *__restrict__ tg) {
  const int chain = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (chain >= n_chains) return;
  double s = 0.0, Q = 0.0, p = 0.0;
  for (int b = lane; b < nblk; b += 32) {
    s += partials[2 * ((size_t)chain * nblk + b) + 0];
    Q += partials[2 * ((size_t)chain * nblk + b) + 1];
  }
  for (int b = lane; b < nblk_p; b += 32) p += ppart[(size_t)chain * nblk_p + b];
  s = warp_sum(s);
  Q = warp_sum(Q);
  p = warp_sum(p);
  if (lane == 0) tg[chain] = *c0 - Q * s + cP - p;
}

}  // namespace

int gcv_blocks(const Geometry &g) {
  // enough blocks per chain to stream the chain's storage at full bandwidth
  const int64_t per = (int64_t)g.chain_elems / (kGcvThreads * 16);
  int b = per < 1 ? 1 : (per > 64 ? 64 : (int)per);
  return b;
}

cudaError_t gcv_solve(const Geometry &g, const double *rho_nat, double *u_nat, float *h32,
                      float *v_layout, double *scratch, int nblk_red, int n_iter, double *res,
                      cudaStream_t s) {
  const int64_t n = (int64_t)g.Lx * g.Ly * g.Lz;
  const int threads = 256;
  const int blocks = (int)((n + threads - 1) / threads > 4096 ? 4096 : (n + threads - 1) / threads);
  // SOR factor from the Jacobi spectral radius of the Dirichlet box
  const double rj = (std::cos(M_PI / (g.Lx + 1)) + std::cos(M_PI / (g.Ly + 1)) +
                     std::cos(M_PI / (g.Lz + 1))) / 3.0;
  const double omega = 2.0 / (1.0 + std::sqrt(1.0 - rj * rj));
  cudaError_t e = cudaMemsetAsync(u_nat, 0, sizeof(double) * n, s);
  if (e != cudaSuccess) return e;
  for (int it = 0; it < n_iter; ++it)
    for (int c = 0; c < 2; ++c)
      gcv_sor_kernel<<<blocks, threads, 0, s>>>(u_nat, rho_nat, g.Lx, g.Ly, g.Lz, c, omega);
  gcv_check_kernel<<<nblk_red, kGcvThreads, 0, s>>>(u_nat, rho_nat, g.Lx, g.Ly, g.Lz, scratch);
  gcv_check_sums_kernel<<<1, 32, 0, s>>>(scratch, nblk_red, res);
  double hres[3] = {0, 0, 0};
  if ((e = cudaMemcpyAsync(hres, res, sizeof(hres), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return e;
  // largest k with 13 max|u| 2^k < 2^24 (v = A h~ then fits 24 bits exactly)
  int k = 0;
  if (hres[2] > 0.0) {
    k = (int)std::floor(std::log2((16777216.0 - 1.0) / (13.0 * hres[2])));
    if (k > 60) k = 60;
    if (k < -60) k = -60;
  }
  const double scale = std::ldexp(1.0, k), inv_scale = std::ldexp(1.0, -k);
  gcv_quantize_kernel<<<nblk_red, kGcvThreads, 0, s>>>(u_nat, rho_nat, n, scale, inv_scale, h32,
                                                       scratch);
  gcv_c0_kernel<<<1, 32, 0, s>>>(scratch, nblk_red, res);
  if ((e = cudaMemsetAsync(v_layout, 0, sizeof(float) * g.chain_elems, s)) != cudaSuccess) return e;
  gcv_v_kernel<<<blocks, threads, 0, s>>>(h32, g, v_layout);
  return cudaGetLastError();
}

// The local term (DRAM-latency-bound charge neighbourhoods) runs on `side`
// beside the v . phi sums (bandwidth-bound), forked and joined by events
// (two branches of a captured graph).
cudaError_t gcv_eval(const Geometry &g, const void *field, const float *v_layout,
                     const uint32_t *idx, const double *q, int64_t n_q, double *partials,
                     int nblk, const double *c0, const float *kt, int R, double cP,
                     double *ppart, double *tg, cudaStream_t s, cudaStream_t side,
                     cudaEvent_t fork, cudaEvent_t join) {
  const int nblk_p = R > 0 && n_q > 0 ? (int)((n_q + 7) / 8) : 0;
  cudaError_t e;
  if (nblk_p > 0) {
    if ((e = cudaEventRecord(fork, s)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(side, fork, 0)) != cudaSuccess)
      return e;
    dim3 pgrid(nblk_p, g.n_chains);
    if (g.precision == COULPS_F32)
      gcv_p_kernel<float><<<pgrid, 256, 0, side>>>(reinterpret_cast<const float *>(field), g, idx,
                                                  q, n_q, kt, R, ppart);
    else
      gcv_p_kernel<double><<<pgrid, 256, 0, side>>>(reinterpret_cast<const double *>(field), g,
                                                   idx, q, n_q, kt, R, ppart);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaEventRecord(join, side)) != cudaSuccess)
      return e;
  }
  dim3 grid(nblk, g.n_chains);
  if (g.precision == COULPS_F32)
    gcv_sample_kernel<float><<<grid, kGcvThreads, 0, s>>>(
        reinterpret_cast<const float *>(field), g.chain_elems, v_layout, idx, q, n_q, partials);
  else
    gcv_sample_kernel<double><<<grid, kGcvThreads, 0, s>>>(
        reinterpret_cast<const double *>(field), g.chain_elems, v_layout, idx, q, n_q, partials);
  if (nblk_p > 0 && (e = cudaStreamWaitEvent(s, join, 0)) != cudaSuccess) return e;
  gcv_finish_kernel<<<(g.n_chains + 7) / 8, 256, 0, s>>>(partials, nblk, ppart, nblk_p,
                                                        g.n_chains, c0, nblk_p > 0 ? cP : 0.0, tg);
  return cudaGetLastError();
}

}  // namespace coulps
