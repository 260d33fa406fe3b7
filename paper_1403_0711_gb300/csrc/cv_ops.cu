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
#include <algorithm>
#include <cstdint>

#include <cuda_bf16.h>

#include "device_common.cuh"
#include "internal.h"

namespace coulps {
namespace {

// Site offsets of a batch of nb boxes ex x ey x ez: site (b, z, y, x) at
// b sb + z sz + y sy + x.  Dense: [b][z][y][x].  Interleaved: the boxes sit
// side by side along x, each followed by one zero column (a gutter), i.e. one
// (nb (ex + 1)) x ey x ez lattice whose 3x3x3 convolutions equal the boxes'
// own with zero padding as long as the gutters stay 0.  xw: columns per box
// row in memory.
struct BoxLayout {
  int64_t sb, sz, sy;
  int xw;
};

inline BoxLayout box_layout(int interleave, int nb, int ex, int ey, int ez) {
  BoxLayout L;
  if (interleave) {
    L.xw = ex + 1;
    L.sb = L.xw;
    L.sy = (int64_t)nb * L.xw;
    L.sz = L.sy * ey;
  } else {
    L.xw = ex;
    L.sb = (int64_t)ex * ey * ez;
    L.sz = (int64_t)ex * ey;
    L.sy = ex;
  }
  return L;
}

__device__ __forceinline__ float ld_field(const float *f, const Geometry &g, int chain, int x,
                                          int y, int z) {
  if (x < 0 || y < 0 || z < 0 || x >= g.Lx || y >= g.Ly || z >= g.Lz) return 0.f;
  const int c = (x + y + z) & 1;
  return f[(size_t)chain * g.chain_elems + (size_t)c * g.colour_elems +
           ((size_t)z * g.Ly + y) * g.W + (x >> 1)];
}

// Packs the sub-box [o, o + e) of every chain (the whole box when o = 0,
// e = L) into the layout L: rho is the full box's density.  Columns x >= e
// of a box row (the interleaved layout's gutter) are written as 0.
__global__ void cv_pack_kernel(const float *__restrict__ field, Geometry g,
                               const float *__restrict__ rho, __nv_bfloat16 *__restrict__ act,
                               float *__restrict__ Aphi, int ox, int oy, int oz, int ex, int ey,
                               int ez, BoxLayout L) {
  const int64_t n = (int64_t)L.xw * ey * ez;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int chain = blockIdx.y;
  if (i >= n) return;
  const int xl = (int)(i % L.xw), yl = (int)((i / L.xw) % ey), zl = (int)(i / ((int64_t)L.xw * ey));
  const int64_t o = (int64_t)chain * L.sb + zl * L.sz + yl * L.sy + xl;
  __align__(16) __nv_bfloat16 v[16];
  uint4 *dst = reinterpret_cast<uint4 *>(act + o * 16);
  if (xl >= ex) {
    Aphi[o] = 0.f;
    dst[0] = make_uint4(0, 0, 0, 0);
    dst[1] = make_uint4(0, 0, 0, 0);
    return;
  }
  const int x = ox + xl, y = oy + yl, z = oz + zl;
  const float p = ld_field(field, g, chain, x, y, z);
  const float S = ld_field(field, g, chain, x - 1, y, z) + ld_field(field, g, chain, x + 1, y, z) +
                  ld_field(field, g, chain, x, y - 1, z) + ld_field(field, g, chain, x, y + 1, z) +
                  ld_field(field, g, chain, x, y, z - 1) + ld_field(field, g, chain, x, y, z + 1);
  Aphi[o] = 6.f * p - S;
  const float r = rho[((int64_t)z * g.Ly + y) * g.Lx + x];
  v[0] = __float2bfloat16_rn(p);
  v[1] = __float2bfloat16_rn(r);
  v[2] = __float2bfloat16_rn(r * p);
#pragma unroll
  for (int k = 3; k < 16; ++k) v[k] = __float2bfloat16_rn(0.f);
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
// masks 1, 2, 3, 4, 6, 7 mapped to the index 0..5, class = ix + 6 iy + 36 iz;
// Ktab holds K[class][e][c2][c1].
// The sites q next to R split, per axis, into at most 5 runs of one class
// (q = lo-1, q = lo, lo < q < hi-1, q = hi-1, q = hi, clipped to E and merged
// when R is thin), so R + 1 is a union of at most 125 boxes of one class each.
// One CTA takes up to kRedThreads (q, chain, dz) items of one box: it stages
// the box's kernel K[class] in shared memory as [e][c2][c1] and each thread
// forms D[c2] = sum_{c1, e} K[c2][c1][e] s1[c1, q + e] over the 9 offsets e
// of its z plane dz (K reads are warp-wide broadcasts, four FMAs per 16-byte
// load), then its partial s2[q] . D; a site's three partials (one per dz) are
// added in the finish.  (A thread per site and all 27 offsets gave a third
// of the threads and waited on their loads.)
struct RegionRuns {
  int start[3][5], len[3][5], cls[3][5];
  int nrun[3];
  int n_box;               // nrun[0] * nrun[1] * nrun[2]
  int cta_first[126];      // first CTA of each box (prefix over boxes)
  int ex, ey, ez;          // E
  int nqx, nqy, nqz;       // R + 1 within E: offsets of the partial buffer
  int qx0, qy0, qz0;
  int nb;
  BoxLayout L;
};

constexpr int kRegionKFloats = 27 * 16 * 16;

__global__ void __launch_bounds__(kRedThreads)
    cv_region_div_kernel(const __nv_bfloat16 *__restrict__ s1, const __nv_bfloat16 *__restrict__ s2,
                         const float *__restrict__ Ktab, const RegionRuns r,
                         double *__restrict__ part) {
  __shared__ __align__(16) float K[kRegionKFloats];  // [e][c2][c1]
  int box = 0;
  while (box + 1 < r.n_box && r.cta_first[box + 1] <= (int)blockIdx.x) ++box;
  const int bx = box % r.nrun[0], by = (box / r.nrun[0]) % r.nrun[1], bz = box / (r.nrun[0] * r.nrun[1]);
  const int cls = r.cls[0][bx] + 6 * r.cls[1][by] + 36 * r.cls[2][bz];
  // the class's kernel, stored [e][c2][c1] as staged: a 16-byte copy
  const float4 *kg = reinterpret_cast<const float4 *>(Ktab + (size_t)cls * kRegionKFloats);
  for (int i = threadIdx.x; i < kRegionKFloats / 4; i += kRedThreads)
    reinterpret_cast<float4 *>(K)[i] = kg[i];
  __syncthreads();
  const int lx = r.len[0][bx], ly = r.len[1][by], lz = r.len[2][bz];
  const int nq = lx * ly * lz;
  // a warp takes one z plane dz of 32 consecutive items, so its K reads stay
  // warp-wide broadcasts
  const int item3 = (blockIdx.x - r.cta_first[box]) * kRedThreads + threadIdx.x;
  const int dzi = (item3 >> 5) % 3, item = (item3 / 96) * 32 + (item3 & 31);
  if (item >= nq * r.nb) return;
  const int chain = item / nq, k = item % nq;
  const int x = r.start[0][bx] + k % lx, y = r.start[1][by] + (k / lx) % ly, z = r.start[2][bz] + k / (lx * ly);
  const __nv_bfloat16 *s1c = s1 + chain * r.L.sb * 16;
  float D[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) D[c] = 0.f;
  for (int e = 9 * dzi; e < 9 * dzi + 9; ++e) {
    const int xx = x + e % 3 - 1, yy = y + (e / 3) % 3 - 1, zz = z + e / 9 - 1;
    if (xx < 0 || yy < 0 || zz < 0 || xx >= r.ex || yy >= r.ey || zz >= r.ez) continue;
    const uint4 *sp = reinterpret_cast<const uint4 *>(s1c + (zz * r.L.sz + yy * r.L.sy + xx) * 16);
    const uint4 u0 = sp[0], u1 = sp[1];
    float v[16];
    const __nv_bfloat162 *h0 = reinterpret_cast<const __nv_bfloat162 *>(&u0);
    const __nv_bfloat162 *h1 = reinterpret_cast<const __nv_bfloat162 *>(&u1);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 a = __bfloat1622float2(h0[i]), b = __bfloat1622float2(h1[i]);
      v[2 * i] = a.x; v[2 * i + 1] = a.y; v[8 + 2 * i] = b.x; v[8 + 2 * i + 1] = b.y;
    }
    const float4 *ke = reinterpret_cast<const float4 *>(K + e * 256);
#pragma unroll
    for (int c2 = 0; c2 < 16; ++c2) {
      float d = D[c2];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float4 w = ke[c2 * 4 + j];
        d = fmaf(w.x, v[4 * j], d);
        d = fmaf(w.y, v[4 * j + 1], d);
        d = fmaf(w.z, v[4 * j + 2], d);
        d = fmaf(w.w, v[4 * j + 3], d);
      }
      D[c2] = d;
    }
  }
  const uint4 *sq = reinterpret_cast<const uint4 *>(s2 + (chain * r.L.sb + z * r.L.sz + y * r.L.sy + x) * 16);
  const uint4 w0 = sq[0], w1 = sq[1];
  const __nv_bfloat162 *g0 = reinterpret_cast<const __nv_bfloat162 *>(&w0);
  const __nv_bfloat162 *g1 = reinterpret_cast<const __nv_bfloat162 *>(&w1);
  float acc = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 a = __bfloat1622float2(g0[i]), b = __bfloat1622float2(g1[i]);
    acc = fmaf(a.x, D[2 * i], acc);
    acc = fmaf(a.y, D[2 * i + 1], acc);
    acc = fmaf(b.x, D[8 + 2 * i], acc);
    acc = fmaf(b.y, D[8 + 2 * i + 1], acc);
  }
  const int qi = ((z - r.qz0) * r.nqy + (y - r.qy0)) * r.nqx + (x - r.qx0);
  part[((size_t)chain * ((size_t)r.nqx * r.nqy * r.nqz) + qi) * 3 + dzi] = (double)acc;
}

// out[b] = sum_q part[b][q] - sum_{x in R} g_x (A phi)_x, one CTA per chain
// (part holds nq partials per chain)
__global__ void __launch_bounds__(kRedThreads)
    cv_region_finish_kernel(const double *__restrict__ part, int nq, const float *__restrict__ g16,
                            const float *__restrict__ Aphi, BoxLayout L, int lox, int loy,
                            int loz, int hix, int hiy, int hiz, double *__restrict__ out) {
  const int chain = blockIdx.x;
  double acc = 0.0;
  for (int k = threadIdx.x; k < nq; k += kRedThreads) acc += part[(size_t)chain * nq + k];
  const int nrx = hix - lox, nry = hiy - loy, nrz = hiz - loz;
  const int nr = nrx * nry * nrz;
  for (int k = threadIdx.x; k < nr; k += kRedThreads) {
    const int x = lox + k % nrx, y = loy + (k / nrx) % nry, z = loz + k / (nrx * nry);
    const int64_t o = chain * L.sb + z * L.sz + y * L.sy + x;
    acc -= (double)g16[o * 16] * (double)Aphi[o];
  }
  block_sum_to(acc, out + chain);
}

// Per-axis runs of one class over q in [lo-1, hi] within [0, e).
static int axis_runs(int lo, int hi, int e, int *start, int *len, int *cls) {
  int n = 0;
  for (int q = lo - 1; q <= hi; ++q) {
    if (q < 0 || q >= e) continue;
    int m = 0;
    for (int f = -1; f <= 1; ++f)
      if (q - f >= lo && q - f < hi) m |= 1 << (f + 1);
    const int c = m == 1 ? 0 : m == 2 ? 1 : m == 3 ? 2 : m == 4 ? 3 : m == 6 ? 4 : m == 7 ? 5 : -1;
    if (c < 0) continue;
    if (n > 0 && cls[n - 1] == c && start[n - 1] + len[n - 1] == q) {
      ++len[n - 1];
    } else {
      if (n == 5) return -1;  // cannot happen for a box
      start[n] = q;
      len[n] = 1;
      cls[n] = c;
      ++n;
    }
  }
  return n;
}

// Charge-site term of the divergence: phi_x also enters h1 through the
// rho phi channel, with weight rho_x W1[c1][2][u].  For a charge at x,
//   rho_x sum_p sum_c2 s2[c2, x + f_p] sum_c1 M[p][c2][c1] s1[c1, x + f_p + e_p],
// over the 343 pairs (f, e) with f + e a kernel offset; per axis the pair
// index a = 0..6 stands for (f, e) = (-1,0) (-1,1) (0,-1) (0,0) (0,1) (1,-1)
// (1,0) and p = 49 az + 7 ay + ax.  Positions outside the box are 0.
__device__ __forceinline__ void pair_axis(int a, int &f, int &e) {
  f = a < 2 ? -1 : (a < 5 ? 0 : 1);
  e = a < 2 ? a : (a < 5 ? a - 3 : a - 6);
}

// One CTA per (charge, 16 chains, (ay, az)): thread (chain, c2) walks the 7
// pairs of one (y, z) offset class; the 16 chains of a CTA share each M row.
// (With a CTA per z class, 49 pairs of dependent global loads per thread
// left the kernel waiting on load latency.)
__global__ void __launch_bounds__(kRedThreads)
    cv_charge_partial_kernel(const __nv_bfloat16 *__restrict__ s1,
                             const __nv_bfloat16 *__restrict__ s2, const float *__restrict__ M,
                             const int32_t *__restrict__ qxyz, const float *__restrict__ qrho,
                             int n_q, int nb, int ex, int ey, int ez, BoxLayout L,
                             double *__restrict__ partials) {
  const int k = blockIdx.x;
  const int c2 = threadIdx.x & 15;
  const int chain = blockIdx.y * (kRedThreads / 16) + (threadIdx.x >> 4);
  const bool live = chain < nb;
  const int x = qxyz[3 * k], y = qxyz[3 * k + 1], z = qxyz[3 * k + 2];
  const __nv_bfloat16 *s1c = s1 + (live ? chain : 0) * L.sb * 16;
  const __nv_bfloat16 *s2c = s2 + (live ? chain : 0) * L.sb * 16;
  float acc = 0.f;
  const int p0 = 7 * blockIdx.z;
#pragma unroll
  for (int p = p0; p < p0 + 7; ++p) {
    if (!live) break;
    int fx, fy, fz, exx, eyy, ezz;
    pair_axis(p % 7, fx, exx);
    pair_axis((p / 7) % 7, fy, eyy);
    pair_axis(p / 49, fz, ezz);
    const int qx = x + fx, qy = y + fy, qz = z + fz;
    if (qx < 0 || qy < 0 || qz < 0 || qx >= ex || qy >= ey || qz >= ez) continue;
    const int rx = qx + exx, ry = qy + eyy, rz = qz + ezz;
    if (rx < 0 || ry < 0 || rz < 0 || rx >= ex || ry >= ey || rz >= ez) continue;
    const uint4 *sp = reinterpret_cast<const uint4 *>(s1c + (rz * L.sz + ry * L.sy + rx) * 16);
    const uint4 u0 = sp[0], u1 = sp[1];
    const __nv_bfloat162 *h0 = reinterpret_cast<const __nv_bfloat162 *>(&u0);
    const __nv_bfloat162 *h1 = reinterpret_cast<const __nv_bfloat162 *>(&u1);
    const float4 *m = reinterpret_cast<const float4 *>(M + ((size_t)p * 16 + c2) * 16);
    float d = 0.f;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const float2 a0 = __bfloat1622float2(h0[2 * i]), a1 = __bfloat1622float2(h0[2 * i + 1]);
      const float2 b0 = __bfloat1622float2(h1[2 * i]), b1 = __bfloat1622float2(h1[2 * i + 1]);
      const float4 wa = m[i], wb = m[2 + i];
      d = fmaf(wa.x, a0.x, d); d = fmaf(wa.y, a0.y, d); d = fmaf(wa.z, a1.x, d); d = fmaf(wa.w, a1.y, d);
      d = fmaf(wb.x, b0.x, d); d = fmaf(wb.y, b0.y, d); d = fmaf(wb.z, b1.x, d); d = fmaf(wb.w, b1.y, d);
    }
    acc = fmaf(__bfloat162float(s2c[(qz * L.sz + qy * L.sy + qx) * 16 + c2]), d, acc);
  }
  // sum over the 16 c2 lanes of this chain (xor butterfly within the half-warp)
  double v = (double)acc;
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (live && c2 == 0) partials[((size_t)chain * n_q + k) * 49 + blockIdx.z] = v * (double)qrho[k];
}

// out[b] += sum_k partials[b][k], k in order
__global__ void cv_add_partials_kernel(const double *__restrict__ partials, int n_q, int nb,
                                       double *__restrict__ out) {
  // one warp per chain: lane l adds entries l, l + 32, ..., then a fixed butterfly
  const int b = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= nb) return;  // whole warps
  double s = 0.0;
  for (int k = lane; k < n_q; k += 32) s += partials[(size_t)b * n_q + k];
  s = warp_sum(s);
  if (lane == 0) out[b] += s;
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
                           int interleave, const int32_t *lo, const int32_t *hi, double *scratch,
                           int64_t scratch_doubles, double *out, void *stream) {
  if (!g16 || !s1_bf16 || !s2_bf16 || !Aphi || !Ktab || !edims || !lo || !hi || !scratch || !out)
    return COULPS_EINVAL;
  if (nb < 1) return COULPS_EINVAL;
  for (int k = 0; k < 3; ++k)
    if (edims[k] < 1 || lo[k] < 0 || hi[k] > edims[k] || lo[k] >= hi[k]) return COULPS_EINVAL;
  if ((reinterpret_cast<uintptr_t>(s1_bf16) | reinterpret_cast<uintptr_t>(s2_bf16) |
       reinterpret_cast<uintptr_t>(Ktab)) & 15)
    return COULPS_EINVAL;
  RegionRuns r{};
  r.ex = edims[0]; r.ey = edims[1]; r.ez = edims[2];
  r.nb = nb;
  r.L = box_layout(interleave, nb, edims[0], edims[1], edims[2]);
  for (int k = 0; k < 3; ++k) {
    r.nrun[k] = axis_runs(lo[k], hi[k], edims[k], r.start[k], r.len[k], r.cls[k]);
    if (r.nrun[k] < 1) return COULPS_EINVAL;
  }
  r.qx0 = std::max(lo[0] - 1, 0); r.nqx = std::min(hi[0] + 1, edims[0]) - r.qx0;
  r.qy0 = std::max(lo[1] - 1, 0); r.nqy = std::min(hi[1] + 1, edims[1]) - r.qy0;
  r.qz0 = std::max(lo[2] - 1, 0); r.nqz = std::min(hi[2] + 1, edims[2]) - r.qz0;
  const int64_t nq = (int64_t)r.nqx * r.nqy * r.nqz;
  if (scratch_doubles < 3 * nq * nb) return COULPS_EINVAL;
  r.n_box = r.nrun[0] * r.nrun[1] * r.nrun[2];
  int64_t ctas = 0;
  for (int b = 0; b < r.n_box; ++b) {
    const int bx = b % r.nrun[0], by = (b / r.nrun[0]) % r.nrun[1], bz = b / (r.nrun[0] * r.nrun[1]);
    // 3 threads per item (one per z plane), in groups of 96 per 32 items
    const int64_t items = 96 * (((int64_t)r.len[0][bx] * r.len[1][by] * r.len[2][bz] * nb + 31) / 32);
    r.cta_first[b] = (int)ctas;
    ctas += (items + kRedThreads - 1) / kRedThreads;
    if (ctas > 0x7fffffff) return COULPS_EINVAL;
  }
  r.cta_first[r.n_box] = (int)ctas;
  cudaStream_t s = (cudaStream_t)stream;
  cv_region_div_kernel<<<(unsigned)ctas, kRedThreads, 0, s>>>(
      (const __nv_bfloat16 *)s1_bf16, (const __nv_bfloat16 *)s2_bf16, Ktab, r, scratch);
  cv_region_finish_kernel<<<nb, kRedThreads, 0, s>>>(scratch, (int)(3 * nq), g16, Aphi, r.L, lo[0],
                                                     lo[1], lo[2], hi[0], hi[1], hi[2], out);
  return cudaGetLastError() == cudaSuccess ? COULPS_OK : COULPS_ECUDA;
}

int coulps_cv_charge_term(const void *s1_bf16, const void *s2_bf16, const float *M,
                          const int32_t *q_xyz, const float *q_rho, int n_q, int nb,
                          const int32_t *edims, int interleave, double *scratch,
                          int64_t scratch_doubles, double *out, void *stream) {
  if (!s1_bf16 || !s2_bf16 || !M || !edims || !scratch || !out) return COULPS_EINVAL;
  if (nb < 1 || n_q < 0 || (n_q > 0 && (!q_xyz || !q_rho))) return COULPS_EINVAL;
  if (edims[0] < 1 || edims[1] < 1 || edims[2] < 1) return COULPS_EINVAL;
  if (n_q == 0) return COULPS_OK;
  if (nb > 65535 * 16) return COULPS_EINVAL;
  if (scratch_doubles < (int64_t)nb * n_q * 49) return COULPS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if ((reinterpret_cast<uintptr_t>(s1_bf16) | reinterpret_cast<uintptr_t>(M)) & 15)
    return COULPS_EINVAL;
  cv_charge_partial_kernel<<<dim3(n_q, (nb + 15) / 16, 49), kRedThreads, 0, s>>>(
      (const __nv_bfloat16 *)s1_bf16, (const __nv_bfloat16 *)s2_bf16, M, q_xyz, q_rho, n_q, nb,
      edims[0], edims[1], edims[2], box_layout(interleave, nb, edims[0], edims[1], edims[2]),
      scratch);
  cv_add_partials_kernel<<<(nb + 3) / 4, 128, 0, s>>>(scratch, 49 * n_q, nb, out);
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
                              int interleave, cudaStream_t s) {
  const BoxLayout L = box_layout(interleave, g.n_chains, dims[0], dims[1], dims[2]);
  const int64_t n = (int64_t)L.xw * dims[1] * dims[2];
  dim3 grid((unsigned)((n + 255) / 256), g.n_chains);
  cv_pack_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<const float *>(field), g, rho,
                                      (__nv_bfloat16 *)act_bf16, Aphi, origin[0], origin[1],
                                      origin[2], dims[0], dims[1], dims[2], L);
  return cudaGetLastError() == cudaSuccess ? COULPS_OK : COULPS_ECUDA;
}
