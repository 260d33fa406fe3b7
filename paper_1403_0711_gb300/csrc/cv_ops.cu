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
#include "tc_common.cuh"

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
// The divergence over each box is a GEMM on the tensor cores (tcgen05).  A
// tile is two x-adjacent sites of the box times 64 chains: 128 rows (the MMA's
// M), row 64 s + c = site s, chain 64 g + c of chain group g, and
//   D[row][n] = sum_e sum_c1 s1[c1, q + e] B_e[n][c1],
// with B_e[16 p + c2][c1] the p-th BF16 part of K[class][e][c2][c1]: K = hi +
// mid + lo, each part the BF16 rounding of what the parts before it leave,
// so the three hold K's 24-bit FP32 significand and each product with a BF16
// s1 value is exact (only the FP32 accumulation order differs from FP32
// arithmetic).  One MMA of K = 16 per offset e (27 per tile) accumulates
// N = 48 columns in TMEM; the epilogue adds the parts, dots the sum with
// s2[q] and writes one FP32 value per (chain, site).  The tile's operand A
// comes from one TMA box: the 4 x 3 x 3 sites around the two sites for the
// 64 chains, [z][y][x][chain][16 channels], 32-byte rows in the 32-byte
// swizzle that TMA writes and the tensor core reads (K-major, 8-row atoms of
// 256 bytes whose rows 4-7 have their two 16-byte halves exchanged), so the
// 64 rows of one site and one offset are 2 KB of consecutive atoms and the
// second site's rows follow 2 KB later, one x step on: each offset's A is a
// descriptor into the box, with no per-offset copy.  (Before: the same sums
// on the FMA pipes, then a gather of every (row, offset) by 16-byte copies,
// both 55 us per evaluation of 64 chains x 1000 sites; then two unswizzled
// boxes of 8 channels per tile, whose 16-byte pieces the TMA unit issued at
// about one per 2.7 cycles per SM: 27.5 us.)
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

constexpr int kRgThreads = 128;               // 4 warps = the 128 TMEM lanes
constexpr int kRgTPC = 4;                       // tiles per CTA (all of one box)
constexpr int kRgPos = 64 * 32;                // one block position: 64 chains x 32 B
constexpr int kRgABuf = 36 * kRgPos;            // a tile's block: 73,728 B
constexpr int kRgBe = 48 * 16 * 2;              // one offset's B: 48 rows x 16 channels BF16
constexpr int kRgAOff = 1024;                   // header: mbarriers at 0, TMEM address at 64
constexpr int kRgBOff = kRgAOff + 2 * kRgABuf;  // two A buffers
constexpr int kRgSmem = kRgBOff + 27 * kRgBe;   // 189,952 bytes
// tcgen05 instruction descriptor, kind::f16: D = F32, A = B = BF16, both
// K-major, N = 48, M = 128
constexpr uint32_t kRgIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((48u >> 3) << 17) |
                              ((128u >> 4) << 24);

// The class kernels' B operands, formed once per set of weights: for class
// cls, kRgBBytes bytes laid out as the region kernel keeps them in shared
// memory (K-major no-swizzle core matrices: element (n, c1) of offset e at
// e kRgBe + (n / 8) 128 + (c1 / 8) 768 + (n % 8) 16 + (c1 % 8) 2, row
// n = 16 p + c2 holding part p of K[cls][e][c2][c1]).  One CTA per class,
// 8 channels c1 per thread and unit.
constexpr int kRgBBytes = 27 * kRgBe;  // 41,472

__global__ void __launch_bounds__(256)
    cv_region_pack_kernel(const float *__restrict__ Ktab, unsigned char *__restrict__ kpack) {
  const int cls = blockIdx.x;
  const float *kc = Ktab + (size_t)cls * kRegionKFloats;
  unsigned char *dst = kpack + (size_t)cls * kRgBBytes;
  for (int u = threadIdx.x; u < 27 * 16 * 2; u += blockDim.x) {
    const int e = u >> 5, c2 = (u >> 1) & 15, hh = u & 1;
    const float4 *src = reinterpret_cast<const float4 *>(kc + e * 256 + c2 * 16 + 8 * hh);
    const float4 f0 = src[0], f1 = src[1];
    const float v[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
    __align__(16) __nv_bfloat16 pt[3][8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float x = v[i];
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        pt[p][i] = __float2bfloat16_rn(x);
        x -= __bfloat162float(pt[p][i]);  // exact: x minus its own rounding
      }
    }
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      const int n = 16 * p + c2;
      *reinterpret_cast<uint4 *>(dst + e * kRgBe + (n >> 3) * 128 + hh * 768 + (n & 7) * 16) =
          *reinterpret_cast<const uint4 *>(pt[p]);
    }
  }
}

// One CTA runs up to kRgTPC tiles of one class box.  Shared memory: the
// class's B (one bulk copy of its packed operand, see cv_region_pack_kernel;
// staging and splitting the FP32 kernel in every CTA cost it 27 KB of loads
// before its first tile) and two A buffers, filled by TMA one tile ahead.  Tile t's
// 27 MMAs read buffer t % 2; once they have completed, that buffer is
// refilled with tile t + 2 while the warps read the accumulator.  Every wait
// is bounded: on a timeout the CTA sets the error word, writes nothing more,
// waits (bounded) for its copies and MMAs in flight and frees its TMEM.
__global__ void __launch_bounds__(kRgThreads)
    cv_region_mma_kernel(const __grid_constant__ CUtensorMap tm_s1,
                         const __nv_bfloat16 *__restrict__ s2,
                         const unsigned char *__restrict__ kpack, const RegionRuns r,
                         double *__restrict__ part, int *err) {
  extern __shared__ unsigned char smem_raw[];
  // 1 KB aligned: the A buffers' 32-byte swizzle repeats every 256 bytes
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem);  // [0..1] A buffers, [2] MMAs, [3] B
  volatile uint32_t *tmem_slot = reinterpret_cast<volatile uint32_t *>(smem + 64);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 80);
  const uint32_t sA = smem_addr(smem + kRgAOff), sB = smem_addr(smem + kRgBOff);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // the box of this CTA: the last with cta_first[box] <= blockIdx.x
  int box = 0;
  for (int lo = 0, hi = r.n_box - 1; lo <= hi;) {
    const int mid = (lo + hi) >> 1;
    if (r.cta_first[mid] <= (int)blockIdx.x) {
      box = mid;
      lo = mid + 1;
    } else {
      hi = mid - 1;
    }
  }
  const int bx = box % r.nrun[0], by = (box / r.nrun[0]) % r.nrun[1], bz = box / (r.nrun[0] * r.nrun[1]);
  const int cls = r.cls[0][bx] + 6 * r.cls[1][by] + 36 * r.cls[2][bz];
  const int lx = r.len[0][bx], ly = r.len[1][by], lz = r.len[2][bz];
  const int nxp = (lx + 1) >> 1, ncg = (r.nb + 63) >> 6;
  const int tiles = nxp * ly * lz * ncg;
  const int t0 = ((int)blockIdx.x - r.cta_first[box]) * kRgTPC;
  const int nt = min(kRgTPC, tiles - t0);
  const int64_t nq = (int64_t)r.nqx * r.nqy * r.nqz;

  // tile t of this CTA: chain group, first site (x of site 0)
  auto tile_of = [&](int t, int &cg, int &xs, int &ys, int &zs) {
    int u = t0 + t;
    cg = u % ncg;
    u /= ncg;
    xs = r.start[0][bx] + 2 * (u % nxp);
    u /= nxp;
    ys = r.start[1][by] + u % ly;
    zs = r.start[2][bz] + u / ly;
  };
  auto issue = [&](int t) {  // thread 0
    int cg, xs, ys, zs;
    tile_of(t, cg, xs, ys, zs);
    const uint32_t bar = smem_addr(&bars[t & 1]);
    mbar_arrive_expect_tx(bar, kRgABuf);
    tma_load_5d(sA + (uint32_t)((t & 1) * kRgABuf), &tm_s1, 0, 64 * cg, xs - 1, ys - 1, zs - 1,
                bar);
  };

  int issued = 0, waited = 0, mma_issued = 0, mma_waited = 0;  // thread 0's counts
  bool b_ok = false;  // thread 0: the class's B has landed
  if (tid == 0) {
    prefetch_tensormap(&tm_s1);
    for (int i = 0; i < 4; ++i) mbar_init(smem_addr(&bars[i]), 1);
    *abort_flag = 0;
    fence_mbar_init();
    mbar_arrive_expect_tx(smem_addr(&bars[3]), kRgBBytes);
    bulk_load(sB, kpack + (size_t)cls * kRgBBytes, kRgBBytes, smem_addr(&bars[3]));
    for (; issued < 2 && issued < nt; ++issued) issue(issued);
  }
  if (warp == 0) {
    tmem_alloc(smem_addr((const void *)tmem_slot), 64);
    tmem_relinquish();
  }

  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  bool aborted = false;
  for (int t = 0; t < nt; ++t) {
    int cg, xs, ys, zs;
    tile_of(t, cg, xs, ys, zs);
    // this thread's row: site s = tid / 64 (x = xs + s), chain 64 cg + tid % 64;
    // its s2 is loaded before the waits
    const int s = tid >> 6, chain = 64 * cg + (tid & 63);
    const int x = xs + s;
    const bool valid = chain < r.nb && x - r.start[0][bx] < lx;
    uint4 w0 = make_uint4(0, 0, 0, 0), w1 = w0;
    if (valid) {
      const uint4 *sq = reinterpret_cast<const uint4 *>(
          s2 + ((size_t)chain * r.L.sb + zs * r.L.sz + ys * r.L.sy + x) * 16);
      w0 = sq[0];
      w1 = sq[1];
    }
    bool ok = true;
    if (tid == 0) {
      ok = mbar_wait_bounded(smem_addr(&bars[t & 1]), (uint32_t)((t >> 1) & 1));
      if (ok) ++waited;
      if (ok && !b_ok) ok = b_ok = mbar_wait_bounded(smem_addr(&bars[3]), 0);
      if (ok) {
        fence_after_sync();
        const uint32_t abuf = sA + (uint32_t)((t & 1) * kRgABuf);
        for (int e = 0; e < 27; ++e) {
          const int dx = e % 3, dy = (e / 3) % 3, dz = e / 9;  // offset + 1 per axis
          const uint32_t pos = (uint32_t)((dz * 3 + dy) * 4 + dx);  // site 0's x is box x 1
          mma_bf16(tmem, smem_desc_sw32(abuf + pos * kRgPos),
                   smem_desc(sB + (uint32_t)(e * kRgBe), 768, 128), kRgIdesc, e > 0 ? 1u : 0u);
        }
        mma_commit(smem_addr(&bars[2]));
        ++mma_issued;
      }
    }
    ok = ok && mbar_wait_bounded(smem_addr(&bars[2]), (uint32_t)(t & 1));
    if (tid == 0 && ok) {
      ++mma_waited;
      if (issued < nt) issue(issued++);  // the buffer of tile t is free: tile t + 2
    }
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) {
      if (lane == 0) atomicOr(err, kErrTimeout);
      *abort_flag = 1;
    }
    fence_after_sync();
    if (ok) {
      float hi[16], mid[16], lo[16];
      const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16);
      tmem_ld16(ta, hi);
      tmem_ld16(ta + 16, mid);
      tmem_ld16(ta + 32, lo);
      if (valid) {
        const __nv_bfloat162 *g0 = reinterpret_cast<const __nv_bfloat162 *>(&w0);
        const __nv_bfloat162 *g1 = reinterpret_cast<const __nv_bfloat162 *>(&w1);
        float acc = 0.f;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float2 a = __bfloat1622float2(g0[i]), b = __bfloat1622float2(g1[i]);
          acc = fmaf(a.x, (lo[2 * i] + mid[2 * i]) + hi[2 * i], acc);
          acc = fmaf(a.y, (lo[2 * i + 1] + mid[2 * i + 1]) + hi[2 * i + 1], acc);
          acc = fmaf(b.x, (lo[8 + 2 * i] + mid[8 + 2 * i]) + hi[8 + 2 * i], acc);
          acc = fmaf(b.y, (lo[9 + 2 * i] + mid[9 + 2 * i]) + hi[9 + 2 * i], acc);
        }
        const int qi = ((zs - r.qz0) * r.nqy + (ys - r.qy0)) * r.nqx + (x - r.qx0);
        part[(size_t)chain * nq + qi] = (double)acc;
      }
    }
    fence_before_sync();
    __syncthreads();  // the accumulator is free for the next tile's MMAs
    fence_after_sync();
    if (*abort_flag) {
      aborted = true;
      break;
    }
  }
  if (aborted && tid == 0) {
    // leave no copy or MMA in flight (bounded waits, in order)
    if (!b_ok) mbar_wait_bounded(smem_addr(&bars[3]), 0);
    for (int k = waited; k < issued; ++k)
      if (!mbar_wait_bounded(smem_addr(&bars[k & 1]), (uint32_t)((k >> 1) & 1))) break;
    for (int k = mma_waited; k < mma_issued; ++k)
      if (!mbar_wait_bounded(smem_addr(&bars[2]), (uint32_t)(k & 1))) break;
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 64);
}

// g_x (A phi)_x for every chain and site x of R into gpart[chain][k] (k the
// site's index in R, x fastest).  g_x, the net's output, is formed from the
// second layer's activations a2 and the last layer's weights (w3g [o][ci], 27 x
// 16 floats holding BF16 values, o = 9 kz + 3 ky + kx for the offset (kx, ky,
// kz) - 1, and bias b3g): only the sites of R need it.  Their neighbours lie
// in E, or outside the lattice where E is clipped by its faces (zero padding,
// as in the convs).  Four lanes per site take the offsets o = j, j + 4, ...
// (7, 7, 7 and 6 of them), all loads issued first; their FP32 sums are added
// by a fixed xor butterfly.  (A tensor-core conv of all of E for the one
// output channel cost 20 us per evaluation of 64 chains; one thread per site
// with three rounds of loads, 14 us.)
__global__ void __launch_bounds__(kRedThreads)
    cv_region_g_kernel(const __nv_bfloat16 *__restrict__ a2, const float *__restrict__ w3g,
                       float b3g, const float *__restrict__ Aphi, BoxLayout L, int nb, int ex,
                       int ey, int ez, int lox, int loy, int loz, int nrx, int nry, int nrz,
                       double *__restrict__ gpart) {
  __shared__ __align__(16) float w[27 * 16];
  for (int i = threadIdx.x; i < 27 * 16; i += kRedThreads) w[i] = w3g[i];
  __syncthreads();
  const int nr = nrx * nry * nrz;
  const int64_t t = (int64_t)blockIdx.x * kRedThreads + threadIdx.x;
  const int64_t i = t >> 2;  // (chain, site); whole warps stay for the shuffles
  const int j = (int)(t & 3);
  const bool live = i < (int64_t)nr * nb;
  const int chain = live ? (int)(i / nr) : 0, k = live ? (int)(i % nr) : 0;
  const int x = lox + k % nrx, y = loy + (k / nrx) % nry, z = loz + k / (nrx * nry);
  uint4 u[7][2];
#pragma unroll
  for (int m = 0; m < 7; ++m) {
    const int o = j + 4 * m;
    const int xx = x + o % 3 - 1, yy = y + (o / 3) % 3 - 1, zz = z + o / 9 - 1;
    const bool in = live && o < 27 && xx >= 0 && yy >= 0 && zz >= 0 && xx < ex && yy < ey &&
                    zz < ez;
    u[m][0] = u[m][1] = make_uint4(0, 0, 0, 0);
    if (in) {
      const uint4 *ap = reinterpret_cast<const uint4 *>(
          a2 + (chain * L.sb + zz * L.sz + yy * L.sy + xx) * 16);
      u[m][0] = ap[0];
      u[m][1] = ap[1];
    }
  }
  float g = 0.f;
#pragma unroll
  for (int m = 0; m < 7; ++m) {
    const int o = j + 4 * m;
    if (o >= 27) continue;
    const __nv_bfloat162 *h0 = reinterpret_cast<const __nv_bfloat162 *>(&u[m][0]);
    const __nv_bfloat162 *h1 = reinterpret_cast<const __nv_bfloat162 *>(&u[m][1]);
    const float *wo = w + o * 16;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 p = __bfloat1622float2(h0[q]), r = __bfloat1622float2(h1[q]);
      g = fmaf(wo[2 * q], p.x, g);
      g = fmaf(wo[2 * q + 1], p.y, g);
      g = fmaf(wo[8 + 2 * q], r.x, g);
      g = fmaf(wo[9 + 2 * q], r.y, g);
    }
  }
  g += __shfl_xor_sync(0xffffffffu, g, 1);
  g += __shfl_xor_sync(0xffffffffu, g, 2);
  if (live && j == 0)
    gpart[i] = (double)(g + b3g) * (double)Aphi[chain * L.sb + z * L.sz + y * L.sy + x];
}

// out[b] = sum_q part[b][q] - sum_k gpart[b][k], one CTA per chain (part
// holds nq partials per chain, gpart nr), fixed order.
__global__ void __launch_bounds__(kRedThreads)
    cv_region_finish_kernel(const double *__restrict__ part, int nq,
                            const double *__restrict__ gpart, int nr, double *__restrict__ out) {
  const int chain = blockIdx.x;
  double acc = 0.0;
  for (int k = threadIdx.x; k < nq; k += kRedThreads) acc += part[(size_t)chain * nq + k];
  for (int k = threadIdx.x; k < nr; k += kRedThreads) acc -= gpart[(size_t)chain * nr + k];
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

// One CTA per (charge, (ay, az) class, 64 chains), one thread per chain: the
// class's seven M matrices are staged in shared memory and read as warp-wide
// broadcasts (every lane of a warp reads the same element), and a thread
// loads, per pair, its chain's s1 at x + f + e and s2 at x + f (two 32-byte
// rows; positions outside the box are clamped into it and their terms
// multiplied by 0) before forming sum_c2 s2[c2] sum_c1 M[c2][c1] s1[c1] in
// FP32.  (A thread per (chain, c2) with M read from global memory made every
// load instruction touch 16 different M rows: 27.5 us per evaluation of 8
// charges x 64 chains, bound by L1 wavefronts and load latency.)
constexpr int kChThreads = 64;

__global__ void __launch_bounds__(kChThreads)
    cv_charge_partial_kernel(const __nv_bfloat16 *__restrict__ s1,
                             const __nv_bfloat16 *__restrict__ s2, const float *__restrict__ M,
                             const int32_t *__restrict__ qxyz, const float *__restrict__ qrho,
                             int n_q, int nb, int ex, int ey, int ez, BoxLayout L,
                             double *__restrict__ partials) {
  __shared__ __align__(16) float Ms[7 * 256];  // [pair a][c2][c1]
  const int k = blockIdx.x;
  const int cz = blockIdx.z;  // (ay, az) class: pairs 7 cz .. 7 cz + 6
  const int chain = blockIdx.y * kChThreads + threadIdx.x;
  const bool live = chain < nb;
  {
    const float4 *src = reinterpret_cast<const float4 *>(M + (size_t)7 * cz * 256);
    for (int i = threadIdx.x; i < 7 * 64; i += kChThreads) reinterpret_cast<float4 *>(Ms)[i] = src[i];
  }
  const int x = qxyz[3 * k], y = qxyz[3 * k + 1], z = qxyz[3 * k + 2];
  const __nv_bfloat16 *s1c = s1 + (size_t)(live ? chain : 0) * L.sb * 16;
  const __nv_bfloat16 *s2c = s2 + (size_t)(live ? chain : 0) * L.sb * 16;
  int fy, fz, eyy, ezz;
  pair_axis(cz % 7, fy, eyy);
  pair_axis(cz / 7, fz, ezz);
  const int qy = y + fy, qz = z + fz, ry = qy + eyy, rz = qz + ezz;
  const bool yz_in = qy >= 0 && qz >= 0 && qy < ey && qz < ez && ry >= 0 && rz >= 0 && ry < ey && rz < ez;
  const int qyc = min(max(qy, 0), ey - 1), qzc = min(max(qz, 0), ez - 1);
  const int ryc = min(max(ry, 0), ey - 1), rzc = min(max(rz, 0), ez - 1);
  uint4 u[7][2], w[7][2];
  float on[7];
#pragma unroll
  for (int a = 0; a < 7; ++a) {
    int fx, exx;
    pair_axis(a, fx, exx);
    const int qx = x + fx, rx = qx + exx;
    on[a] = (live && yz_in && qx >= 0 && qx < ex && rx >= 0 && rx < ex) ? 1.f : 0.f;
    const int qxc = min(max(qx, 0), ex - 1), rxc = min(max(rx, 0), ex - 1);
    const uint4 *sp = reinterpret_cast<const uint4 *>(s1c + (rzc * L.sz + ryc * L.sy + rxc) * 16);
    const uint4 *sq = reinterpret_cast<const uint4 *>(s2c + (qzc * L.sz + qyc * L.sy + qxc) * 16);
    u[a][0] = sp[0];
    u[a][1] = sp[1];
    w[a][0] = sq[0];
    w[a][1] = sq[1];
  }
  __syncthreads();  // Ms
  float acc = 0.f;
#pragma unroll
  for (int a = 0; a < 7; ++a) {
    float v[16], g[16];
    const __nv_bfloat162 *h0 = reinterpret_cast<const __nv_bfloat162 *>(&u[a][0]);
    const __nv_bfloat162 *h1 = reinterpret_cast<const __nv_bfloat162 *>(&u[a][1]);
    const __nv_bfloat162 *g0 = reinterpret_cast<const __nv_bfloat162 *>(&w[a][0]);
    const __nv_bfloat162 *g1 = reinterpret_cast<const __nv_bfloat162 *>(&w[a][1]);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 p0 = __bfloat1622float2(h0[i]), p1 = __bfloat1622float2(h1[i]);
      const float2 q0 = __bfloat1622float2(g0[i]), q1 = __bfloat1622float2(g1[i]);
      v[2 * i] = p0.x; v[2 * i + 1] = p0.y; v[8 + 2 * i] = p1.x; v[8 + 2 * i + 1] = p1.y;
      g[2 * i] = q0.x; g[2 * i + 1] = q0.y; g[8 + 2 * i] = q1.x; g[8 + 2 * i + 1] = q1.y;
    }
    const float4 *ma = reinterpret_cast<const float4 *>(Ms + a * 256);
    float sa = 0.f;
#pragma unroll
    for (int c2 = 0; c2 < 16; ++c2) {
      float d = 0.f;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float4 m = ma[c2 * 4 + j];
        d = fmaf(m.x, v[4 * j], d);
        d = fmaf(m.y, v[4 * j + 1], d);
        d = fmaf(m.z, v[4 * j + 2], d);
        d = fmaf(m.w, v[4 * j + 3], d);
      }
      sa = fmaf(g[c2], d, sa);
    }
    acc = fmaf(on[a], sa, acc);
  }
  if (live) partials[((size_t)chain * n_q + k) * 49 + cz] = (double)acc * (double)qrho[k];
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

int coulps_cv_stein_region(const void *a2_bf16, const float *w3g, float b3g,
                           const void *s1_bf16, const void *s2_bf16,
                           const float *Aphi, const void *kpack, int nb, const int32_t *edims,
                           int interleave, const int32_t *lo, const int32_t *hi, double *scratch,
                           int64_t scratch_doubles, double *out, int *err, void *stream) {
  if (!a2_bf16 || !w3g || !s1_bf16 || !s2_bf16 || !Aphi || !kpack || !edims || !lo || !hi ||
      !scratch || !out ||
      !err)
    return COULPS_EINVAL;
  if (nb < 1) return COULPS_EINVAL;
  for (int k = 0; k < 3; ++k)
    if (edims[k] < 1 || lo[k] < 0 || hi[k] > edims[k] || lo[k] >= hi[k]) return COULPS_EINVAL;
  if ((reinterpret_cast<uintptr_t>(s1_bf16) | reinterpret_cast<uintptr_t>(s2_bf16) |
       reinterpret_cast<uintptr_t>(a2_bf16) | reinterpret_cast<uintptr_t>(kpack)) & 15)
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
  const int64_t nr_all = (int64_t)(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
  if (scratch_doubles < (nq + nr_all) * nb) return COULPS_EINVAL;
  r.n_box = r.nrun[0] * r.nrun[1] * r.nrun[2];
  int64_t ctas = 0;
  const int64_t ncg = (nb + 63) / 64;
  for (int b = 0; b < r.n_box; ++b) {
    const int bx = b % r.nrun[0], by = (b / r.nrun[0]) % r.nrun[1], bz = b / (r.nrun[0] * r.nrun[1]);
    // tiles of two x-adjacent sites x 64 chains, kRgTPC per CTA
    const int64_t tiles = (int64_t)((r.len[0][bx] + 1) / 2) * r.len[1][by] * r.len[2][bz] * ncg;
    if (tiles > 0x7fffffff) return COULPS_EINVAL;
    r.cta_first[b] = (int)ctas;
    ctas += (tiles + kRgTPC - 1) / kRgTPC;
    if (ctas > 0x7fffffff) return COULPS_EINVAL;
  }
  r.cta_first[r.n_box] = (int)ctas;
  // s1 as a 5D tensor (channel, chain, x, y, z) of E with zero fill outside
  // it; box (16 channels, 64 chains, 4 x, 3 y, 3 z), 32-byte swizzle
  auto enc = tensor_map_encoder();
  if (!enc) return COULPS_ECUDA;
  CUtensorMap tm;
  cuuint64_t dims[5] = {16, (cuuint64_t)nb, (cuuint64_t)edims[0], (cuuint64_t)edims[1],
                        (cuuint64_t)edims[2]};
  cuuint64_t strides[4] = {(cuuint64_t)r.L.sb * 32, 32, (cuuint64_t)r.L.sy * 32,
                           (cuuint64_t)r.L.sz * 32};
  cuuint32_t box[5] = {16, 64, 4, 3, 3};
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(s1_bf16), dims, strides,
          box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return COULPS_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const int smem = kRgSmem + 1024;  // + alignment slack
  static bool configured = false;
  if (!configured) {
    if (cudaFuncSetAttribute(cv_region_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem) != cudaSuccess) {
      cudaGetLastError();
      return COULPS_ECUDA;
    }
    configured = true;
  }
  cv_region_mma_kernel<<<(unsigned)ctas, kRgThreads, smem, s>>>(
      tm, (const __nv_bfloat16 *)s2_bf16, (const unsigned char *)kpack, r, scratch, err);
  const int nrx = hi[0] - lo[0], nry = hi[1] - lo[1], nrz = hi[2] - lo[2];
  const int64_t nr = (int64_t)nrx * nry * nrz;
  double *gpart = scratch + nq * nb;
  cv_region_g_kernel<<<(unsigned)((4 * nr * nb + kRedThreads - 1) / kRedThreads), kRedThreads, 0,
                       s>>>(
      (const __nv_bfloat16 *)a2_bf16, w3g, b3g, Aphi, r.L, nb, edims[0], edims[1], edims[2],
      lo[0], lo[1], lo[2], nrx, nry, nrz, gpart);
  cv_region_finish_kernel<<<nb, kRedThreads, 0, s>>>(scratch, (int)nq, gpart, (int)nr, out);
  return cudaGetLastError() == cudaSuccess ? COULPS_OK : COULPS_ECUDA;
}

int coulps_cv_region_pack(const float *Ktab, void *kpack, void *stream) {
  if (!Ktab || !kpack) return COULPS_EINVAL;
  if ((reinterpret_cast<uintptr_t>(Ktab) | reinterpret_cast<uintptr_t>(kpack)) & 15)
    return COULPS_EINVAL;
  cv_region_pack_kernel<<<216, 256, 0, (cudaStream_t)stream>>>(
      Ktab, reinterpret_cast<unsigned char *>(kpack));
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
  if ((nb + kChThreads - 1) / kChThreads > 65535) return COULPS_EINVAL;
  if (scratch_doubles < (int64_t)nb * n_q * 49) return COULPS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if ((reinterpret_cast<uintptr_t>(s1_bf16) | reinterpret_cast<uintptr_t>(s2_bf16) |
       reinterpret_cast<uintptr_t>(M)) & 15)
    return COULPS_EINVAL;
  cv_charge_partial_kernel<<<dim3(n_q, (nb + kChThreads - 1) / kChThreads, 49), kChThreads, 0, s>>>(
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
