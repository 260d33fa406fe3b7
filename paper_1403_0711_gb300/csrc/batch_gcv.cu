// Global control variate of every system of a batch (coulps_batch_gcv_*).
//
// Per system s the control variate of gcv.cu: g_x = Q_s(phi) h_x with
// h = -G rho_s from red/black SOR on the system's box (rounded to the
// fixed-point grid that makes v = A h exact in FP32), Stein term
//   T g = h . rho_s - Q_s (A h) . phi_s,
// plus, for R > 0, the local term of P with the Dirichlet Green function of
// the (2R+1)^3 cube: k(0) sum q^2 - sum_i q_i^2 phi(r_i) w_i.  Both have mean 0
// under exp(-H_L) for any h and kernel, so e - c T g estimates E_N without
// bias for any c.
//
// Work per sample, all systems at once: the v . phi sums over fixed-size
// chunks of the batch's field array (one CTA per chunk, chunks never cross a
// system), one warp per charge for q phi and q^2 phi w, and one warp per
// system adding its chunks and charges in a fixed order.  The SOR update is
// the lattice solver's (same formula, same colour order), so a system's h is
// the one coulps_gcv_create makes for the same box and charges.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "batch_internal.h"
#include "device_common.cuh"
#include "internal.h"

namespace coulps {
namespace {

constexpr int kBgcvThreads = 256;
constexpr long long kBgcvChunk = 16384;  // field elements per CTA of the v . phi sums

struct BgcvSystem {
  int Lx, Ly, Lz, W;
  long long nat_off;       // first site of the system in the natural-order arrays
  long long field_off;     // first element of the system's field in the batch layout
  long long colour_elems;  // Lz Ly W
  double omega;            // SOR factor of the box
};

struct BgcvChunk {
  int sys;
  long long begin, end;  // elements of the batch field array
};

__device__ __forceinline__ double nat_at(const double *u, const BgcvSystem &S, int x, int y, int z) {
  if (x < 0 || y < 0 || z < 0 || x >= S.Lx || y >= S.Ly || z >= S.Lz) return 0.0;
  return u[((size_t)z * S.Ly + y) * S.Lx + x];
}

// one red/black SOR half-sweep of A u = -rho in every system (blockIdx.y)
__global__ void bgcv_sor_kernel(double *__restrict__ u, const double *__restrict__ rho,
                                const BgcvSystem *__restrict__ sys, int colour) {
  const BgcvSystem S = sys[blockIdx.y];
  double *us = u + S.nat_off;
  const double *rs = rho + S.nat_off;
  const int64_t n = (int64_t)S.Lx * S.Ly * S.Lz;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % S.Lx), y = (int)((i / S.Lx) % S.Ly),
              z = (int)(i / ((int64_t)S.Lx * S.Ly));
    if (((x + y + z) & 1) != colour) continue;
    const double sum = nat_at(us, S, x - 1, y, z) + nat_at(us, S, x + 1, y, z) +
                       nat_at(us, S, x, y - 1, z) + nat_at(us, S, x, y + 1, z) +
                       nat_at(us, S, x, y, z - 1) + nat_at(us, S, x, y, z + 1);
    us[i] = (1.0 - S.omega) * us[i] + S.omega * (sum - rs[i]) / 6.0;
  }
}

// block sums of (a, b) in a fixed order; thread 0 returns them
__device__ __forceinline__ void block_sum2(double &a, double &b) {
  __shared__ double red[2][kBgcvThreads / 32];
  a = warp_sum(a);
  b = warp_sum(b);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) {
    red[0][wid] = a;
    red[1][wid] = b;
  }
  __syncthreads();
  if (wid == 0) {
    a = lane < kBgcvThreads / 32 ? red[0][lane] : 0.0;
    b = lane < kBgcvThreads / 32 ? red[1][lane] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
  }
}

// per system (blockIdx.x): res[3 s] = |A u + rho| / |rho|, res[3 s + 1] =
// max |u|, res[3 s + 2] = |rho|^2
__global__ void __launch_bounds__(kBgcvThreads)
    bgcv_check_kernel(const double *__restrict__ u, const double *__restrict__ rho,
                      const BgcvSystem *__restrict__ sys, double *__restrict__ res) {
  const BgcvSystem S = sys[blockIdx.x];
  const double *us = u + S.nat_off;
  const double *rs = rho + S.nat_off;
  const int64_t n = (int64_t)S.Lx * S.Ly * S.Lz;
  double r2 = 0.0, b2 = 0.0, mx = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += kBgcvThreads) {
    const int x = (int)(i % S.Lx), y = (int)((i / S.Lx) % S.Ly),
              z = (int)(i / ((int64_t)S.Lx * S.Ly));
    const double sum = nat_at(us, S, x - 1, y, z) + nat_at(us, S, x + 1, y, z) +
                       nat_at(us, S, x, y - 1, z) + nat_at(us, S, x, y + 1, z) +
                       nat_at(us, S, x, y, z - 1) + nat_at(us, S, x, y, z + 1);
    const double r = 6.0 * us[i] - sum + rs[i];
    r2 += r * r;
    b2 += rs[i] * rs[i];
    mx = fmax(mx, fabs(us[i]));
  }
  block_sum2(r2, b2);
  __shared__ double m[kBgcvThreads / 32];
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) m[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kBgcvThreads / 32; ++w) mx = fmax(mx, m[w]);
    res[3 * blockIdx.x + 0] = b2 > 0.0 ? sqrt(r2 / b2) : 0.0;
    res[3 * blockIdx.x + 1] = mx;
    res[3 * blockIdx.x + 2] = b2;
  }
}

// per system: h~ = round(u 2^k) 2^-k (FP32 value), c0[s] = h~ . rho
__global__ void __launch_bounds__(kBgcvThreads)
    bgcv_quantize_kernel(const double *__restrict__ u, const double *__restrict__ rho,
                         const BgcvSystem *__restrict__ sys, const double *__restrict__ scale,
                         float *__restrict__ h32, double *__restrict__ c0) {
  const BgcvSystem S = sys[blockIdx.x];
  const double sc = scale[2 * blockIdx.x], inv = scale[2 * blockIdx.x + 1];
  const int64_t n = (int64_t)S.Lx * S.Ly * S.Lz;
  double hr = 0.0, zero = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += kBgcvThreads) {
    const float h = (float)(rint(u[S.nat_off + i] * sc) * inv);
    h32[S.nat_off + i] = h;
    hr += (double)h * rho[S.nat_off + i];
  }
  block_sum2(hr, zero);
  if (threadIdx.x == 0) c0[blockIdx.x] = hr;
}

// v = A h~ in every system's part of the batch layout (exact in FP32)
__global__ void bgcv_v_kernel(const float *__restrict__ h32, const BgcvSystem *__restrict__ sys,
                              float *__restrict__ v) {
  const BgcvSystem S = sys[blockIdx.y];
  const float *hs = h32 + S.nat_off;
  const int64_t n = (int64_t)S.Lx * S.Ly * S.Lz;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % S.Lx), y = (int)((i / S.Lx) % S.Ly),
              z = (int)(i / ((int64_t)S.Lx * S.Ly));
    auto at = [&](int xx, int yy, int zz) -> double {
      if (xx < 0 || yy < 0 || zz < 0 || xx >= S.Lx || yy >= S.Ly || zz >= S.Lz) return 0.0;
      return (double)hs[((size_t)zz * S.Ly + yy) * S.Lx + xx];
    };
    const double val = 6.0 * (double)hs[i] - at(x - 1, y, z) - at(x + 1, y, z) -
                       at(x, y - 1, z) - at(x, y + 1, z) - at(x, y, z - 1) - at(x, y, z + 1);
    const int c = (x + y + z) & 1;
    v[S.field_off + (long long)c * S.colour_elems + ((long long)z * S.Ly + y) * S.W + (x >> 1)] =
        (float)val;
  }
}

// one CTA per chunk: s = v . phi over the chunk (FP32 products summed in
// FP32 over 16 elements, those sums in FP64, as gcv.cu)
template <typename T>
__global__ void __launch_bounds__(kBgcvThreads)
    bgcv_dot_kernel(const T *__restrict__ field, const float *__restrict__ v,
                    const BgcvChunk *__restrict__ chunks, double *__restrict__ partials) {
  const BgcvChunk ch = chunks[blockIdx.x];
  double s = 0.0, zero = 0.0;
  if (sizeof(T) == 4) {
    // chunk bounds are multiples of 16 elements (system fields start and end so)
    const float4 *f4 = reinterpret_cast<const float4 *>(field) + ch.begin / 4;
    const float4 *v4 = reinterpret_cast<const float4 *>(v) + ch.begin / 4;
    const long long n16 = (ch.end - ch.begin) / 16;
    for (long long k = threadIdx.x; k < n16; k += kBgcvThreads) {
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
  } else {
    for (long long e = ch.begin + threadIdx.x; e < ch.end; e += kBgcvThreads)
      s += (double)v[e] * (double)field[e];
  }
  block_sum2(s, zero);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// phi at (x, y, z) of system S in the batch layout (0 outside the box)
template <typename T>
__device__ __forceinline__ double phi_at(const T *f, const BgcvSystem &S, int x, int y, int z) {
  if (x < 0 || y < 0 || z < 0 || x >= S.Lx || y >= S.Ly || z >= S.Lz) return 0.0;
  const int c = (x + y + z) & 1;
  return (double)f[S.field_off + (long long)c * S.colour_elems + ((long long)z * S.Ly + y) * S.W +
                   (x >> 1)];
}

// warp per charge: out[2 i] = q_i phi(r_i); out[2 i + 1] = q_i^2 phi(r_i) w_i
// (R > 0), w_i = sum_d k(d) (A phi)(r_i + d) over the cube inside the box.
// The charges' neighbourhoods are scattered over the field and mostly not in
// L2 after a sweep, so the kernel is bound by DRAM latency: lane t takes cube
// point t and issues its seven loads unconditionally (coordinates clamped
// into the box, the value masked after), and a warp loops over charges with
// the next charge's record loaded before the current one's sums.
template <typename T, int R>
__global__ void __launch_bounds__(256)
    bgcv_charge_kernel(const T *__restrict__ field, const BgcvSystem *__restrict__ sys,
                       const int4 *__restrict__ qsite, const double *__restrict__ q, int64_t n_q,
                       const float *__restrict__ kt, double *__restrict__ out) {
  constexpr int m = 2 * R + 1, m3 = m * m * m;
  constexpr int kPts = (m3 + 31) / 32;  // cube points per lane
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= n_q) return;  // whole warps
  float kl[kPts];
#pragma unroll
  for (int u = 0; u < kPts; ++u) kl[u] = lane + 32 * u < m3 ? __ldg(kt + lane + 32 * u) : 0.f;
  int4 r = __ldg(qsite + i);
  double qi = __ldg(q + i);
  for (; i < n_q; i += warps) {
    const BgcvSystem S = sys[r.w];
    const int4 rn = i + warps < n_q ? __ldg(qsite + i + warps) : r;
    const double qn = i + warps < n_q ? __ldg(q + i + warps) : 0.0;
    const T *f = field + S.field_off;
    const long long ce = S.colour_elems;
    // phi at an in-box site (x, y, z), in the field's precision: FP32 fields
    // keep A phi and the lane's share of w in FP32 (GB300's FP64 rate made the
    // FP64 form of this kernel several times slower; any kernel k keeps the
    // Stein term's mean 0, and FP32 rounding of w adds a zero-mean error of
    // about 1e-6 relative), FP64 fields in FP64
    auto at = [&](int x, int y, int z) -> T {
      return f[(long long)((x + y + z) & 1) * ce + ((long long)z * S.Ly + y) * S.W + (x >> 1)];
    };
    const double p = (double)at(r.x, r.y, r.z);
    T w = T(0);
#pragma unroll
    for (int u = 0; u < kPts; ++u) {
      const int t = lane + 32 * u;
      const int xx = r.x + t % m - R, yy = r.y + (t / m) % m - R, zz = r.z + t / (m * m) - R;
      const bool in = t < m3 && xx >= 0 && yy >= 0 && zz >= 0 && xx < S.Lx && yy < S.Ly && zz < S.Lz;
      // the point and its six neighbours, clamped into the box; a neighbour
      // outside the box is 0
      const int xc = min(max(xx, 0), S.Lx - 1), yc = min(max(yy, 0), S.Ly - 1),
                zc = min(max(zz, 0), S.Lz - 1);
      const int xm = max(xc - 1, 0), xp = min(xc + 1, S.Lx - 1);
      const int ym = max(yc - 1, 0), yp = min(yc + 1, S.Ly - 1);
      const int zm = max(zc - 1, 0), zp = min(zc + 1, S.Lz - 1);
      const T c0 = at(xc, yc, zc);
      const T vxm = at(xm, yc, zc), vxp = at(xp, yc, zc);
      const T vym = at(xc, ym, zc), vyp = at(xc, yp, zc);
      const T vzm = at(xc, yc, zm), vzp = at(xc, yc, zp);
      const T Ap = T(6) * c0 - (xc > 0 ? vxm : T(0)) - (xc < S.Lx - 1 ? vxp : T(0)) -
                   (yc > 0 ? vym : T(0)) - (yc < S.Ly - 1 ? vyp : T(0)) -
                   (zc > 0 ? vzm : T(0)) - (zc < S.Lz - 1 ? vzp : T(0));
      if (in) w += (T)kl[u] * Ap;
    }
    const double wsum = warp_sum((double)w);
    if (lane == 0) {
      out[2 * i] = qi * p;
      out[2 * i + 1] = qi * qi * p * wsum;
    }
    r = rn;
    qi = qn;
  }
}

// R = 0: out[2 i] = q_i phi(r_i), out[2 i + 1] = 0 (thread per charge)
template <typename T>
__global__ void bgcv_charge0_kernel(const T *__restrict__ field, const BgcvSystem *__restrict__ sys,
                                    const int4 *__restrict__ qsite, const double *__restrict__ q,
                                    int64_t n_q, double *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_q) return;
  const int4 r = qsite[i];
  const BgcvSystem S = sys[r.w];
  const double p = (double)field[S.field_off + (long long)((r.x + r.y + r.z) & 1) * S.colour_elems +
                                 ((long long)r.z * S.Ly + r.y) * S.W + (r.x >> 1)];
  out[2 * i] = q[i] * p;
  out[2 * i + 1] = 0.0;
}

// warp per system: fixed-order sums of its chunks and charges, then
// T g = h~ . rho - Q s + cP - sum_i q_i^2 phi_i w_i
__global__ void bgcv_finish_kernel(const double *__restrict__ dpart,
                                   const int *__restrict__ chunk_begin,
                                   const double *__restrict__ qpart,
                                   const int64_t *__restrict__ q_begin,
                                   const double *__restrict__ c0, const double *__restrict__ cP,
                                   int n_sys, double *__restrict__ tg) {
  const int s = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= n_sys) return;  // whole warps
  double d = 0.0, Q = 0.0, p = 0.0;
  for (int b = chunk_begin[s] + lane; b < chunk_begin[s + 1]; b += 32) d += dpart[b];
#pragma unroll 4
  for (int64_t i = q_begin[s] + lane; i < q_begin[s + 1]; i += 32) {
    Q += qpart[2 * i];
    p += qpart[2 * i + 1];
  }
  d = warp_sum(d);
  Q = warp_sum(Q);
  p = warp_sum(p);
  if (lane == 0) tg[s] = c0[s] - Q * d + cP[s] - p;
}

}  // namespace
}  // namespace coulps

using namespace coulps;

struct coulps_batch_gcv {
  coulps_batch *B = nullptr;
  int R = 0;
  std::vector<BgcvSystem> sys;
  std::vector<BgcvChunk> chunks;
  std::vector<int> chunk_begin;  // [n_sys + 1]
  long long n_nat = 0;
  BgcvSystem *d_sys = nullptr;
  BgcvChunk *d_chunks = nullptr;
  int *d_chunk_begin = nullptr;
  int64_t *d_q_begin = nullptr;
  float *d_h32 = nullptr;  // natural order, all systems
  float *d_v = nullptr;    // batch layout
  double *d_res = nullptr;    // [3 n_sys]: residual, max |u|, |rho|^2
  double *d_c0 = nullptr;     // [n_sys] h~ . rho
  double *d_cP = nullptr;     // [n_sys] k(0) sum q^2
  int4 *d_qsite = nullptr;
  double *d_q = nullptr;
  int64_t n_q = 0;
  float *d_k = nullptr;
  double *d_dpart = nullptr, *d_qpart = nullptr, *d_tg = nullptr, *d_cvstats = nullptr;
  int sms = 0;  // multiprocessors of the device
  // the charge kernel (DRAM-latency-bound) runs on a side stream beside the
  // v . phi kernel (bandwidth-bound); fork and join by events, which a stream
  // capture turns into two branches of the graph
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_hb = -1, graph_or = -1;
  double graph_c = 0.0;
};

namespace {

#define CK(expr)                          \
  do {                                    \
    cudaError_t e_ = (expr);              \
    if (e_ != cudaSuccess) {              \
      cudaGetLastError();                 \
      return COULPS_ECUDA;                \
    }                                     \
  } while (0)

template <typename P>
void gfree(coulps_batch_gcv *G, P *&p) {
  dev_free(G->B->alloc, (void *)p, G->B->stream);
  p = nullptr;
}

void drop_graph(coulps_batch_gcv *G) {
  if (G->graph) cudaGraphExecDestroy(G->graph);
  G->graph = nullptr;
}

// q phi and the local P term of every charge: persistent warps (8 per block,
// 8 blocks per SM)
template <typename T>
cudaError_t launch_charge(coulps_batch_gcv *G, const T *field, cudaStream_t st) {
  if (G->R == 0) {
    bgcv_charge0_kernel<T><<<(int)((G->n_q + 255) / 256), 256, 0, st>>>(
        field, G->d_sys, G->d_qsite, G->d_q, G->n_q, G->d_qpart);
    return cudaGetLastError();
  }
  const int64_t need = (G->n_q + 7) / 8;
  const int blocks = (int)std::min<int64_t>(need, (int64_t)G->sms * 8);
  switch (G->R) {
    case 1:
      bgcv_charge_kernel<T, 1><<<blocks, 256, 0, st>>>(field, G->d_sys, G->d_qsite, G->d_q,
                                                               G->n_q, G->d_k, G->d_qpart);
      break;
    case 2:
      bgcv_charge_kernel<T, 2><<<blocks, 256, 0, st>>>(field, G->d_sys, G->d_qsite, G->d_q,
                                                               G->n_q, G->d_k, G->d_qpart);
      break;
    case 3:
      bgcv_charge_kernel<T, 3><<<blocks, 256, 0, st>>>(field, G->d_sys, G->d_qsite, G->d_q,
                                                               G->n_q, G->d_k, G->d_qpart);
      break;
    default:
      bgcv_charge_kernel<T, 4><<<blocks, 256, 0, st>>>(field, G->d_sys, G->d_qsite, G->d_q,
                                                               G->n_q, G->d_k, G->d_qpart);
      break;
  }
  return cudaGetLastError();
}

// T g of every system's current field into tg (device, n_sys doubles)
int bgcv_enqueue_eval(coulps_batch_gcv *G, double *tg) {
  coulps_batch *B = G->B;
  const int n_chunks = (int)G->chunks.size();
  const bool fork = G->n_q > 0;
  if (fork) {
    CK(cudaEventRecord(G->ev_fork, B->stream));
    CK(cudaStreamWaitEvent(G->side, G->ev_fork, 0));
    CK(B->precision == COULPS_F32
           ? launch_charge<float>(G, reinterpret_cast<const float *>(B->field), G->side)
           : launch_charge<double>(G, reinterpret_cast<const double *>(B->field), G->side));
    CK(cudaEventRecord(G->ev_join, G->side));
  }
  if (B->precision == COULPS_F32)
    bgcv_dot_kernel<float><<<n_chunks, kBgcvThreads, 0, B->stream>>>(
        reinterpret_cast<const float *>(B->field), G->d_v, G->d_chunks, G->d_dpart);
  else
    bgcv_dot_kernel<double><<<n_chunks, kBgcvThreads, 0, B->stream>>>(
        reinterpret_cast<const double *>(B->field), G->d_v, G->d_chunks, G->d_dpart);
  CK(cudaGetLastError());
  if (fork) CK(cudaStreamWaitEvent(B->stream, G->ev_join, 0));
  bgcv_finish_kernel<<<(B->n_sys + 7) / 8, 256, 0, B->stream>>>(
      G->d_dpart, G->d_chunk_begin, G->d_qpart, G->d_q_begin, G->d_c0, G->d_cP, B->n_sys, tg);
  CK(cudaGetLastError());
  return COULPS_OK;
}

int bgcv_enqueue_step(coulps_batch_gcv *G, int n_hb, int n_or, double c) {
  coulps_batch *B = G->B;
  int st = batch_enqueue(B, n_hb, n_or, true);
  if (st) return st;
  st = bgcv_enqueue_eval(G, G->d_tg);
  if (st) return st;
  CK(launch_cv_record(B->d_stats, G->d_tg, c, G->d_cvstats, B->n_sys, B->d_err, B->stream));
  return COULPS_OK;
}

}  // namespace

extern "C" {

void coulps_batch_gcv_destroy(coulps_batch_gcv_t G) {
  if (!G) return;
  drop_graph(G);
  if (G->B && G->B->stream) cudaStreamSynchronize(G->B->stream);
  if (G->side) cudaStreamSynchronize(G->side);
  if (G->ev_fork) cudaEventDestroy(G->ev_fork);
  if (G->ev_join) cudaEventDestroy(G->ev_join);
  if (G->side) cudaStreamDestroy(G->side);
  gfree(G, G->d_sys);
  gfree(G, G->d_chunks);
  gfree(G, G->d_chunk_begin);
  gfree(G, G->d_q_begin);
  gfree(G, G->d_h32);
  gfree(G, G->d_v);
  gfree(G, G->d_res);
  gfree(G, G->d_c0);
  gfree(G, G->d_cP);
  gfree(G, G->d_qsite);
  gfree(G, G->d_q);
  gfree(G, G->d_k);
  gfree(G, G->d_dpart);
  gfree(G, G->d_qpart);
  gfree(G, G->d_tg);
  gfree(G, G->d_cvstats);
  delete G;
}

int coulps_batch_gcv_create(coulps_batch_t B, int n_iter, int R, coulps_batch_gcv_t *out) {
  if (!B || !out || n_iter < 0 || R < 0 || R > 4) return COULPS_EINVAL;
  *out = nullptr;
  if (!B->has_charges) return COULPS_EINVAL;
  coulps_batch_gcv *G = new (std::nothrow) coulps_batch_gcv();
  if (!G) return COULPS_ENOMEM;
  G->B = B;
  const int n_sys = B->n_sys;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&G->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaStreamCreateWithFlags(&G->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&G->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&G->ev_join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      coulps_batch_gcv_destroy(G);
      return COULPS_ECUDA;
    }
  }
  G->n_q = B->offsets[n_sys];
  G->R = G->n_q > 0 ? R : 0;
  // systems, natural-order offsets, chunks of the field array
  long long nat = 0;
  G->chunk_begin.assign(n_sys + 1, 0);
  for (int s = 0; s < n_sys; ++s) {
    const BatchSystem &S = B->sys[s];
    BgcvSystem g;
    g.Lx = S.Lx; g.Ly = S.Ly; g.Lz = S.Lz; g.W = S.W;
    g.nat_off = nat;
    g.field_off = S.field_off;
    g.colour_elems = S.colour_elems;
    // SOR factor from the Jacobi spectral radius of the Dirichlet box
    const double rj = (std::cos(M_PI / (S.Lx + 1)) + std::cos(M_PI / (S.Ly + 1)) +
                       std::cos(M_PI / (S.Lz + 1))) / 3.0;
    g.omega = 2.0 / (1.0 + std::sqrt(1.0 - rj * rj));
    G->sys.push_back(g);
    nat += (long long)S.Lx * S.Ly * S.Lz;
    G->chunk_begin[s] = (int)G->chunks.size();
    const long long b0 = S.field_off, b1 = S.field_off + 2 * S.colour_elems;
    for (long long b = b0; b < b1; b += kBgcvChunk)
      G->chunks.push_back(BgcvChunk{s, b, std::min(b + kBgcvChunk, b1)});
  }
  G->chunk_begin[n_sys] = (int)G->chunks.size();
  G->n_nat = nat;
  const size_t field_elems = B->field_bytes / B->es;
  auto A = [&](size_t bytes) { return dev_alloc(B->alloc, std::max<size_t>(bytes, 16), B->stream); };
  G->d_sys = (BgcvSystem *)A(G->sys.size() * sizeof(BgcvSystem));
  G->d_chunks = (BgcvChunk *)A(G->chunks.size() * sizeof(BgcvChunk));
  G->d_chunk_begin = (int *)A(G->chunk_begin.size() * sizeof(int));
  G->d_q_begin = (int64_t *)A((n_sys + 1) * sizeof(int64_t));
  G->d_h32 = (float *)A(nat * sizeof(float));
  G->d_v = (float *)A(field_elems * sizeof(float));
  G->d_res = (double *)A(3 * (size_t)n_sys * sizeof(double));
  G->d_c0 = (double *)A((size_t)n_sys * sizeof(double));
  G->d_cP = (double *)A((size_t)n_sys * sizeof(double));
  G->d_qsite = (int4 *)A((size_t)G->n_q * sizeof(int4));
  G->d_q = (double *)A((size_t)G->n_q * sizeof(double));
  G->d_dpart = (double *)A(G->chunks.size() * sizeof(double));
  G->d_qpart = (double *)A(2 * (size_t)G->n_q * sizeof(double));
  G->d_tg = (double *)A((size_t)n_sys * sizeof(double));
  G->d_cvstats = (double *)A((size_t)n_sys * kStatStride * sizeof(double));
  double *d_rho = (double *)A(nat * sizeof(double));
  double *d_u = (double *)A(nat * sizeof(double));
  double *d_scale = (double *)A(2 * (size_t)n_sys * sizeof(double));
  auto fail = [&](int code) {
    dev_free(B->alloc, d_rho, B->stream);
    dev_free(B->alloc, d_u, B->stream);
    dev_free(B->alloc, d_scale, B->stream);
    coulps_batch_gcv_destroy(G);
    return code;
  };
  if (!G->d_sys || !G->d_chunks || !G->d_chunk_begin || !G->d_q_begin || !G->d_h32 || !G->d_v ||
      !G->d_res || !G->d_c0 || !G->d_cP || !G->d_qsite || !G->d_q || !G->d_dpart ||
      !G->d_qpart || !G->d_tg || !G->d_cvstats || !d_rho || !d_u || !d_scale)
    return fail(COULPS_ENOMEM);
  // host side: charge density, per-charge sites, the cube kernel and cP
  std::vector<double> rho, cP(n_sys, 0.0);
  std::vector<int4> qsite;
  std::vector<float> kt;
  try {
    rho.assign((size_t)nat, 0.0);
    qsite.resize((size_t)G->n_q);
  } catch (...) {
    return fail(COULPS_ENOMEM);
  }
  if (G->R > 0) kt = cube_green(G->R);
  const int m = 2 * G->R + 1;
  const double k0 = G->R > 0 ? (double)kt[(G->R * m + G->R) * m + G->R] : 0.0;
  // each system's charges in site order (z, y, x): the warps working at one
  // time then read neighbouring parts of the field (L2 reuse)
  std::vector<double> qs;
  try {
    qs.resize((size_t)G->n_q);
  } catch (...) {
    return fail(COULPS_ENOMEM);
  }
  std::vector<int64_t> perm;
  for (int s = 0; s < n_sys; ++s) {
    const BgcvSystem &g = G->sys[s];
    perm.clear();
    for (int64_t i = B->offsets[s]; i < B->offsets[s + 1]; ++i) perm.push_back(i);
    auto key = [&](int64_t i) {
      const int32_t *p = &B->sites[3 * i];
      return ((int64_t)p[2] * g.Ly + p[1]) * g.Lx + p[0];
    };
    std::stable_sort(perm.begin(), perm.end(), [&](int64_t a, int64_t b) { return key(a) < key(b); });
    // rho in the charges' input order (as the single-lattice solver adds them)
    for (int64_t i = B->offsets[s]; i < B->offsets[s + 1]; ++i) {
      const int32_t *p = &B->sites[3 * i];
      rho[g.nat_off + ((size_t)p[2] * g.Ly + p[1]) * g.Lx + p[0]] += B->q[i];
    }
    for (size_t k = 0; k < perm.size(); ++k) {
      const int64_t i = perm[k], o = B->offsets[s] + (int64_t)k;
      const int32_t *p = &B->sites[3 * i];
      qsite[o] = make_int4(p[0], p[1], p[2], s);
      qs[o] = B->q[i];
      cP[s] += k0 * B->q[i] * B->q[i];
    }
  }
  if (G->R > 0) {
    G->d_k = (float *)A(kt.size() * sizeof(float));
    if (!G->d_k) return fail(COULPS_ENOMEM);
  }
  const cudaStream_t st = B->stream;
  auto up = [&](void *d, const void *h, size_t bytes) {
    return bytes == 0 || cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, st) == cudaSuccess;
  };
  if (!up(G->d_sys, G->sys.data(), G->sys.size() * sizeof(BgcvSystem)) ||
      !up(G->d_chunks, G->chunks.data(), G->chunks.size() * sizeof(BgcvChunk)) ||
      !up(G->d_chunk_begin, G->chunk_begin.data(), G->chunk_begin.size() * sizeof(int)) ||
      !up(G->d_q_begin, B->offsets.data(), (n_sys + 1) * sizeof(int64_t)) ||
      !up(G->d_qsite, qsite.data(), qsite.size() * sizeof(int4)) ||
      !up(G->d_q, qs.data(), qs.size() * sizeof(double)) ||
      !up(G->d_cP, cP.data(), cP.size() * sizeof(double)) ||
      !up(d_rho, rho.data(), rho.size() * sizeof(double)) ||
      (G->R > 0 && !up(G->d_k, kt.data(), kt.size() * sizeof(float))))
    return fail(COULPS_ECUDA);
  // SOR on every system at once, then residual and max |u| per system
  if (cudaMemsetAsync(d_u, 0, (size_t)nat * sizeof(double), st) != cudaSuccess)
    return fail(COULPS_ECUDA);
  const dim3 sgrid(32, n_sys);
  for (int it = 0; it < n_iter; ++it)
    for (int c = 0; c < 2; ++c)
      bgcv_sor_kernel<<<sgrid, 256, 0, st>>>(d_u, d_rho, G->d_sys, c);
  bgcv_check_kernel<<<n_sys, kBgcvThreads, 0, st>>>(d_u, d_rho, G->d_sys, G->d_res);
  std::vector<double> res(3 * (size_t)n_sys);
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(res.data(), G->d_res, res.size() * sizeof(double), cudaMemcpyDeviceToHost,
                      st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(COULPS_ECUDA);
  // per system the largest k with 13 max|u| 2^k < 2^24 (v = A h~ exact in FP32)
  std::vector<double> scale(2 * (size_t)n_sys);
  for (int s = 0; s < n_sys; ++s) {
    int k = 0;
    const double mx = res[3 * s + 1];
    if (mx > 0.0) {
      k = (int)std::floor(std::log2((16777216.0 - 1.0) / (13.0 * mx)));
      k = std::max(-60, std::min(60, k));
    }
    scale[2 * s] = std::ldexp(1.0, k);
    scale[2 * s + 1] = std::ldexp(1.0, -k);
  }
  if (!up(d_scale, scale.data(), scale.size() * sizeof(double)) ||
      cudaMemsetAsync(G->d_v, 0, field_elems * sizeof(float), st) != cudaSuccess)
    return fail(COULPS_ECUDA);
  bgcv_quantize_kernel<<<n_sys, kBgcvThreads, 0, st>>>(d_u, d_rho, G->d_sys, d_scale, G->d_h32,
                                                      G->d_c0);
  bgcv_v_kernel<<<sgrid, 256, 0, st>>>(G->d_h32, G->d_sys, G->d_v);
  if (cudaGetLastError() != cudaSuccess ||
      launch_reset_stats(G->d_cvstats, n_sys, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)  // host vectors leave scope
    return fail(COULPS_ECUDA);
  dev_free(B->alloc, d_rho, st);
  dev_free(B->alloc, d_u, st);
  dev_free(B->alloc, d_scale, st);
  *out = G;
  return COULPS_OK;
}

int coulps_batch_gcv_info(coulps_batch_gcv_t G, double *out) {
  if (!G || !out) return COULPS_EINVAL;
  coulps_batch *B = G->B;
  std::vector<double> res(3 * (size_t)B->n_sys), c0(B->n_sys);
  CK(cudaMemcpyAsync(res.data(), G->d_res, res.size() * sizeof(double), cudaMemcpyDeviceToHost,
                     B->stream));
  CK(cudaMemcpyAsync(c0.data(), G->d_c0, c0.size() * sizeof(double), cudaMemcpyDeviceToHost,
                     B->stream));
  int s = batch_sync(B);
  if (s) return s;
  for (int k = 0; k < B->n_sys; ++k) {
    out[2 * k] = c0[k];
    out[2 * k + 1] = res[3 * k];
  }
  return COULPS_OK;
}

int coulps_batch_gcv_h(coulps_batch_gcv_t G, int system, float *host_xyz) {
  if (!G || !host_xyz || system < 0 || system >= G->B->n_sys) return COULPS_EINVAL;
  const BgcvSystem &g = G->sys[system];
  CK(cudaMemcpyAsync(host_xyz, G->d_h32 + g.nat_off,
                     (size_t)g.Lx * g.Ly * g.Lz * sizeof(float), cudaMemcpyDeviceToHost,
                     G->B->stream));
  return batch_sync(G->B);
}

int coulps_batch_gcv_eval(coulps_batch_gcv_t G, double *tg) {
  if (!G) return COULPS_EINVAL;
  return bgcv_enqueue_eval(G, tg ? tg : G->d_tg);
}

int coulps_batch_gcv_run(coulps_batch_gcv_t G, int n_meas, int n_hb, int n_or, double c) {
  if (!G || n_meas < 0 || n_hb < 0 || n_or < 0 || n_hb + n_or == 0 || !std::isfinite(c))
    return COULPS_EINVAL;
  coulps_batch *B = G->B;
  if (n_meas == 0) return COULPS_OK;
  const bool capturable = B->stream != nullptr;
  if (capturable && (!G->graph || G->graph_hb != n_hb || G->graph_or != n_or || G->graph_c != c)) {
    drop_graph(G);
    cudaGraph_t gr = nullptr;
    CK(cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
    const int s1 = bgcv_enqueue_step(G, n_hb, n_or, c);
    cudaError_t e = cudaStreamEndCapture(B->stream, &gr);
    if (s1 || e != cudaSuccess) {
      cudaGetLastError();
      if (gr) cudaGraphDestroy(gr);
      return s1 ? s1 : COULPS_ECUDA;
    }
    e = cudaGraphInstantiate(&G->graph, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
      cudaGetLastError();
      G->graph = nullptr;
      return COULPS_ECUDA;
    }
    G->graph_hb = n_hb;
    G->graph_or = n_or;
    G->graph_c = c;
  }
  for (int k = 0; k < n_meas; ++k) {
    if (capturable) {
      CK(cudaGraphLaunch(G->graph, B->stream));
    } else {
      const int st = bgcv_enqueue_step(G, n_hb, n_or, c);
      if (st) return st;
    }
    B->pass += (uint64_t)(n_hb + n_or);
  }
  return COULPS_OK;
}

int coulps_batch_gcv_reset(coulps_batch_gcv_t G) {
  if (!G) return COULPS_EINVAL;
  CK(launch_reset_stats(G->d_cvstats, G->B->n_sys, G->B->stream));
  return COULPS_OK;
}

int coulps_batch_gcv_stats(coulps_batch_gcv_t G, double *out, int64_t cap) {
  if (!G || !out) return COULPS_EINVAL;
  const int64_t need = (int64_t)G->B->n_sys * kStatStride;
  if (cap < need) return COULPS_EINVAL;
  CK(cudaMemcpyAsync(out, G->d_cvstats, need * sizeof(double), cudaMemcpyDeviceToHost,
                     G->B->stream));
  return batch_sync(G->B);
}

int coulps_batch_gcv_estimate(coulps_batch_gcv_t G, double *mean, double *stderr_bm,
                              double *tau_int, int64_t *n) {
  if (!G) return COULPS_EINVAL;
  coulps_batch *B = G->B;
  std::vector<double> st((size_t)B->n_sys * kStatStride);
  int s = coulps_batch_gcv_stats(G, st.data(), (int64_t)st.size());
  if (s) return s;
  for (int k = 0; k < B->n_sys; ++k) {
    double m, e, t;
    int64_t c;
    s = coulps_pool_stats(st.data() + (size_t)k * kStatStride, 1, &m, &e, &t, &c);
    if (s && s != COULPS_ENONFINITE) return s;
    if (mean) mean[k] = m;
    if (stderr_bm) stderr_bm[k] = e;
    if (tau_int) tau_int[k] = t;
    if (n) n[k] = c;
  }
  return COULPS_OK;
}

}  // extern "C"
