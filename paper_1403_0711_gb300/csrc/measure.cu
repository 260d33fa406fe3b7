// Estimator kernels: one term of Eq. (nsum2) per chain and the running sums.
//
//   gather:   Q = sum_i q_i phi(r_i),  P = sum_i (q_i phi(r_i))^2
//             Each product q_i * phi(r_i) is formed in FP64 (exact for an
//             FP32 field), summed per thread, then by warp shuffles and a
//             shared-memory tree into one (Q, P) partial per CTA.
//   finalize: per chain, the CTA partials are added in a fixed order (so the
//             result is bitwise reproducible), e = Q^2 - P is formed in FP64
//             (the cancelling difference of the estimator), and the running
//             sums, batch sums and optional sample log are updated.
//
// This replaces the paper's per-core partial sums and mpi_reduce with a
// deterministic two-level reduction on the device.
#include "device_common.cuh"
#include "internal.h"

namespace coulps {
namespace {

constexpr int kGatherThreads = 256;

// CHECKED (offsets from the caller's device memory, coulps_measure_static):
// an offset >= chain_elems is skipped and counted in *bad; the sums of valid
// offsets are formed in the same order as unchecked.
template <typename T, bool CHECKED>
__global__ void __launch_bounds__(kGatherThreads)
    gather_kernel(const T *__restrict__ field, size_t chain_elems,
                  const uint32_t *__restrict__ idx, const double *__restrict__ q, int64_t n,
                  double *__restrict__ partials, int nblk, int first, int stride,
                  unsigned *__restrict__ bad) {
  const int chain = first + (int)blockIdx.y * stride;
  const T *f = field + (size_t)chain * chain_elems;
  double sq = 0.0, sp = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kGatherThreads + threadIdx.x; i < n;
       i += (int64_t)nblk * kGatherThreads) {
    const uint32_t at = idx[i];
    if (CHECKED && at >= chain_elems) {
      atomicAdd(bad, 1u);
      continue;
    }
    const double t = q[i] * (double)f[at];
    sq += t;
    sp += t * t;
  }
  sq = warp_sum(sq);
  sp = warp_sum(sp);
  __shared__ double red[2][kGatherThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = sq;
    red[1][wid] = sp;
  }
  __syncthreads();
  if (wid == 0) {
    sq = lane < kGatherThreads / 32 ? red[0][lane] : 0.0;
    sp = lane < kGatherThreads / 32 ? red[1][lane] : 0.0;
    sq = warp_sum(sq);
    sp = warp_sum(sp);
    if (lane == 0) {
      partials[2 * ((size_t)chain * nblk + blockIdx.x) + 0] = sq;
      partials[2 * ((size_t)chain * nblk + blockIdx.x) + 1] = sp;
    }
  }
}

// One warp per chain: lane l adds the partials l, l + 32, ... in order, then
// a fixed butterfly adds the lanes (same order every run).
constexpr int kFinalizeWarps = 8;

__global__ void finalize_kernel(const double *__restrict__ partials, int nblk, int n_chains,
                                double *__restrict__ stats, double *__restrict__ log,
                                int64_t log_cap, int *err, double *__restrict__ Qout) {
  const int chain = blockIdx.x * kFinalizeWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (chain >= n_chains) return;  // whole warps leave together
  double Q, P;
  chain_QP(partials, nblk, chain, lane, Q, P);
  if (lane != 0) return;
  if (Qout != nullptr) Qout[chain] = Q;
  double *st = stats + (size_t)chain * kStatStride;
  const int64_t s = (int64_t)st[kStatN];
  double *row = (log != nullptr && s < log_cap) ? log + 3 * ((size_t)s * n_chains + chain) : nullptr;
  record_sample(st, Q, P, row, err);
}

// finalize for the chains first, first + stride, ... only
__global__ void finalize_group_kernel(const double *__restrict__ partials, int nblk, int n_chains,
                                      int first, int stride, double *__restrict__ stats,
                                      double *__restrict__ log, int64_t log_cap, int *err) {
  const int chain = first + (blockIdx.x * kFinalizeWarps + (threadIdx.x >> 5)) * stride;
  const int lane = threadIdx.x & 31;
  if (chain >= n_chains) return;  // whole warps leave together
  double Q, P;
  chain_QP(partials, nblk, chain, lane, Q, P);
  if (lane != 0) return;
  double *st = stats + (size_t)chain * kStatStride;
  const int64_t s = (int64_t)st[kStatN];
  double *row = (log != nullptr && s < log_cap) ? log + 3 * ((size_t)s * n_chains + chain) : nullptr;
  record_sample(st, Q, P, row, err);
}

__global__ void cv_record_kernel(const double *__restrict__ stats, const double *__restrict__ tg,
                                 double c, double *__restrict__ cv, int n_chains, int *err) {
  const int chain = blockIdx.x * blockDim.x + threadIdx.x;
  if (chain >= n_chains) return;
  const double e = stats[(size_t)chain * kStatStride + kStatLast];
  record_value(cv + (size_t)chain * kStatStride, e - c * tg[chain], err);
}

__global__ void reset_stats_kernel(double *stats, int n_chains) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_chains * kStatStride) return;
  stats[i] = (i % kStatStride == kStatBatchLen) ? 1.0 : 0.0;
}

// Off-lattice charges: particle i sees phi~_i = sum_c w_ic phi(corner c)
// (trilinear weights, eight corners given as storage offsets).  Per CTA the
// same (Q, P) partials as gather_kernel, with t_i = q_i phi~_i.
template <typename T>
__global__ void __launch_bounds__(kGatherThreads)
    gather_off_kernel(const T *__restrict__ field, size_t chain_elems,
                      const uint32_t *__restrict__ oidx, const double *__restrict__ ow,
                      const double *__restrict__ q, int64_t n, double *__restrict__ partials,
                      int nblk, int row, double *__restrict__ tout) {
  const int chain = blockIdx.y;
  const T *f = field + (size_t)chain * chain_elems;
  double sq = 0.0, sp = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kGatherThreads + threadIdx.x; i < n;
       i += (int64_t)nblk * kGatherThreads) {
    double p = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) p += ow[8 * i + c] * (double)f[oidx[8 * i + c]];
    const double t = q[i] * p;
    if (tout) tout[(size_t)chain * n + i] = t;
    sq += t;
    sp += t * t;
  }
  sq = warp_sum(sq);
  sp = warp_sum(sp);
  __shared__ double red[2][kGatherThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = sq;
    red[1][wid] = sp;
  }
  __syncthreads();
  if (wid == 0) {
    sq = lane < kGatherThreads / 32 ? red[0][lane] : 0.0;
    sp = lane < kGatherThreads / 32 ? red[1][lane] : 0.0;
    sq = warp_sum(sq);
    sp = warp_sum(sp);
    if (lane == 0) {
      partials[2 * ((size_t)chain * row + blockIdx.x) + 0] = sq;
      partials[2 * ((size_t)chain * row + blockIdx.x) + 1] = sp;
    }
  }
}

// Near pairs of an off-lattice set (CSR, both directions): thread per
// particle i, u_i = sum_{j near i} t_j with t = q phi~ of the same sample;
// the CTA's s_N part sum_i t_i u_i (= 2 sum over pairs) goes into the P slot
// of partial block `first + blockIdx.x`, so the finalize forms
// e = Q^2 - P - s_N.  u is kept for the force kernel.
__global__ void __launch_bounds__(kGatherThreads)
    near_kernel(const double *__restrict__ t, const int64_t *__restrict__ nptr,
                const uint32_t *__restrict__ nbr, int64_t n, double *__restrict__ u,
                double *__restrict__ partials, int row, int first) {
  const int chain = blockIdx.y;
  const double *tc = t + (size_t)chain * n;
  const int64_t i = (int64_t)blockIdx.x * kGatherThreads + threadIdx.x;
  double s = 0.0;
  if (i < n) {
    double ui = 0.0;
    for (int64_t k = nptr[i]; k < nptr[i + 1]; ++k) ui += tc[nbr[k]];
    u[(size_t)chain * n + i] = ui;
    s = tc[i] * ui;
  }
  s = warp_sum(s);
  __shared__ double red[kGatherThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = s;
  __syncthreads();
  if (wid == 0) {
    s = lane < kGatherThreads / 32 ? red[lane] : 0.0;
    s = warp_sum(s);
    if (lane == 0) {
      partials[2 * ((size_t)chain * row + first + blockIdx.x) + 0] = 0.0;
      partials[2 * ((size_t)chain * row + first + blockIdx.x) + 1] = s;
    }
  }
}

// Force sample of particle i in chain b (thread per (i, b)), added to the
// chain's running sums: -de/dr_i = -2 q_i (Q - q_i phi~_i) grad phi~_i with
// grad phi~_i = sum_c grad w_ic phi(corner c) and Q of the same sample.
template <typename T>
__global__ void force_off_kernel(const T *__restrict__ field, size_t chain_elems,
                                 const uint32_t *__restrict__ oidx, const double *__restrict__ ow,
                                 const double *__restrict__ og, const double *__restrict__ q,
                                 int64_t n, const double *__restrict__ Qc,
                                 const double *__restrict__ u, double *__restrict__ fsum) {
  const int chain = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T *f = field + (size_t)chain * chain_elems;
  double p = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const double v = (double)f[oidx[8 * i + c]];
    p += ow[8 * i + c] * v;
    gx += og[3 * (8 * i + c) + 0] * v;
    gy += og[3 * (8 * i + c) + 1] * v;
    gz += og[3 * (8 * i + c) + 2] * v;
  }
  // near pairs (u) are left out of the sample's energy, so of its derivative
  const double un = u ? u[(size_t)chain * n + i] : 0.0;
  const double a = -2.0 * q[i] * (Qc[chain] - q[i] * p - un);
  double *o = fsum + 3 * ((size_t)chain * n + i);
  o[0] += a * gx;
  o[1] += a * gy;
  o[2] += a * gz;
}

// Several charge sets on the same fields (the samples do not depend on where
// the charges sit): CTA (b, chain, s) does block b of set s; sets with fewer
// blocks leave early.  Same per-CTA arithmetic as gather_kernel.
template <typename T>
__global__ void __launch_bounds__(kGatherThreads)
    gather_sets_kernel(const T *__restrict__ field, size_t chain_elems, const SetTable t) {
  const int set = blockIdx.z;
  const int nblk = t.nblk[set];
  if ((int)blockIdx.x >= nblk) return;
  const int chain = blockIdx.y;
  const T *f = field + (size_t)chain * chain_elems;
  const uint32_t *idx = t.idx[set];
  const double *q = t.q[set];
  const int64_t n = t.n[set];
  double sq = 0.0, sp = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kGatherThreads + threadIdx.x; i < n;
       i += (int64_t)nblk * kGatherThreads) {
    const double v = q[i] * (double)f[idx[i]];
    sq += v;
    sp += v * v;
  }
  sq = warp_sum(sq);
  sp = warp_sum(sp);
  __shared__ double red[2][kGatherThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = sq;
    red[1][wid] = sp;
  }
  __syncthreads();
  if (wid == 0) {
    sq = lane < kGatherThreads / 32 ? red[0][lane] : 0.0;
    sp = lane < kGatherThreads / 32 ? red[1][lane] : 0.0;
    sq = warp_sum(sq);
    sp = warp_sum(sp);
    if (lane == 0) {
      t.partials[set][2 * ((size_t)chain * nblk + blockIdx.x) + 0] = sq;
      t.partials[set][2 * ((size_t)chain * nblk + blockIdx.x) + 1] = sp;
    }
  }
}

// warp per (chain, set)
__global__ void finalize_sets_kernel(const SetTable t, int n_chains, int *err) {
  const int set = blockIdx.y;
  const int chain = blockIdx.x * kFinalizeWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (chain >= n_chains) return;
  double Q, P;
  chain_QP(t.partials[set], t.nblk[set], chain, lane, Q, P);
  if (lane != 0) return;
  double *st = t.stats[set] + (size_t)chain * kStatStride;
  const int64_t s = (int64_t)st[kStatN];
  double *log = t.log[set];
  double *row = (log != nullptr && s < t.log_cap[set]) ? log + 3 * ((size_t)s * n_chains + chain)
                                                        : nullptr;
  record_sample(st, Q, P, row, err);
}

}  // namespace

cudaError_t launch_gather_off(const Geometry &g, const void *field, const uint32_t *oidx,
                              const double *ow, const double *q, int64_t n, double *partials,
                              int nblk, int row, double *tout, cudaStream_t s) {
  dim3 grid(nblk, g.n_chains);
  if (g.precision == COULPS_F32)
    gather_off_kernel<float><<<grid, kGatherThreads, 0, s>>>(
        reinterpret_cast<const float *>(field), g.chain_elems, oidx, ow, q, n, partials, nblk,
        row, tout);
  else
    gather_off_kernel<double><<<grid, kGatherThreads, 0, s>>>(
        reinterpret_cast<const double *>(field), g.chain_elems, oidx, ow, q, n, partials, nblk,
        row, tout);
  return cudaGetLastError();
}

int near_blocks(int64_t n) { return (int)((n + kGatherThreads - 1) / kGatherThreads); }

cudaError_t launch_near(const double *t, const int64_t *nptr, const uint32_t *nbr, int64_t n,
                        int n_chains, double *u, double *partials, int row, int first,
                        cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  dim3 grid(near_blocks(n), n_chains);
  near_kernel<<<grid, kGatherThreads, 0, s>>>(t, nptr, nbr, n, u, partials, row, first);
  return cudaGetLastError();
}

cudaError_t launch_force_off(const Geometry &g, const void *field, const uint32_t *oidx,
                             const double *ow, const double *og, const double *q, int64_t n,
                             const double *Qc, const double *u, double *fsum, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  dim3 grid((unsigned)((n + 127) / 128), g.n_chains);
  if (g.precision == COULPS_F32)
    force_off_kernel<float><<<grid, 128, 0, s>>>(reinterpret_cast<const float *>(field),
                                                  g.chain_elems, oidx, ow, og, q, n, Qc, u, fsum);
  else
    force_off_kernel<double><<<grid, 128, 0, s>>>(reinterpret_cast<const double *>(field),
                                                   g.chain_elems, oidx, ow, og, q, n, Qc, u, fsum);
  return cudaGetLastError();
}

cudaError_t launch_measure_sets(const Geometry &g, const void *field, const SetTable &t,
                                int *err, cudaStream_t s) {
  if (t.n_sets < 1) return cudaSuccess;
  int max_nblk = 1;
  for (int k = 0; k < t.n_sets; ++k) max_nblk = t.nblk[k] > max_nblk ? t.nblk[k] : max_nblk;
  dim3 grid(max_nblk, g.n_chains, t.n_sets);
  if (g.precision == COULPS_F32)
    gather_sets_kernel<float><<<grid, kGatherThreads, 0, s>>>(
        reinterpret_cast<const float *>(field), g.chain_elems, t);
  else
    gather_sets_kernel<double><<<grid, kGatherThreads, 0, s>>>(
        reinterpret_cast<const double *>(field), g.chain_elems, t);
  dim3 fgrid((g.n_chains + kFinalizeWarps - 1) / kFinalizeWarps, t.n_sets);
  finalize_sets_kernel<<<fgrid, 32 * kFinalizeWarps, 0, s>>>(t, g.n_chains, err);
  return cudaGetLastError();
}

int gather_blocks(int64_t n) {
  // about 4 charges per thread, at least one CTA, at most 64 per chain
  int64_t b = (n + 4 * kGatherThreads - 1) / (4 * kGatherThreads);
  if (b < 1) b = 1;
  if (b > 64) b = 64;
  return (int)b;
}

cudaError_t launch_gather_group(const Geometry &g, const void *field, const uint32_t *idx,
                                const double *q, int64_t n, double *partials, int nblk, int first,
                                int stride, cudaStream_t s) {
  const unsigned count = launch_chains(g.n_chains, first, stride);
  if (count == 0) return cudaSuccess;
  dim3 grid(nblk, count);
  if (g.precision == COULPS_F32)
    gather_kernel<float, false><<<grid, kGatherThreads, 0, s>>>(
        reinterpret_cast<const float *>(field), g.chain_elems, idx, q, n, partials, nblk, first,
        stride, nullptr);
  else
    gather_kernel<double, false><<<grid, kGatherThreads, 0, s>>>(
        reinterpret_cast<const double *>(field), g.chain_elems, idx, q, n, partials, nblk, first,
        stride, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_gather_checked(const Geometry &g, const void *field, const uint32_t *idx,
                                  const double *q, int64_t n, double *partials, int nblk,
                                  unsigned *bad, cudaStream_t s) {
  dim3 grid(nblk, g.n_chains);
  if (g.precision == COULPS_F32)
    gather_kernel<float, true><<<grid, kGatherThreads, 0, s>>>(
        reinterpret_cast<const float *>(field), g.chain_elems, idx, q, n, partials, nblk, 0, 1,
        bad);
  else
    gather_kernel<double, true><<<grid, kGatherThreads, 0, s>>>(
        reinterpret_cast<const double *>(field), g.chain_elems, idx, q, n, partials, nblk, 0, 1,
        bad);
  return cudaGetLastError();
}

cudaError_t launch_gather(const Geometry &g, const void *field, const uint32_t *idx,
                          const double *q, int64_t n, double *partials, int nblk,
                          cudaStream_t s) {
  return launch_gather_group(g, field, idx, q, n, partials, nblk, 0, 1, s);
}

cudaError_t launch_finalize(const double *partials, int nblk, int n_chains, double *stats,
                            double *log, int64_t log_cap, int *err, cudaStream_t s,
                            double *Qout) {
  finalize_kernel<<<(n_chains + kFinalizeWarps - 1) / kFinalizeWarps, 32 * kFinalizeWarps, 0, s>>>(
      partials, nblk, n_chains, stats, log, log_cap, err, Qout);
  return cudaGetLastError();
}

cudaError_t launch_finalize_group(const double *partials, int nblk, int n_chains, int first,
                                  int stride, double *stats, double *log, int64_t log_cap,
                                  int *err, cudaStream_t s) {
  const int count = (n_chains - first + stride - 1) / stride;
  if (count <= 0) return cudaSuccess;
  finalize_group_kernel<<<(count + kFinalizeWarps - 1) / kFinalizeWarps, 32 * kFinalizeWarps, 0,
                          s>>>(partials, nblk, n_chains, first, stride, stats, log, log_cap, err);
  return cudaGetLastError();
}

cudaError_t launch_cv_record(const double *stats, const double *tg, double c, double *cv,
                             int n_chains, int *err, cudaStream_t s) {
  cv_record_kernel<<<(n_chains + 127) / 128, 128, 0, s>>>(stats, tg, c, cv, n_chains, err);
  return cudaGetLastError();
}

cudaError_t launch_reset_stats(double *stats, int n_chains, cudaStream_t s) {
  const int total = n_chains * kStatStride;
  reset_stats_kernel<<<(total + 255) / 256, 256, 0, s>>>(stats, n_chains);
  return cudaGetLastError();
}

}  // namespace coulps
