// Allocation-free variant of the measurement (coulps_measure_static).
//
// Some callers cannot allocate device memory at the moment they measure: code
// that runs while a CUDA stream is being captured into a graph (cudaMalloc is
// not allowed there), real-time or embedded controllers that forbid dynamic
// allocation after start-up, and plugins whose host application has already
// reserved all device memory.  They still own their input and output buffers.
// For them this entry point computes the same (Q, P, e) per chain as
// coulps_measure, with the gather's per-CTA partial sums placed in a fixed,
// file-scope device array instead of a buffer the library allocates.
//
// The array is loaded with the library on every GPU that loads it and stays
// there until the process exits.  Its device address is looked up once per
// device (with that device current) by cudaGetSymbolAddress; host code never
// hands the array's name itself to a kernel, because on the host that name
// denotes a host-side stand-in, not device memory.
#include <mutex>

#include "device_common.cuh"
#include "internal.h"

// Per-CTA (Q, P) partial sums of every call on this device.
static __device__ __align__(256) double g_static_scratch[COULPS_STATIC_SCRATCH_DOUBLES];

namespace coulps {
namespace {

constexpr int kMaxDevices = 64;
double *g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

// Device address of g_static_scratch on the current device (looked up once).
int static_scratch(double **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return COULPS_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return COULPS_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return COULPS_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_ptr[dev];
  return COULPS_OK;
}

// Fixed-order sum of each chain's CTA partials into (Q, P, e = Q^2 - P).
__global__ void static_qpe_kernel(const double *__restrict__ partials, int nblk, int n_chains,
                                  double *__restrict__ QPe) {
  const int chain = blockIdx.x * blockDim.x + threadIdx.x;
  if (chain >= n_chains) return;
  double Q = 0.0, P = 0.0;
  for (int b = 0; b < nblk; ++b) {
    Q += partials[2 * ((size_t)chain * nblk + b) + 0];
    P += partials[2 * ((size_t)chain * nblk + b) + 1];
  }
  QPe[3 * (size_t)chain + 0] = Q;
  QPe[3 * (size_t)chain + 1] = P;
  QPe[3 * (size_t)chain + 2] = Q * Q - P;
}

}  // namespace
}  // namespace coulps

extern "C" int coulps_measure_static(const void *field, int Lx, int Ly, int Lz, int n_chains,
                                     int precision, const uint32_t *site_index, const double *q,
                                     int64_t n, double *QPe, void *stream) {
  using namespace coulps;
  if (!field || !QPe || n < 0 || (n > 0 && (!site_index || !q))) return COULPS_EINVAL;
  if (Lx < 1 || Ly < 1 || Lz < 1 || Lx > 512 || Ly > 65535 || Lz > 65535) return COULPS_EINVAL;
  if (n_chains < 1 || n_chains > 65535) return COULPS_EINVAL;
  if (precision != COULPS_F32 && precision != COULPS_F64) return COULPS_EINVAL;
  if (n > ((int64_t)1 << 31)) return COULPS_EINVAL;
  // the storage layout of coulps_lattice_create
  Geometry g;
  g.Lx = Lx; g.Ly = Ly; g.Lz = Lz;
  g.n_chains = n_chains;
  g.precision = precision;
  g.es = precision == COULPS_F32 ? 4 : 8;
  g.Wq = (Lx + 7) / 8;
  const int align_elems = 32 / g.es;
  g.W = ((4 * g.Wq + align_elems - 1) / align_elems) * align_elems;
  g.colour_elems = (size_t)Lz * Ly * g.W;
  g.chain_elems = 2 * g.colour_elems;
  const int nblk = gather_blocks(n);
  if ((int64_t)n_chains * nblk * 2 > COULPS_STATIC_SCRATCH_DOUBLES) return COULPS_EINVAL;
  double *scratch = nullptr;
  const int st = static_scratch(&scratch);
  if (st) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (launch_gather(g, field, site_index, q, n, scratch, nblk, s) != cudaSuccess) {
    cudaGetLastError();
    return COULPS_ECUDA;
  }
  static_qpe_kernel<<<(n_chains + 127) / 128, 128, 0, s>>>(scratch, nblk, n_chains, QPe);
  if (cudaGetLastError() != cudaSuccess) return COULPS_ECUDA;
  return COULPS_OK;
}
