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
// denotes a host-side stand-in, not device memory.  A device reset while the
// library is loaded is not supported: the looked-up address would be stale.
#include <mutex>

#include "device_common.cuh"
#include "internal.h"

// Per-CTA (Q, P) partial sums of every call on this device.
static __device__ __align__(256) double g_static_scratch[COULPS_STATIC_SCRATCH_DOUBLES];
// Count of charge offsets of the current call that lie outside a chain's field.
static __device__ __align__(256) unsigned g_static_bad[1];

namespace coulps {
namespace {

constexpr int kMaxDevices = 64;
double *g_scratch_ptr[kMaxDevices] = {};
unsigned *g_bad_ptr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

// Device addresses of g_static_scratch and g_static_bad on the current device
// (looked up once per device).
int static_scratch(double **out, unsigned **bad) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return COULPS_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return COULPS_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr, *b = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr ||
        cudaGetSymbolAddress(&b, g_static_bad) != cudaSuccess || b == nullptr) {
      cudaGetLastError();
      return COULPS_ECUDA;
    }
    g_bad_ptr[dev] = static_cast<unsigned *>(b);
    g_scratch_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_ptr[dev];
  *bad = g_bad_ptr[dev];
  return COULPS_OK;
}

// Each chain's CTA partials added in the order of coulps_measure's finalize
// (one warp per chain, chain_QP), so both return bitwise the same (Q, P, e);
// NaN for every chain when an offset was out of range.
constexpr int kQpeWarps = 8;
__global__ void static_qpe_kernel(const double *__restrict__ partials, int nblk, int n_chains,
                                  const unsigned *__restrict__ bad, double *__restrict__ QPe) {
  const int chain = blockIdx.x * kQpeWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (chain >= n_chains) return;  // whole warps leave together
  double Q, P;
  chain_QP(partials, nblk, chain, lane, Q, P);
  if (lane != 0) return;
  if (*bad != 0u) Q = P = __longlong_as_double(0x7ff8000000000000ll);
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
  if (g.chain_elems > 0xffffffffull) return COULPS_EINVAL;  // 32-bit offsets
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The work must go to the current device, whose array address is used.
  // The stream's device is queried only outside a stream capture (the query
  // would invalidate a capture in global mode); the legacy default stream is
  // always the current device's.
  if (s != nullptr) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
      cudaGetLastError();
      return COULPS_ECUDA;
    }
    if (cs == cudaStreamCaptureStatusNone) {
      int dev = 0, sdev = 0;
      if (cudaGetDevice(&dev) != cudaSuccess || cudaStreamGetDevice(s, &sdev) != cudaSuccess) {
        cudaGetLastError();
        return COULPS_ECUDA;
      }
      if (sdev != dev) return COULPS_EINVAL;
    }
  }
  double *scratch = nullptr;
  unsigned *bad = nullptr;
  const int st = static_scratch(&scratch, &bad);
  if (st) return st;
  if (cudaMemsetAsync(bad, 0, sizeof(unsigned), s) != cudaSuccess ||
      launch_gather_checked(g, field, site_index, q, n, scratch, nblk, bad, s) != cudaSuccess) {
    cudaGetLastError();
    return COULPS_ECUDA;
  }
  static_qpe_kernel<<<(n_chains + kQpeWarps - 1) / kQpeWarps, 32 * kQpeWarps, 0, s>>>(
      scratch, nblk, n_chains, bad, QPe);
  if (cudaGetLastError() != cudaSuccess) return COULPS_ECUDA;
  return COULPS_OK;
}
