// 3x3x3 convolution, 16 -> 16 channels, BF16 in / FP32 accumulate, on the
// 5th-generation tensor cores (tcgen05), for the learned Stein control variate.
//
//   h[b, z, y, x, co] = bias[co] + sum_{dz,dy,dx in -1..1} sum_{ci < 16}
//                        W[dz, dy, dx, co, ci] * a[b, z+dz, y+dy, x+dx, ci]
//
// with a = 0 outside the box (zero padding).  Layout: channels last,
// a[b][z][y][x][16] BF16 (32 bytes per site), h[b][z][y][x][16] FP32.
//
// Implicit GEMM.  One tile = 128 consecutive sites of one x row (the MMA's M),
// N = 16 output channels, and K = 27 offsets x 16 input channels, issued as 27
// tcgen05.mma of shape 128 x 16 x 16 (kind::f16, BF16 operands, FP32
// accumulator in 16 TMEM columns).  The A operand of offset (dz, dy, dx) is the
// tile's x range shifted by dx in input row (y + dy, z + dz): the input rows
// (x0-1 .. x0+128) are kept in shared memory as two planes of 8 channels (16
// bytes per site), which is exactly the tensor core's K-major core-matrix
// layout without swizzle (8 rows x 16 bytes per core matrix, next 8 rows at
// +128 bytes, the second 8 channels at +plane): a shift by dx is just a +16
// byte start address.  The rows are copied by the CTA's threads with
// coalesced 16-byte loads (a row of one plane is 130 x 32 contiguous bytes)
// and 16-byte shared stores into the two planes, out-of-box rows, planes and
// x written as 0.  (TMA boxes of 8 channels made 780 copies of 16 bytes per
// tile, and the TMA unit's rate for such small pieces, about one per 2.7
// cycles per SM, set the kernel's time: 21 us per conv of 64 interleaved
// 14^3 boxes.)  A CTA walks the y range of a work item (a
// chunk of y_chunk rows of a column (b, z, x tile)), keeping 4 rows per input
// plane in a ring, so each tile loads one new row per plane, one tile ahead;
// the chunk length is chosen so that there are enough items to fill the GPU
// (short chunks re-load two halo rows per chunk).  Weights sit in shared memory in the same layout
// (prepared on the host), loaded once per CTA.  One elected thread issues the
// MMAs of tile y into one of two TMEM accumulators and commits them to an
// mbarrier while the warps read tile y-1 from the other (tcgen05.ld: 32 lanes
// = sites x 16 columns = channels per warp), add the bias and store either h
// (FP32) or tanh(h) and 1 - tanh(h)^2 (BF16).  Every wait is bounded; on a
// timeout the CTA sets the error word, waits for its own copies and MMAs
// (bounded again), frees its TMEM and returns.
#include <cstdint>
#include <cstring>

#include <cuda_bf16.h>

#include "device_common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace coulps {
namespace {

constexpr int kCvThreads = 128;       // 4 warps = the 128 TMEM lanes
constexpr int kTileX = 128;           // sites per tile (MMA M)
constexpr int kRowSites = kTileX + 2; // with the x halo
// 8 channels x 2 B per site, + 32 bytes: the planes then start 64 bytes
// apart modulo 128, so a quarter-warp's stores of 4 sites x 2 halves cover
// the 32 banks once
constexpr int kPlaneBytes = kRowSites * 16 + 32;
constexpr int kRowBytes = 2 * kPlaneBytes;               // both channel halves
constexpr int kRing = 4;                                 // input rows kept per z plane
constexpr int kABytes = 3 * kRing * kRowBytes;           // 3 planes x 4 rows
constexpr int kWBytes = 27 * 512;                        // 27 offsets x (16 x 16) BF16
// Shared memory: [header 128][A: 3 planes x 4-row ring][W 27 x 512]
constexpr int kHdr = 128;
constexpr int kAOff = kHdr;
constexpr int kWOff = kAOff + ((kABytes + 127) / 128) * 128;
constexpr int kCvSmem = kWOff + kWBytes;

// tcgen05 instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1),
// A = B = BF16 (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) |
                            ((128u >> 4) << 24);



struct CvConvArgs {
  const __nv_bfloat16 *in;  // [b][z][y][x][16] BF16
  const uint4 *wpack;  // kWBytes of weights in shared-memory order
  const float *bias;   // 16
  float *out;          // mode 0: h [b][z][y][x][16] FP32
  __nv_bfloat16 *out_a, *out_s;  // mode 1: tanh(h), 1 - tanh(h)^2, BF16
  int mode;
  int Lx, Ly, Lz, nb;
  int x_period;        // > 0: output columns x with x % x_period == x_period - 1 are 0
  int y0, y1, z0, z1;  // output rows computed: y in [y0, y1), z in [z0, z1)
  int n_cols;          // nb * (z1 - z0) * ceil(Lx / 128): one column = the y rows of (b, z, x tile)
  int y_chunk;         // rows of y per work item
  int n_items;         // n_cols * ceil((y1 - y0) / y_chunk)
  int *err;
};

// One CTA walks work items (a column (b, z, x tile) and a chunk of rows
// y0 .. y1-1) and, within an item, the tiles y = y0 .. y1-1.  Tile y needs
// input rows y-1, y, y+1 of planes z-1, z, z+1; the rows of each plane sit in
// a 4-row ring.  While tile y's 27 MMAs run (into TMEM buffer count & 1) the
// threads load row y+2 of the three planes into registers, read tile y-1 from
// the other TMEM buffer, and then store the new row into the ring slot that
// tile y-1 used; one barrier per tile publishes both.
__global__ void __launch_bounds__(kCvThreads, 3) cv_conv3d_kernel(const CvConvArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem);  // [4..5] MMA buffers, [6] weights
  volatile uint32_t *tmem_slot = reinterpret_cast<volatile uint32_t *>(smem + 64);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 80);
  unsigned char *ringp = smem + kAOff;
  const uint32_t sA = smem_addr(ringp), sW = smem_addr(smem + kWOff);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // the weights: one bulk copy (a loop of 16-byte loads per thread left every
  // CTA waiting on L2 latency before its first tile)
  if (tid == 0) {
    for (int i = 4; i < 7; ++i) mbar_init(smem_addr(&bars[i]), 1);
    *abort_flag = 0;
    fence_mbar_init();
    mbar_arrive_expect_tx(smem_addr(&bars[6]), kWBytes);
    bulk_load(smem_addr(smem + kWOff), a.wpack, kWBytes, smem_addr(&bars[6]));
  }
  if (warp == 0) {
    tmem_alloc(smem_addr((const void *)tmem_slot), 32);
    tmem_relinquish();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  // only thread 0 issues MMAs: it alone waits for the weights, before its
  // first MMA (the first rows are loaded by then)
  bool w_ok = false;
  float bias[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) bias[i] = a.bias[i];

  const int xt = (a.Lx + kTileX - 1) / kTileX;
  int64_t grow = 0;   // rows this CTA has stored (ring position)
  int64_t gtile = 0;  // tiles this CTA has issued MMAs for (TMEM buffer and phase)
  int64_t mma_issued = 0, mma_waited = 0;  // thread 0's counts, for draining after a timeout
  bool aborted = false;

  // ring slot of row g (of this CTA's sequence): 3 planes x 2 channel halves
  auto row_off = [&](int dzi, int64_t g) { return (dzi * kRing + (int)(g % kRing)) * kRowBytes; };
  // One row (input row yrow of planes z-1, z, z+1, sites x0-1 .. x0+128) is
  // 3 x 130 x 2 pieces of 16 bytes; thread t takes pieces t, t + 128, ...:
  // piece c = (plane dzi = c / 260, site j = (c % 260) / 2, half h = c % 2),
  // so a warp reads 512 contiguous bytes of one plane's row.
  constexpr int kPieces = 3 * kRowSites * 2;
  constexpr int kPer = (kPieces + kCvThreads - 1) / kCvThreads;  // 7
  auto load_row = [&](int b, int z, int yrow, int x0, uint4 (&v)[kPer]) {
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int c = tid + kCvThreads * i;
      const int dzi = c / (2 * kRowSites), j = (c % (2 * kRowSites)) >> 1, h = c & 1;
      const int zz = z + dzi - 1, x = x0 - 1 + j;
      v[i] = make_uint4(0, 0, 0, 0);
      if (c < kPieces && zz >= 0 && zz < a.Lz && yrow >= 0 && yrow < a.Ly && x >= 0 && x < a.Lx)
        v[i] = *reinterpret_cast<const uint4 *>(
            a.in + ((((size_t)b * a.Lz + zz) * a.Ly + yrow) * a.Lx + x) * 16 + 8 * h);
    }
  };
  auto store_row = [&](int64_t g, const uint4 (&v)[kPer]) {
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int c = tid + kCvThreads * i;
      if (c >= kPieces) continue;
      const int dzi = c / (2 * kRowSites), j = (c % (2 * kRowSites)) >> 1, h = c & 1;
      *reinterpret_cast<uint4 *>(ringp + row_off(dzi, g) + h * kPlaneBytes + j * 16) = v[i];
    }
  };

  auto epilogue = [&](int64_t tt, int b, int z, int y, int x0) {
    float v[16];
    tmem_ld16(tmem + (uint32_t)((tt & 1) * 16) + ((uint32_t)(32 * warp) << 16), v);
    const int x = x0 + 32 * warp + lane;
    if (x < a.Lx) {
      const size_t site = (((size_t)b * a.Lz + z) * a.Ly + y) * a.Lx + x;
      if (a.x_period > 0 && x % a.x_period == a.x_period - 1) {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = -bias[i];  // the gutter column stays 0
      }
      if (a.mode == 0) {
        float4 *o4 = reinterpret_cast<float4 *>(a.out + site * 16);
#pragma unroll
        for (int i = 0; i < 4; ++i)
          o4[i] = make_float4(v[4 * i] + bias[4 * i], v[4 * i + 1] + bias[4 * i + 1],
                              v[4 * i + 2] + bias[4 * i + 2], v[4 * i + 3] + bias[4 * i + 3]);
      } else {
        __align__(16) __nv_bfloat16 ta[16], ts[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const float t = tanhf(v[i] + bias[i]);
          ta[i] = __float2bfloat16_rn(t);
          ts[i] = __float2bfloat16_rn(1.f - t * t);
        }
        uint4 *pa = reinterpret_cast<uint4 *>(a.out_a + site * 16);
        uint4 *ps = reinterpret_cast<uint4 *>(a.out_s + site * 16);
        pa[0] = reinterpret_cast<const uint4 *>(ta)[0];
        pa[1] = reinterpret_cast<const uint4 *>(ta)[1];
        ps[0] = reinterpret_cast<const uint4 *>(ts)[0];
        ps[1] = reinterpret_cast<const uint4 *>(ts)[1];
      }
    }
  };

  const int n_chunks = (a.y1 - a.y0 + a.y_chunk - 1) / a.y_chunk;
  const int nz = a.z1 - a.z0;
  for (int item = blockIdx.x; item < a.n_items && !aborted; item += gridDim.x) {
    int r = item / n_chunks;
    const int ylo = a.y0 + (item % n_chunks) * a.y_chunk;
    const int ny = min(a.y_chunk, a.y1 - ylo);
    const int x0 = (r % xt) * kTileX;
    r /= xt;
    const int z = a.z0 + r % nz;
    const int b = r / nz;
    const int nrows = ny + 2;  // row k of the item is input row ylo - 1 + k
    // rows 0 .. 2 before the first tile (nrows >= 3), all loads in flight
    {
      uint4 v0[kPer], v1[kPer], v2[kPer];
      load_row(b, z, ylo - 1, x0, v0);
      load_row(b, z, ylo, x0, v1);
      load_row(b, z, ylo + 1, x0, v2);
      store_row(grow, v0);
      store_row(grow + 1, v1);
      store_row(grow + 2, v2);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    for (int y = 0; y < ny; ++y) {  // tile ylo + y: rows y .. y + 2 of the item
      bool ok = true;
      if (tid == 0) {
        if (!w_ok) ok = w_ok = mbar_wait_bounded(smem_addr(&bars[6]), 0);
        if (ok) {
          const int64_t tt = gtile;
          const uint32_t d = tmem + (uint32_t)((tt & 1) * 16);
          for (int o = 0; o < 27; ++o) {
            const int dzi = o / 9, dyi = (o / 3) % 3, dx = o % 3;
            const uint64_t da = smem_desc(sA + (uint32_t)row_off(dzi, grow + y + dyi) + dx * 16,
                                          kPlaneBytes, 128);
            const uint64_t db = smem_desc(sW + o * 512, 256, 128);
            mma_bf16(d, da, db, kIdesc, o > 0 ? 1u : 0u);
          }
          mma_commit(smem_addr(&bars[4 + (tt & 1)]));
          ++mma_issued;
        }
      }
      // the next row (y + 3) into registers while the MMAs run
      uint4 nv[kPer];
      const bool more = y + 3 < nrows;
      if (more) load_row(b, z, ylo + y + 2, x0, nv);
      if (y > 0) {
        const int64_t tp = gtile - 1;
        ok = ok && mbar_wait_bounded(smem_addr(&bars[4 + (tp & 1)]), (uint32_t)((tp >> 1) & 1));
        if (tid == 0 && ok) ++mma_waited;
        ok = __all_sync(0xffffffffu, ok);
        fence_after_sync();
        if (ok) epilogue(tp, b, z, ylo + y - 1, x0);
      }
      // row y + 3 takes the slot of row y - 1, which only tile y - 1 (done) read
      if (ok && more) store_row(grow + y + 3, nv);
      if (!ok) {
        if (lane == 0) atomicOr(a.err, kErrTimeout);
        *abort_flag = 1;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      fence_before_sync();
      __syncthreads();  // the new row and the free TMEM buffer, for tile y + 1
      fence_after_sync();
      ++gtile;
      if (*abort_flag) {
        aborted = true;
        break;
      }
    }
    if (aborted) break;
    // last tile of the column
    {
      const int64_t tp = gtile - 1;
      bool ok = mbar_wait_bounded(smem_addr(&bars[4 + (tp & 1)]), (uint32_t)((tp >> 1) & 1));
      if (tid == 0 && ok) ++mma_waited;
      ok = __all_sync(0xffffffffu, ok);
      fence_after_sync();
      if (ok) {
        epilogue(tp, b, z, ylo + ny - 1, x0);
      } else {
        if (lane == 0) atomicOr(a.err, kErrTimeout);
        *abort_flag = 1;
      }
      fence_before_sync();
      __syncthreads();  // the ring and both TMEM buffers are free for the next item
      fence_after_sync();
      if (*abort_flag) {
        aborted = true;
        break;
      }
    }
    grow += nrows;
  }
  if (aborted && tid == 0) {
    // leave no copy or MMA in flight: the weights and every committed tile
    // not yet waited, in order, with bounded waits
    if (!w_ok) mbar_wait_bounded(smem_addr(&bars[6]), 0);  // its phase 0, done or not
    for (int64_t t = mma_waited; t < mma_issued; ++t)
      if (!mbar_wait_bounded(smem_addr(&bars[4 + (t & 1)]), (uint32_t)((t >> 1) & 1))) break;
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 32);
}

}  // namespace

int cv_conv3d_launch(const void *in_bf16, const void *wpack, const float *bias, float *out,
                     void *out_a, void *out_s, int nb, int Lx, int Ly, int Lz, int x_period,
                     int y0, int y1, int z0, int z1, int *err, cudaStream_t s) {
  CvConvArgs a;
  a.in = reinterpret_cast<const __nv_bfloat16 *>(in_bf16);
  a.wpack = reinterpret_cast<const uint4 *>(wpack);
  a.bias = bias;
  a.out = out;
  a.out_a = reinterpret_cast<__nv_bfloat16 *>(out_a);
  a.out_s = reinterpret_cast<__nv_bfloat16 *>(out_s);
  a.mode = out ? 0 : 1;
  a.Lx = Lx; a.Ly = Ly; a.Lz = Lz; a.nb = nb;
  a.x_period = x_period;
  a.y0 = y0; a.y1 = y1; a.z0 = z0; a.z1 = z1;
  a.n_cols = nb * (z1 - z0) * ((Lx + kTileX - 1) / kTileX);
  a.err = err;
  static bool configured = false;
  const int smem = kCvSmem + 128;  // + alignment slack
  if (!configured) {
    // the largest shared-memory carveout: the occupancy query below (and the
    // launch) then count the 3 CTAs per SM that shared memory allows
    if (cudaFuncSetAttribute(cv_conv3d_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared) != cudaSuccess ||
        cudaFuncSetAttribute(cv_conv3d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem) != cudaSuccess) {
      cudaGetLastError();
      return COULPS_ECUDA;
    }
    configured = true;
  }
  // CTAs per SM from the device's limits and the kernel's registers (the
  // occupancy query answered 1 for this kernel where shared memory allows
  // 3), computed once
  static int per_sm = 0, sms = 0;
  if (per_sm == 0) {
    int dev = 0, smem_sm = 0, regs_sm = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) !=
            cudaSuccess ||
        cudaFuncGetAttributes(&fa, cv_conv3d_kernel) != cudaSuccess) {
      cudaGetLastError();
      return COULPS_ECUDA;
    }
    const int by_smem = smem_sm / (smem + 1024);  // 1 KB reserved per CTA
    const int by_regs = regs_sm / ((fa.numRegs + 7) / 8 * 8 * kCvThreads);
    int n = by_smem < by_regs ? by_smem : by_regs;
    if (n > 8) n = 8;  // 8 x 32 TMEM columns of 512
    per_sm = n < 1 ? 1 : n;
  }
  // rows per item: whole columns when there are enough of them, else chunks
  // of at least 2 rows, so that about two items per resident CTA exist
  const int slots = sms * per_sm;
  const int ny = y1 - y0;
  a.y_chunk = ny;
  while (a.y_chunk > 2 && (int64_t)a.n_cols * ((ny + a.y_chunk - 1) / a.y_chunk) < 2 * slots)
    a.y_chunk = (a.y_chunk + 1) / 2;
  a.n_items = a.n_cols * ((ny + a.y_chunk - 1) / a.y_chunk);
  int grid = slots;
  if (grid > a.n_items) grid = a.n_items;
  if (grid < 1) return COULPS_OK;
  cv_conv3d_kernel<<<grid, kCvThreads, smem, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? COULPS_OK : COULPS_ECUDA;
}

}  // namespace coulps

extern "C" int coulps_cv_pack_weights(const float *w, uint16_t *out) {
  // w: PyTorch conv3d layout [co][ci][kz][ky][kx] (16 x 16 x 3 x 3 x 3).
  // out: 27 blocks of 256 BF16 (one per offset o = 9 kz + 3 ky + kx) in the
  // tensor core's K-major no-swizzle layout: element (co, ci) at byte
  // (co / 8) * 128 + (ci / 8) * 256 + (co % 8) * 16 + (ci % 8) * 2.
  if (!w || !out) return COULPS_EINVAL;
  for (int o = 0; o < 27; ++o)
    for (int co = 0; co < 16; ++co)
      for (int ci = 0; ci < 16; ++ci) {
        const float v = w[((co * 16 + ci) * 27) + o];
        uint32_t bits;
        std::memcpy(&bits, &v, 4);
        // round to nearest even BF16
        const uint32_t lsb = (bits >> 16) & 1u;
        uint16_t bf = (uint16_t)((bits + 0x7FFFu + lsb) >> 16);
        if ((bits & 0x7F800000u) == 0x7F800000u) bf = (uint16_t)(bits >> 16);  // inf / nan
        const int byte = o * 512 + (co / 8) * 128 + (ci / 8) * 256 + (co % 8) * 16 + (ci % 8) * 2;
        out[byte / 2] = bf;
      }
  return COULPS_OK;
}

extern "C" int coulps_cv_conv3d(const void *in_bf16, const void *wpack, const float *bias,
                                float *out, int nb, int Lx, int Ly, int Lz, int x_period,
                                int *err, void *stream) {
  if (!in_bf16 || !wpack || !bias || !out || !err) return COULPS_EINVAL;
  if (nb < 1 || Lx < 1 || Ly < 1 || Lz < 1 || x_period < 0) return COULPS_EINVAL;
  if ((int64_t)nb * Lz * ((Lx + 127) / 128) > 0x7fffffff) return COULPS_EINVAL;
  const uintptr_t align = reinterpret_cast<uintptr_t>(in_bf16) | reinterpret_cast<uintptr_t>(wpack) |
                          reinterpret_cast<uintptr_t>(out);
  if (align & 15) return COULPS_EINVAL;
  return coulps::cv_conv3d_launch(in_bf16, wpack, bias, out, nullptr, nullptr, nb, Lx, Ly, Lz,
                                  x_period, 0, Ly, 0, Lz, err, static_cast<cudaStream_t>(stream));
}

extern "C" int coulps_cv_conv3d_tanh(const void *in_bf16, const void *wpack, const float *bias,
                                     void *a_bf16, void *s_bf16, int nb, int Lx, int Ly, int Lz,
                                     int x_period, int *err, void *stream) {
  if (!in_bf16 || !wpack || !bias || !a_bf16 || !s_bf16 || !err) return COULPS_EINVAL;
  if (nb < 1 || Lx < 1 || Ly < 1 || Lz < 1 || x_period < 0) return COULPS_EINVAL;
  if ((int64_t)nb * Lz * ((Lx + 127) / 128) > 0x7fffffff) return COULPS_EINVAL;
  const uintptr_t align = reinterpret_cast<uintptr_t>(in_bf16) | reinterpret_cast<uintptr_t>(wpack) |
                          reinterpret_cast<uintptr_t>(a_bf16) | reinterpret_cast<uintptr_t>(s_bf16);
  if (align & 15) return COULPS_EINVAL;
  return coulps::cv_conv3d_launch(in_bf16, wpack, bias, nullptr, a_bf16, s_bf16, nb, Lx, Ly, Lz,
                                  x_period, 0, Ly, 0, Lz, err, static_cast<cudaStream_t>(stream));
}

extern "C" int coulps_cv_conv3d_tanh_rows(const void *in_bf16, const void *wpack,
                                          const float *bias, void *a_bf16, void *s_bf16, int nb,
                                          int Lx, int Ly, int Lz, int x_period, int y0, int y1,
                                          int z0, int z1, int *err, void *stream) {
  if (!in_bf16 || !wpack || !bias || !a_bf16 || !s_bf16 || !err) return COULPS_EINVAL;
  if (nb < 1 || Lx < 1 || Ly < 1 || Lz < 1 || x_period < 0) return COULPS_EINVAL;
  if (y0 < 0 || y1 > Ly || y0 >= y1 || z0 < 0 || z1 > Lz || z0 >= z1) return COULPS_EINVAL;
  if ((int64_t)nb * Lz * ((Lx + 127) / 128) > 0x7fffffff) return COULPS_EINVAL;
  const uintptr_t align = reinterpret_cast<uintptr_t>(in_bf16) | reinterpret_cast<uintptr_t>(wpack) |
                          reinterpret_cast<uintptr_t>(a_bf16) | reinterpret_cast<uintptr_t>(s_bf16);
  if (align & 15) return COULPS_EINVAL;
  return coulps::cv_conv3d_launch(in_bf16, wpack, bias, nullptr, a_bf16, s_bf16, nb, Lx, Ly, Lz,
                                  x_period, y0, y1, z0, z1, err, static_cast<cudaStream_t>(stream));
}
