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
// (x0-1 .. x0+128) arrive by TMA, each as two planes
// of 8 channels (16 bytes per site), which is exactly the tensor core's
// K-major core-matrix layout without swizzle (8 rows x 16 bytes per core
// matrix, next 8 rows at +128 bytes, the second 8 channels at +plane): a shift
// by dx is just a +16 byte start address.  Out-of-box rows, planes and x are
// zero-filled by the TMA unit.  A CTA walks the y range of a work item (a
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

namespace coulps {
namespace {

constexpr int kCvThreads = 128;       // 4 warps = the 128 TMEM lanes
constexpr int kTileX = 128;           // sites per tile (MMA M)
constexpr int kRowSites = kTileX + 2; // with the x halo
constexpr int kPlaneBytes = ((kRowSites * 16 + 127) / 128) * 128;  // 8 channels x 2 B per site
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

// Shared-memory matrix descriptor, no swizzle, K-major: start >> 4 (bits
// 0-13), leading byte offset >> 4 (K direction, bits 16-29), stride byte
// offset >> 4 (M/N direction, bits 32-45), descriptor version 1 (bit 46).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap *map, int c0, int c1,
                                            int c2, int c3, int c4, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct CvConvArgs {
  const uint4 *wpack;  // kWBytes of weights in shared-memory order
  const float *bias;   // 16
  float *out;          // mode 0: h [b][z][y][x][16] FP32
  __nv_bfloat16 *out_a, *out_s;  // mode 1: tanh(h), 1 - tanh(h)^2, BF16
  int mode;
  int Lx, Ly, Lz, nb;
  int x_period;        // > 0: output columns x with x % x_period == x_period - 1 are 0
  int n_cols;          // nb * Lz * ceil(Lx / 128): one column = all y of (b, z, x tile)
  int y_chunk;         // rows of y per work item
  int n_items;         // n_cols * ceil(Ly / y_chunk)
  int *err;
};

// One CTA walks work items (a column (b, z, x tile) and a chunk of rows
// y0 .. y1-1) and, within an item, the tiles y = y0 .. y1-1.  Tile y needs
// input rows y-1, y, y+1 of planes z-1, z, z+1; the rows of each plane sit in
// a 4-row ring, so each tile loads one new row per plane (row y+2, one tile
// ahead).  Tile y's 27 MMAs go to TMEM buffer (count & 1) while the warps read
// tile y-1 from the other buffer.
__global__ void __launch_bounds__(kCvThreads)
    cv_conv3d_kernel(const __grid_constant__ CUtensorMap tm_in, const CvConvArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem);  // [0..3] row ring, [4..5] MMA buffers
  volatile uint32_t *tmem_slot = reinterpret_cast<volatile uint32_t *>(smem + 64);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 80);
  const uint32_t sA = smem_addr(smem + kAOff), sW = smem_addr(smem + kWOff);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  for (int i = tid; i < kWBytes / 16; i += kCvThreads)
    reinterpret_cast<uint4 *>(smem + kWOff)[i] = a.wpack[i];
  if (tid == 0) {
    prefetch_tensormap(&tm_in);
    for (int i = 0; i < 6; ++i) mbar_init(smem_addr(&bars[i]), 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 0) {
    tmem_alloc(smem_addr((const void *)tmem_slot), 32);
    tmem_relinquish();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  float bias[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) bias[i] = a.bias[i];

  const int xt = (a.Lx + kTileX - 1) / kTileX;
  int64_t grow = 0;  // rows this CTA has loaded (ring position and phase)
  int64_t gtile = 0;  // tiles this CTA has issued MMAs for (TMEM buffer and phase)
  // thread 0's counts, for draining after a timeout
  int64_t rows_issued = 0, rows_waited = 0, mma_issued = 0, mma_waited = 0;
  bool aborted = false;

  // row k of a column is input row yrow = k - 1; ring slot (grow + k) % 4
  auto row_slot = [&](int64_t g) { return (int)(g % kRing); };
  auto row_parity = [&](int64_t g) { return (uint32_t)((g / kRing) & 1); };
  auto row_base = [&](int dzi, int64_t g) {
    return sA + (uint32_t)((dzi * kRing + row_slot(g)) * kRowBytes);
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

  const int n_chunks = (a.Ly + a.y_chunk - 1) / a.y_chunk;
  for (int item = blockIdx.x; item < a.n_items && !aborted; item += gridDim.x) {
    int r = item / n_chunks;
    const int ylo = (item % n_chunks) * a.y_chunk;
    const int ny = min(a.y_chunk, a.Ly - ylo);
    const int x0 = (r % xt) * kTileX;
    r /= xt;
    const int z = r % a.Lz;
    const int b = r / a.Lz;
    const int nrows = ny + 2;  // row k of the item is input row ylo - 1 + k
    auto issue_row = [&](int k) {  // thread 0
      const int64_t g = grow + k;
      const uint32_t bar = smem_addr(&bars[row_slot(g)]);
      mbar_arrive_expect_tx(bar, 6 * kRowSites * 16);
      for (int dzi = 0; dzi < 3; ++dzi)
        for (int h = 0; h < 2; ++h)
          tma_load_5d(row_base(dzi, g) + h * kPlaneBytes, &tm_in, 8 * h, x0 - 1, ylo + k - 1,
                      z + dzi - 1, b, bar);
      ++rows_issued;
    };
    auto wait_row = [&](int k) -> bool {
      const int64_t g = grow + k;
      return mbar_wait_bounded(smem_addr(&bars[row_slot(g)]), row_parity(g));
    };
    if (tid == 0)
      for (int k = 0; k < kRing && k < nrows; ++k) issue_row(k);
    bool ok = wait_row(0) && wait_row(1);
    if (tid == 0 && ok) rows_waited += 2;
    for (int y = 0; y < ny; ++y) {  // tile ylo + y
      ok = ok && wait_row(y + 2);
      if (tid == 0 && ok) {
        ++rows_waited;
        fence_after_sync();
        const int64_t tt = gtile;
        const uint32_t d = tmem + (uint32_t)((tt & 1) * 16);
        for (int o = 0; o < 27; ++o) {
          const int dzi = o / 9, dyi = (o / 3) % 3, dx = o % 3;
          const uint64_t da = smem_desc(row_base(dzi, grow + y + dyi) + dx * 16, kPlaneBytes, 128);
          const uint64_t db = smem_desc(sW + o * 512, 256, 128);
          mma_bf16(d, da, db, kIdesc, o > 0 ? 1u : 0u);
        }
        mma_commit(smem_addr(&bars[4 + (tt & 1)]));
        ++mma_issued;
      }
      if (y > 0) {
        const int64_t tp = gtile - 1;
        ok = ok && mbar_wait_bounded(smem_addr(&bars[4 + (tp & 1)]), (uint32_t)((tp >> 1) & 1));
        if (tid == 0 && ok) {
          ++mma_waited;
          // row k = y + 3 reuses the ring slot of row k = y - 1, last read by tile y - 1
          if (y + 3 < nrows) issue_row(y + 3);
        }
      }
      if (!ok) {
        atomicOr(a.err, kErrTimeout);
        *abort_flag = 1;
      }
      fence_before_sync();
      __syncthreads();
      fence_after_sync();
      if (*abort_flag) {
        aborted = true;
        break;
      }
      if (y > 0) epilogue(gtile - 1, b, z, ylo + y - 1, x0);
      fence_before_sync();
      __syncthreads();  // the TMEM buffer read above is free for tile y + 1
      fence_after_sync();
      ++gtile;
    }
    if (aborted) break;
    // last tile of the column
    {
      const int64_t tp = gtile - 1;
      ok = mbar_wait_bounded(smem_addr(&bars[4 + (tp & 1)]), (uint32_t)((tp >> 1) & 1));
      if (tid == 0 && ok) ++mma_waited;
      if (!ok) {
        atomicOr(a.err, kErrTimeout);
        *abort_flag = 1;
      }
      fence_before_sync();
      __syncthreads();
      fence_after_sync();
      if (*abort_flag) {
        aborted = true;
        break;
      }
      epilogue(tp, b, z, ylo + ny - 1, x0);
      fence_before_sync();
      __syncthreads();
      fence_after_sync();
    }
    grow += nrows;
  }
  if (aborted && tid == 0) {
    // leave no copy or MMA in flight: every row issued and every committed
    // tile not yet waited, in order, with bounded waits
    for (int64_t g = rows_waited; g < rows_issued; ++g)
      if (!mbar_wait_bounded(smem_addr(&bars[row_slot(g)]), row_parity(g))) break;
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
                     int *err, cudaStream_t s) {
  auto enc = tensor_map_encoder();
  if (!enc) return COULPS_ECUDA;
  CUtensorMap map;
  cuuint64_t dims[5] = {16, (cuuint64_t)Lx, (cuuint64_t)Ly, (cuuint64_t)Lz, (cuuint64_t)nb};
  cuuint64_t strides[4] = {32, (cuuint64_t)Lx * 32, (cuuint64_t)Lx * Ly * 32,
                           (cuuint64_t)Lx * Ly * Lz * 32};
  cuuint32_t box[5] = {8, (cuuint32_t)kRowSites, 1, 1, 1};
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(in_bf16), dims, strides,
          box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return COULPS_ECUDA;
  CvConvArgs a;
  a.wpack = reinterpret_cast<const uint4 *>(wpack);
  a.bias = bias;
  a.out = out;
  a.out_a = reinterpret_cast<__nv_bfloat16 *>(out_a);
  a.out_s = reinterpret_cast<__nv_bfloat16 *>(out_s);
  a.mode = out ? 0 : 1;
  a.Lx = Lx; a.Ly = Ly; a.Lz = Lz; a.nb = nb;
  a.x_period = x_period;
  a.n_cols = nb * Lz * ((Lx + kTileX - 1) / kTileX);
  a.err = err;
  static bool configured = false;
  const int smem = kCvSmem + 1024;
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
  a.y_chunk = Ly;
  while (a.y_chunk > 2 && (int64_t)a.n_cols * ((Ly + a.y_chunk - 1) / a.y_chunk) < 2 * slots)
    a.y_chunk = (a.y_chunk + 1) / 2;
  a.n_items = a.n_cols * ((Ly + a.y_chunk - 1) / a.y_chunk);
  int grid = slots;
  if (grid > a.n_items) grid = a.n_items;
  if (grid < 1) return COULPS_OK;
  cv_conv3d_kernel<<<grid, kCvThreads, smem, s>>>(map, a);
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
                                  x_period, err, static_cast<cudaStream_t>(stream));
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
                                  x_period, err, static_cast<cudaStream_t>(stream));
}
