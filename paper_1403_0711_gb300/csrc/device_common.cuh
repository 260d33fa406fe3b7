// Device helpers shared by the sweep and measurement kernels.
//
//   philox4x32_10     counter-based generator of Salmon, Moraes, Dror & Shaw
//                     (SC'11), 10 rounds, Weyl key schedule.
//   hb_noise_*        the random term -erfc^-1(2r)/sqrt(3) of the heatbath
//                     update Eq. (phi), for r = (w + 1/2) 2^-32, w a 32-bit
//                     Philox word.  For 2r > 1 it uses
//                     erfc^-1(2r) = -erfc^-1(2 - 2r) so that the argument of
//                     erfc^-1 is always the small side, u in (0, 1].
//   mbar_* / tma_*    inline-PTX wrappers for mbarrier and cp.async.bulk.tensor
//                     (TMA).  Every wait is bounded by wall-clock time read
//                     from %globaltimer; a wait that gives up returns false and
//                     the caller records COULPS_ERR_TIMEOUT.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "internal.h"

namespace coulps {

// The dynamic shared-memory window rounded up to a 128-byte boundary (TMA
// destinations).  The offset is added to the __shared__ array itself rather
// than through an integer round trip, so the compiler keeps this pointer and
// everything derived from it in the shared address space (32-bit shared
// loads and stores instead of generic ones).
__device__ __forceinline__ unsigned char *align_smem128(unsigned char *raw) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(raw);
  return raw + ((128u - (a & 127u)) & 127u);
}

// Longest a single mbarrier wait may spin before giving up (ns).
constexpr uint64_t kWaitLimitNs = 2000000000ull;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKeys &K) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ K.k[2 * r], (uint32_t)p1,
                   (uint32_t)(p0 >> 32) ^ c.w ^ K.k[2 * r + 1], (uint32_t)p0);
  }
  return c;
}

// Small-side argument u = (t + 1/2) 2^-31 in (0, 1] and the sign of the
// deviate: w < 2^31 means 2r < 1 and the deviate is -erfc^-1(u)/sqrt(3).
__device__ __forceinline__ uint32_t hb_small_side(uint32_t w) {
  return ((w >> 31) ? ~w : w) & 0x7fffffffu;
}

// The two polynomials of q in FP32 Horner form; V is float or float2 (two
// sites in one packed FP32 instruction, each lane rounded exactly as the
// scalar form).
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
template <typename V> __device__ __forceinline__ V bcast(float c);
template <> __device__ __forceinline__ float bcast<float>(float c) { return c; }
template <> __device__ __forceinline__ float2 bcast<float2>(float c) { return make_float2(c, c); }

template <typename V>
__device__ __forceinline__ V erfcinv_q_main(V z) {  // z = v - 4.5, v < 9
  V q = bcast<V>(9.4230197e-12f);
  q = vfma(q, z, bcast<V>(-9.9730543e-11f));
  q = vfma(q, z, bcast<V>(-7.3713374e-10f));
  q = vfma(q, z, bcast<V>(1.8971662e-08f));
  q = vfma(q, z, bcast<V>(-9.0245905e-08f));
  q = vfma(q, z, bcast<V>(-1.2787358e-06f));
  q = vfma(q, z, bcast<V>(2.4949235e-05f));
  q = vfma(q, z, bcast<V>(-0.00014325297f));
  q = vfma(q, z, bcast<V>(-0.0016700856f));
  q = vfma(q, z, bcast<V>(0.096136749f));
  q = vfma(q, z, bcast<V>(0.95392835f));
  return q;
}

template <typename V>
__device__ __forceinline__ V erfcinv_q_tail(V z) {  // z = sqrt(v) - 3.6, v >= 9
  V q = bcast<V>(6.5457465e-07f);
  q = vfma(q, z, bcast<V>(8.3999657e-07f));
  q = vfma(q, z, bcast<V>(-4.7697853e-05f));
  q = vfma(q, z, bcast<V>(0.00027278936f));
  q = vfma(q, z, bcast<V>(-0.00080441934f));
  q = vfma(q, z, bcast<V>(0.001587657f));
  q = vfma(q, z, bcast<V>(-0.0025733677f));
  q = vfma(q, z, bcast<V>(0.0038068402f));
  q = vfma(q, z, bcast<V>(0.48145568f));
  q = vfma(q, z, bcast<V>(1.6339986f));
  return q;
}

// The heatbath deviate in FP32: erfc^-1(u) / sqrt(3) for u = (s + 1/2) 2^-31,
// s < 2^31, with the sign of the word's top bit.  Both u and
// x = 1 - u = (2^31 - 1 - s + 1/2) 2^-31 are formed from integers, so neither
// inherits the other's rounding (accurate near u = 1 and near u = 0).
// erfc^-1(u) / sqrt(3) = x q(v) with v = -log2(u (2 - u)) = -log2(u + u x);
// q is smooth in v (the change of variable of M. Giles, "Approximating the
// erfinv function", GPU Computing Gems, 2011, here in base 2) and is taken
// as a degree-10 polynomial in v - 4.5 for v < 9 and a degree-9 polynomial in
// sqrt(v) - 3.6 above (u >= 2^-32 keeps v < 32); 1/sqrt(3) is folded into
// the coefficients.  Coefficients: our own weighted least-squares fit
// (fit_erfcinv.py beside this file; fit error 5.5e-9 and 2.9e-8 relative;
// emulated FP32 evaluation 2.5e-7 relative at most).  The split at v = 9
// (u < 2^-10 or so, 1e-3 of the words) rather than 7 makes the tail rare
// enough that a warp's vote over 64 words takes it 6% of the time instead of
// 22%, for one more term in the common polynomial.  Measured against FP64
// erfc^-1 over the whole range: a few FP32 ulps.
__device__ __forceinline__ float hb_noise_f32(uint32_t w) {
  const uint32_t s = hb_small_side(w);
  const float u = fmaf(__uint2float_rn(s), 0x1p-31f, 0x1p-32f);
  const float x = fmaf(__uint2float_rn(0x7fffffffu - s), 0x1p-31f, 0x1p-32f);
  const float v = -__log2f(fmaf(u, x, u));
  float q;
  if (v < 9.0f)
    q = erfcinv_q_main(v - 4.5f);
  else
    q = erfcinv_q_tail(sqrtf(v) - 3.6f);
  // w < 2^31 (2r < 1): a negative term; the sign goes onto x (exact)
  const float xs = __uint_as_float(__float_as_uint(x) | ((~w) & 0x80000000u));
  return xs * q;
}

// hb_noise_f32 of 2 NP words (pairs (w[0], w[1]), (w[2], w[3]), ...) with one
// vote of the warp's active lanes for the tail over all of them, so the words'
// independent chains can interleave; bitwise the same per word.
template <int NP>
__device__ __forceinline__ void hb_noise_pairs_f32(const uint32_t (&w)[2 * NP], float2 (&out)[NP]) {
  const float2 scale = make_float2(0x1p-31f, 0x1p-31f), half = make_float2(0x1p-32f, 0x1p-32f);
  float2 x[NP], v[NP], q[NP];
  bool tail = false;
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const uint32_t s0 = hb_small_side(w[2 * p]), s1 = hb_small_side(w[2 * p + 1]);
    const float2 u =
        __ffma2_rn(make_float2(__uint2float_rn(s0), __uint2float_rn(s1)), scale, half);
    x[p] = __ffma2_rn(
        make_float2(__uint2float_rn(0x7fffffffu - s0), __uint2float_rn(0x7fffffffu - s1)), scale,
        half);
    const float2 t = __ffma2_rn(u, x[p], u);
    v[p] = make_float2(-__log2f(t.x), -__log2f(t.y));
    q[p] = erfcinv_q_main(__fadd2_rn(v[p], make_float2(-4.5f, -4.5f)));
    tail = tail || !(v[p].x < 9.0f) || !(v[p].y < 9.0f);
  }
  if (__any_sync(__activemask(), tail)) {
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const float2 qt = erfcinv_q_tail(
          __fadd2_rn(make_float2(sqrtf(v[p].x), sqrtf(v[p].y)), make_float2(-3.6f, -3.6f)));
      q[p].x = v[p].x < 9.0f ? q[p].x : qt.x;
      q[p].y = v[p].y < 9.0f ? q[p].y : qt.y;
    }
  }
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const float2 xs =
        make_float2(__uint_as_float(__float_as_uint(x[p].x) | ((~w[2 * p]) & 0x80000000u)),
                    __uint_as_float(__float_as_uint(x[p].y) | ((~w[2 * p + 1]) & 0x80000000u)));
    out[p] = __fmul2_rn(xs, q[p]);
  }
}

__device__ __forceinline__ double hb_noise_f64(uint32_t w) {
  const double u = ((double)hb_small_side(w) + 0.5) * 0x1p-31;
  const double y = erfcinv(u) * 0.57735026918962576450914878;  // 1/sqrt(3)
  return (w >> 31) ? y : -y;
}

template <typename T> struct Noise;
template <> struct Noise<float> {
  __device__ __forceinline__ static float of(uint32_t w) { return hb_noise_f32(w); }
};
template <> struct Noise<double> {
  __device__ __forceinline__ static double of(uint32_t w) { return hb_noise_f64(w); }
};

// ---------------------------------------------------------------------------
// mbarrier / TMA
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// try_wait with a suspend-time hint: a thread whose phase is not complete
// sleeps until it completes or the hint (ns) elapses, instead of spinning
// through issue slots that the CTA's other warps need.
constexpr uint32_t kSuspendHintNs = 1000000u;
__device__ __forceinline__ bool mbar_try_wait_sleep(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "n"(kSuspendHintNs)
      : "memory");
  return ok != 0;
}

// Wait until the phase with the given parity has completed, or give up after
// kWaitLimitNs (each try sleeps at most kSuspendHintNs, so the limit is
// overshot by at most 32 hints).  Returns true on completion.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  for (;;) {
#pragma unroll 1
    for (int i = 0; i < 32; ++i)
      if (mbar_try_wait_sleep(bar, parity)) return true;
    if (global_timer_ns() - t0 > kWaitLimitNs) return false;
  }
}

// 4D tiled TMA load global -> shared, completion signalled on `bar`.
// The innermost coordinate c0 must be a multiple of 16 bytes / element size;
// every caller in this library passes c0 = 0.
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1,
                                            int c2, int c3, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap *map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One chain's (Q, P) from its nblk CTA partials [chain][nblk][2], in a fixed
// order: lane l of a warp adds blocks l, l + 32, ..., then the warp's
// butterfly sum.  Every lane of the warp must call it.
__device__ __forceinline__ void chain_QP(const double *__restrict__ partials, int nblk, int chain,
                                         int lane, double &Q, double &P) {
  Q = 0.0;
  P = 0.0;
  for (int b = lane; b < nblk; b += 32) {
    Q += partials[2 * ((size_t)chain * nblk + b) + 0];
    P += partials[2 * ((size_t)chain * nblk + b) + 1];
  }
  Q = warp_sum(Q);
  P = warp_sum(P);
}

// One sample of one chain (or system): e = Q^2 - P formed in FP64 (the
// cancelling difference of Eq. (nsum2)), then the running sums, the batch
// sums (kBatchMin..2*kBatchMin batches; neighbours merge and the batch length
// doubles when 2*kBatchMin complete) and, if row != nullptr, the log row.
// Adds the sample e to one chain's running sums and batch means.
__device__ __forceinline__ void record_value(double *st, double e, int *err) {
  if (!isfinite(e)) atomicOr(err, kErrNonFinite);
  st[kStatLast] = e;
  st[kStatN] += 1.0;
  st[kStatSum] += e;
  st[kStatSum2] += e * e;
  st[kStatCurSum] += e;
  st[kStatCurN] += 1.0;
  if (st[kStatCurN] >= st[kStatBatchLen]) {
    int nb = (int)st[kStatNBatch];
    st[kStatBatch0 + nb] = st[kStatCurSum];
    st[kStatCurSum] = 0.0;
    st[kStatCurN] = 0.0;
    ++nb;
    if (nb == 2 * kBatchMin) {
      for (int i = 0; i < kBatchMin; ++i)
        st[kStatBatch0 + i] = st[kStatBatch0 + 2 * i] + st[kStatBatch0 + 2 * i + 1];
      for (int i = kBatchMin; i < 2 * kBatchMin; ++i) st[kStatBatch0 + i] = 0.0;
      nb = kBatchMin;
      st[kStatBatchLen] *= 2.0;
    }
    st[kStatNBatch] = (double)nb;
  }
}

// Eq. (nsum2) sample e = Q^2 - P, logged to row when it is not null.
__device__ __forceinline__ void record_sample(double *st, double Q, double P, double *row,
                                              int *err) {
  const double e = Q * Q - P;
  if (row != nullptr) {
    row[0] = Q;
    row[1] = P;
    row[2] = e;
  }
  record_value(st, e, err);
}

}  // namespace coulps
