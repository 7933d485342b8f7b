// tcgen05 helpers shared by the tensor-core Gram kernels (forward sweep, adjoint sweeps and
// the adjoint's gradient products): operand element formats, shared-memory and instruction
// descriptors, the MMA issue and commit forms, bounded mbarrier waits, tensor-memory loads,
// and the raw staging loads of F32 / BF16 cores.
#pragma once

#include "t3f_internal.cuh"

namespace t3f {
namespace {

// stride between K-adjacent core matrices of the forward sweep's operands (16-byte skew)
constexpr uint32_t kLBO = 144;

template <int KIND>
struct OpT;
// TF32: 4-byte elements rounded to nearest (ties away) before the tensor core reads them
template <>
struct OpT<0> {
  static constexpr int ES = 4;
  static constexpr uint32_t FMT = 2;
  static constexpr int KI = 8;  // K per instruction
  static __device__ __forceinline__ void st(char* p, float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    *reinterpret_cast<uint32_t*>(p) = r;
  }
  static __device__ __forceinline__ uint32_t cv(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return r;
  }
  static __device__ __forceinline__ uint4 pack(const float (&v)[4]) {
    return make_uint4(cv(v[0]), cv(v[1]), cv(v[2]), cv(v[3]));
  }
};
template <>
struct OpT<1> {
  static constexpr int ES = 2;
  static constexpr uint32_t FMT = 1;
  static constexpr int KI = 16;
  static __device__ __forceinline__ void st(char* p, float v) {
    *reinterpret_cast<__nv_bfloat16*>(p) = __float2bfloat16_rn(v);
  }
  static __device__ __forceinline__ uint32_t cv2(float lo, float hi) {
    const __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&b);
  }
  static __device__ __forceinline__ uint4 pack(const float (&v)[8]) {
    return make_uint4(cv2(v[0], v[1]), cv2(v[2], v[3]), cv2(v[4], v[5]), cv2(v[6], v[7]));
  }
};

// byte offset of element (row r, column k) of a K-major operand whose rows are 8-row groups SBO apart
template <int ES>
__device__ __forceinline__ uint32_t eoff(int r, int k, uint32_t sbo) {
  constexpr int T = 16 / ES;
  return (uint32_t)(r >> 3) * sbo + (uint32_t)(k / T) * kLBO + (uint32_t)(r & 7) * 16u + (uint32_t)(k % T) * ES;
}

__device__ __forceinline__ uint32_t su32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((kLBO >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// D = F32, A and B of format fmt, both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t idesc(uint32_t fmt, uint32_t n) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  if constexpr (KIND == 0) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc));
  }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.b32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the barrier phase with a bound of about one second; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity))
    if (clock64() - t0 > (1ll << 31)) return false;
  return true;
}

__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void async_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 lanes x 16 consecutive FP32 columns (lane = thread's row of the warp's lane quarter)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

template <typename ST>
__device__ __forceinline__ float ldc(const void* p, long long i) {
  return ldf<ST>(static_cast<const ST*>(p), i);
}

// Raw bits of one stored element (F32 or BF16), converted only when the slice is packed, so
// the loads of a slice stay in flight while the products run.
template <typename ST>
__device__ __forceinline__ uint32_t ld_raw(const ST* p);
template <>
__device__ __forceinline__ uint32_t ld_raw<float>(const float* p) { return __float_as_uint(__ldg(p)); }
template <>
__device__ __forceinline__ uint32_t ld_raw<__nv_bfloat16>(const __nv_bfloat16* p) {
  return (uint32_t)__ldg(reinterpret_cast<const unsigned short*>(p));
}

// T raw elements -> one 16-byte operand row (TF32: 4 x 4 bytes, BF16: 8 x 2 bytes)
template <int KIND, typename ST, int T>
__device__ __forceinline__ uint4 pack_raw(const uint32_t (&v)[T]) {
  if constexpr (KIND == 0) {
    return OpT<0>::pack({__uint_as_float(v[0]), __uint_as_float(v[1]), __uint_as_float(v[2]), __uint_as_float(v[3])});
  } else if constexpr (sizeof(ST) == 2) {
    return make_uint4(v[0] | (v[1] << 16), v[2] | (v[3] << 16), v[4] | (v[5] << 16), v[6] | (v[7] << 16));
  } else {
    return make_uint4(OpT<1>::cv2(__uint_as_float(v[0]), __uint_as_float(v[1])),
                      OpT<1>::cv2(__uint_as_float(v[2]), __uint_as_float(v[3])),
                      OpT<1>::cv2(__uint_as_float(v[4]), __uint_as_float(v[5])),
                      OpT<1>::cv2(__uint_as_float(v[6]), __uint_as_float(v[7])));
  }
}

// Two 16-lane x 8-column TMEM loads (columns c and c + 8 of lanes L..L+15): thread t gets
// lanes L + t/4 and L + 8 + t/4, columns 2(t%4) and 2(t%4)+1 of each 8-column block.
__device__ __forceinline__ void tmem_ld_16x16(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.16x256b.x1.b32 {%0,%1,%2,%3}, [%8];\n"
      "tcgen05.ld.sync.aligned.16x256b.x1.b32 {%4,%5,%6,%7}, [%9];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(taddr), "r"(taddr + 8u)
      : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t bf2(uint32_t lo, uint32_t hi) {
  const __nv_bfloat162 b = __floats2bfloat162_rn(__uint_as_float(lo), __uint_as_float(hi));
  return *reinterpret_cast<const uint32_t*>(&b);
}

// Descriptor of a K-major, non-swizzled operand with explicit strides: lbo = bytes between
// K-adjacent core matrices, sbo = bytes between 8-row groups along M / N.
__device__ __forceinline__ uint64_t sdesc2(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// TF32 product whose A operand (M = 128 rows = lanes, K along columns) is read from tensor
// memory; the FP32 values there are read as TF32 (low mantissa bits dropped).
__device__ __forceinline__ void mma_ts_tf32(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
      "r"(a_tmem), "l"(b), "r"(id), "r"(acc));
}

}  // namespace
}  // namespace t3f
