// Tensor-core Gram sweep (paper Section 4 'gram'; batches of Section 3.1) with TF32 or BF16
// operands and FP32 accumulation in tensor memory (tcgen05).
//
// A CTA owns a tile of TA x TB pairs (a, b) with TA = TB = 128 / R, R the ranks of both sides
// zero-padded to 16, 32 or 64. Per mode slice i of core k the left-partial update
// M'_ab = sum_i A_a,i^T M_ab B_b,i is two tensor-core products with M = 128 rows:
//   MMA1 (one per b)  T[(a,al), bp]   = sum_be M_b[(a,al), be] B_b,i[be, bp]   TMEM columns b*R + bp
//   MMA2 (one per a)  D_a[(b,bp), ap] += sum_al T_a[(b,bp), al] A_a,i[al, ap]  TMEM columns 128 + a*R + ap
// T goes TMEM -> registers -> shared memory (rounded to the operand type) between the two
// products; D accumulates the n_k slices of core k in FP32 and becomes the next core's M the
// same way. The final M_d (1 x 1 per pair) is <A_a, B_b>.
//
// Shared-memory operands are K-major without swizzle: 8-row x 16-byte core matrices, rows 16
// bytes apart, core matrices 144 bytes apart along K (a 16-byte skew, so that the column
// writes of the epilogues fall on distinct banks) and SBO = (K / elements-per-16-bytes) * 144
// bytes apart along M/N. Padded rows and columns hold exact zeros, so padding never changes a
// result.
#include "t3f_internal.cuh"

namespace t3f {

namespace {

constexpr uint32_t kLBO = 144;
constexpr int kMmaThreads = 256;
constexpr uint32_t kTmemCols = 256;
constexpr uint32_t kSkew = 64;  // extra bytes between consecutive operands (16-bank shift)

// Slice operands are double-buffered unless that would not fit (TF32 at R = 64).
__host__ __device__ constexpr int slice_buffers(int kind, int R) { return (kind == 0 && R == 64) ? 1 : 2; }

struct GramMmaArgs {
  TTV A, B;
  float* out;      // [bA][bB]
  int* err;        // device error word (nullable)
  uint32_t smem_bytes;
};

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

template <int KIND, int R, typename ST>
__global__ void __launch_bounds__(kMmaThreads) k_gram_mma(const __grid_constant__ GramMmaArgs g) {
  using O = OpT<KIND>;
  constexpr int ES = O::ES;
  constexpr int T = 16 / ES;                                   // elements per 16 bytes
  constexpr int TL = 128 / R;                                  // objects per tile side
  constexpr int NBUF = slice_buffers(KIND, R);                 // slice double buffering
  constexpr uint32_t SBO = (uint32_t)(R / T) * kLBO;          // every operand has K = R
  constexpr uint32_t SZ_BIG = 16u * SBO + kSkew;               // stride of 128 x R operands (M_b, T_a)
  constexpr uint32_t SZ_SL = (uint32_t)(R / 8) * SBO + kSkew;  // stride of R x R operands (slices)
  constexpr uint32_t ID = idesc(O::FMT, R);
  constexpr int KG = R / T;                                    // K groups of T elements
  constexpr int UPT = TL * R * KG / kMmaThreads;               // staged K runs per thread and side
  constexpr int USTEP = kMmaThreads / R;
  static_assert(UPT * kMmaThreads == TL * R * KG && kMmaThreads % R == 0, "slice staging must divide evenly");

  extern __shared__ __align__(128) char sm[];
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ uint32_t s_tmem;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntb = (g.B.batch + TL - 1) / TL;
  const int a0 = (blockIdx.x / ntb) * TL, b0 = (blockIdx.x % ntb) * TL;
  const int na = min(TL, g.A.batch - a0), nb = min(TL, g.B.batch - b0);
  // regions: B slices [NBUF][TL], A slices [NBUF][TL], M_b [TL], T_a [TL]
  char* const bsl = sm;
  char* const asl = sm + NBUF * TL * SZ_SL;
  char* const mop = sm + 2 * NBUF * TL * SZ_SL;
  char* const top = mop + TL * SZ_BIG;

  for (uint32_t e = (uint32_t)tid * 16u; e < g.smem_bytes; e += kMmaThreads * 16u)
    *reinterpret_cast<uint4*>(sm + e) = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  // M_0 = 1 for every pair: element (row a*R, col 0) of every M_b
  if (tid < TL * TL) O::st(mop + (tid / TL) * SZ_BIG + eoff<ES>((tid % TL) * R, 0, SBO), 1.0f);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&s_bar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&s_bar[1])));
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&s_tmem)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  async_fence();
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = s_tmem;
  const uint32_t bar1 = su32(&s_bar[0]), bar2 = su32(&s_bar[1]);
  uint32_t ph1 = 0, ph2 = 0;
  bool pending2 = false;   // an MMA2 batch has been committed and not yet waited for
  int bad = 0;             // this thread saw a wait run out
  bool failed = false;     // block-uniform

  const int q = warp & 3, h = warp >> 2;       // TMEM lane quarter, column half
  const int row = q * 32 + lane;               // TMEM lane = operand row of this thread
  const int sr = tid % R, su = tid / R;        // staging: operand row, first K-run index
  const int d = g.A.d;

  // slice i of core k of both sides -> registers: K run j of this thread covers object
  // o = (su + j*USTEP) / KG, columns c = ((su + j*USTEP) % KG) * T + t, row sr
  float pb[UPT][T], pa[UPT][T];
  auto load_slice = [&](int k, int i) {
    const int rA0 = g.A.r[k], rA1 = g.A.r[k + 1], rB0 = g.B.r[k], rB1 = g.B.r[k + 1], n = g.A.n[k];
    const long long bA = g.A.off[k] + (long long)a0 * g.A.osz[k] + (long long)i * rA1 + sr;
    const long long bB = g.B.off[k] + (long long)b0 * g.B.osz[k] + (long long)i * rB1 + sr;
    const long long sA = (long long)n * rA1, sB = (long long)n * rB1;
#pragma unroll
    for (int j = 0; j < UPT; ++j) {
      const int w = su + j * USTEP, o = w / KG, c0 = (w % KG) * T;
#pragma unroll
      for (int t = 0; t < T; ++t) {
        const int c = c0 + t;
        pb[j][t] = (o < nb && c < rB0 && sr < rB1) ? ldc<ST>(g.B.p, bB + o * g.B.osz[k] + c * sB) : 0.0f;
        pa[j][t] = (o < na && c < rA0 && sr < rA1) ? ldc<ST>(g.A.p, bA + o * g.A.osz[k] + c * sA) : 0.0f;
      }
    }
  };
  // registers -> slice buffer s: one 16-byte store per K run (a whole core-matrix row)
  auto store_slice = [&](int s) {
#pragma unroll
    for (int j = 0; j < UPT; ++j) {
      const int w = su + j * USTEP, o = w / KG, cg = w % KG;
      const uint32_t off = (uint32_t)(sr >> 3) * SBO + (uint32_t)cg * kLBO + (uint32_t)(sr & 7) * 16u;
      *reinterpret_cast<uint4*>(bsl + (s * TL + o) * SZ_SL + off) = O::pack(pb[j]);
      *reinterpret_cast<uint4*>(asl + (s * TL + o) * SZ_SL + off) = O::pack(pa[j]);
    }
  };

  int iter = 0;
  load_slice(0, 0);
  for (int k = 0; k < d && !failed; ++k) {
    const int n = g.A.n[k];
    for (int i = 0; i < n; ++i, ++iter) {
      const int s = NBUF == 2 ? (iter & 1) : 0;
      if (NBUF == 1 && pending2) {  // the single slice buffer is still read by MMA2
        bad |= !mbar_wait(bar2, ph2);
        ph2 ^= 1u;
        pending2 = false;
      }
      store_slice(s);
      async_fence();
      tc_before();
      if (__syncthreads_or(bad)) { failed = true; break; }
      // ---- MMA1: T for every b (TMEM columns b*R .. b*R + R - 1)
      if (tid == 0) {
        tc_after();
#pragma unroll 1
        for (int b = 0; b < TL; ++b) {
          const uint32_t am = su32(mop + b * SZ_BIG), bm = su32(bsl + (s * TL + b) * SZ_SL);
#pragma unroll
          for (int kk = 0; kk < R / O::KI; ++kk)
            mma<KIND>(tmem + (uint32_t)(b * R), sdesc(am + kk * 2 * kLBO, SBO), sdesc(bm + kk * 2 * kLBO, SBO), ID,
                      kk > 0);
        }
        mma_commit(bar1);
      }
      // ---- prefetch the next slice while the products run
      {
        int k2 = k, i2 = i + 1;
        if (i2 == n) { ++k2; i2 = 0; }
        if (k2 < d) load_slice(k2, i2);
      }
      bad |= !mbar_wait(bar1, ph1);
      ph1 ^= 1u;
      if (pending2) {  // T_a is still read by the previous MMA2
        bad |= !mbar_wait(bar2, ph2);
        ph2 ^= 1u;
        pending2 = false;
      }
      tc_after();
      // ---- epilogue 1: T (rows (a, al), cols (b, bp)) -> T_a[(b, bp), al]
      {
        const int a = row / R, al = row % R;
        char* dst = top + a * SZ_BIG;
#pragma unroll
        for (int cc = 0; cc < 64; cc += 16) {
          const int c0 = h * 64 + cc;
          float v[16];
          tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
          for (int j = 0; j < 16; ++j) O::st(dst + eoff<ES>(c0 + j, al, SBO), v[j]);
        }
      }
      async_fence();
      tc_before();
      if (__syncthreads_or(bad)) { failed = true; break; }
      // ---- MMA2: D_a += T_a A_a,i for every a (TMEM columns 128 + a*R ..)
      if (tid == 0) {
        tc_after();
#pragma unroll 1
        for (int a = 0; a < TL; ++a) {
          const uint32_t am = su32(top + a * SZ_BIG), bm = su32(asl + (s * TL + a) * SZ_SL);
#pragma unroll
          for (int kk = 0; kk < R / O::KI; ++kk)
            mma<KIND>(tmem + 128u + (uint32_t)(a * R), sdesc(am + kk * 2 * kLBO, SBO),
                      sdesc(bm + kk * 2 * kLBO, SBO), ID, (i > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(bar2);
      }
      pending2 = true;
    }
    if (failed) break;
    bad |= !mbar_wait(bar2, ph2);
    ph2 ^= 1u;
    pending2 = false;
    tc_after();
    // ---- epilogue 2: D (rows (b, bp), cols (a, ap)) -> M_b[(a, ap), bp], or the Gram entries
    {
      const int b = row / R, bp = row % R;
#pragma unroll
      for (int cc = 0; cc < 64; cc += 16) {
        const int c0 = h * 64 + cc;
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + 128u + (uint32_t)c0, v);
        if (k + 1 < d) {
          char* dst = mop + b * SZ_BIG;
#pragma unroll
          for (int j = 0; j < 16; ++j) O::st(dst + eoff<ES>(c0 + j, bp, SBO), v[j]);
        } else if (bp == 0 && b < nb) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int col = c0 + j;
            if (col % R == 0 && col / R < na)
              g.out[(long long)(a0 + col / R) * g.B.batch + (b0 + b)] = v[j];
          }
        }
      }
    }
    async_fence();
    tc_before();
    if (__syncthreads_or(bad)) failed = true;
    tc_after();
  }
  if (failed) {
    // a product did not signal completion: one more bounded wait for whatever is still
    // in flight before the tensor memory is released, and report the timeout
    if (tid == 0 && g.err) atomicExch(g.err, (int)T3F_ERR_TIMEOUT);
    mbar_wait(bar1, ph1);
    if (pending2) mbar_wait(bar2, ph2);
  }
  tc_before();
  __syncthreads();
  tc_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

int pad_pow2_16(int r) { return r <= 16 ? 16 : (r <= 32 ? 32 : 64); }

// Operand regions for rank R, in this order: B slices [NBUF][TL] (R x R), A slices, M_b [TL]
// (128 x R), T_a [TL]. The square slice operands come first so that every address a
// descriptor can form -- under either assignment of its two stride fields -- stays inside
// the allocation; consecutive operands are kSkew bytes further apart than their size.
uint32_t mma_smem_bytes(int kind, int R) {
  const uint32_t T = 16u / (kind == 0 ? 4u : 2u);
  const uint32_t sbo = (uint32_t)(R / (int)T) * kLBO;
  const uint32_t TL = 128u / (uint32_t)R;
  const uint32_t big = 16u * sbo + kSkew, sl = (uint32_t)(R / 8) * sbo + kSkew;
  return 2u * (uint32_t)slice_buffers(kind, R) * TL * sl + 2u * TL * big;
}

template <int KIND, int R, typename ST>
t3f_status launch_mma(const GramMmaArgs& g0, cudaStream_t s) {
  GramMmaArgs g = g0;
  g.smem_bytes = mma_smem_bytes(KIND, R);
  constexpr int TL = 128 / R;
  const long long grid = (long long)((g.A.batch + TL - 1) / TL) * ((g.B.batch + TL - 1) / TL);
  if (grid <= 0) return T3F_OK;
  if (grid > 0x7fffffffLL) return T3F_ERR_UNSUPPORTED;
  auto kern = k_gram_mma<KIND, R, ST>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem_bytes) != cudaSuccess)
    return T3F_ERR_CUDA;
  kern<<<(unsigned)grid, kMmaThreads, g.smem_bytes, s>>>(g);
  return launch_status();
}

template <int KIND, typename ST>
t3f_status dispatch_r(int R, const GramMmaArgs& g, cudaStream_t s) {
  switch (R) {
    case 16: return launch_mma<KIND, 16, ST>(g, s);
    case 32: return launch_mma<KIND, 32, ST>(g, s);
    default: return launch_mma<KIND, 64, ST>(g, s);
  }
}

}  // namespace

bool gram_mma_supported(const TTV& A, const TTV& B, int math) {
  if (math != T3F_MATH_TF32 && math != T3F_MATH_BF16) return false;
  if (A.is_matrix || B.is_matrix) return false;
  if (A.rmax > 64 || B.rmax > 64) return false;
  if (math == T3F_MATH_TF32 && (A.dtype != T3F_F32 || B.dtype != T3F_F32)) return false;
  if (A.dtype != B.dtype) return false;
  return true;
}

t3f_status run_gram_mma(const TTV& A, const TTV& B, float* out, int math, int* err, cudaStream_t s) {
  GramMmaArgs g;
  memset(&g, 0, sizeof(g));
  g.A = A;
  g.B = B;
  g.out = out;
  g.err = err;
  const int R = pad_pow2_16(A.rmax > B.rmax ? A.rmax : B.rmax);
  if (math == T3F_MATH_TF32) return dispatch_r<0, float>(R, g, s);
  if (A.dtype == T3F_BF16) return dispatch_r<1, __nv_bfloat16>(R, g, s);
  return dispatch_r<1, float>(R, g, s);
}

}  // namespace t3f
