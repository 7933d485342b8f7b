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

struct GramMmaArgs {
  TTV A, B;
  float* out;      // [bA][bB]
  int* err;        // device error word (nullable)
  uint32_t o_mop, o_top, o_as, smem_bytes;  // region offsets (the B slices start at 0)
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
};
template <>
struct OpT<1> {
  static constexpr int ES = 2;
  static constexpr uint32_t FMT = 1;
  static constexpr int KI = 16;
  static __device__ __forceinline__ void st(char* p, float v) {
    *reinterpret_cast<__nv_bfloat16*>(p) = __float2bfloat16_rn(v);
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
  constexpr int T = 16 / ES;
  constexpr int TL = 128 / R;                                  // objects per tile side
  constexpr uint32_t SBO = (uint32_t)(R / T) * kLBO;          // every operand has K = R
  constexpr uint32_t SZ_BIG = 16u * SBO;                       // 128 x R operand (M_b, T_a)
  constexpr uint32_t SZ_SL = (uint32_t)(R / 8) * SBO;          // R x R operand (slices)
  constexpr uint32_t ID = idesc(O::FMT, R);
  constexpr int PER = TL * R * R / kMmaThreads;               // staged elements per thread and side
  static_assert(PER * kMmaThreads == TL * R * R, "slice staging must divide evenly");

  extern __shared__ __align__(128) char sm[];
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ uint32_t s_tmem;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntb = (g.B.batch + TL - 1) / TL;
  const int a0 = (blockIdx.x / ntb) * TL, b0 = (blockIdx.x % ntb) * TL;
  const int na = min(TL, g.A.batch - a0), nb = min(TL, g.B.batch - b0);
  char* bsl = sm;                 // TL operands B_b,i: rows bp, K = be
  char* asl = sm + g.o_as;        // TL operands A_a,i: rows ap, K = al
  char* mop = sm + g.o_mop;       // TL operands M_b: rows (a, al), K = be
  char* top = sm + g.o_top;       // TL operands T_a: rows (b, bp), K = al

  for (uint32_t e = (uint32_t)tid * 16u; e < g.smem_bytes; e += kMmaThreads * 16u)
    *reinterpret_cast<uint4*>(sm + e) = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  // M_0 = 1 for every pair: element (row a*R, col 0) of every M_b
  if (tid < TL * TL) O::st(mop + (tid / TL) * SZ_BIG + eoff<ES>((tid % TL) * R, 0, SBO), 1.0f);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&s_bar)));
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
  const uint32_t bar = su32(&s_bar);
  uint32_t phase = 0;
  bool failed = false;  // block-uniform: set when a tensor-core wait ran out

  // per-thread staging coordinates (identical for both sides): element e = tid + j*256 of
  // the TL x R x R block is (object o, column-of-K c, row r) = (e / R^2, (e / R) % R, e % R)
  const int q = warp & 3, h = warp >> 2;       // TMEM lane quarter, column half
  const int row = q * 32 + lane;               // TMEM lane = operand row of this thread
  const int d = g.A.d;

  for (int k = 0; k < d; ++k) {
    const int rA0 = g.A.r[k], rA1 = g.A.r[k + 1], rB0 = g.B.r[k], rB1 = g.B.r[k + 1], n = g.A.n[k];
    const long long baseA = g.A.off[k] + (long long)a0 * g.A.osz[k];
    const long long baseB = g.B.off[k] + (long long)b0 * g.B.osz[k];
    const long long oszA = g.A.osz[k], oszB = g.B.osz[k];
    for (int i = 0; i < n; ++i) {
      // ---- stage the slices B_b,i (row bp, col be) and A_a,i (row ap, col al)
      float vb[PER], va[PER];
#pragma unroll
      for (int j = 0; j < PER; ++j) {
        const int e = tid + j * kMmaThreads;
        const int o = e / (R * R), c = (e / R) % R, r = e % R;
        vb[j] = (o < nb && c < rB0 && r < rB1) ? ldc<ST>(g.B.p, baseB + o * oszB + ((long long)c * n + i) * rB1 + r)
                                               : 0.0f;
        va[j] = (o < na && c < rA0 && r < rA1) ? ldc<ST>(g.A.p, baseA + o * oszA + ((long long)c * n + i) * rA1 + r)
                                               : 0.0f;
      }
#pragma unroll
      for (int j = 0; j < PER; ++j) {
        const int e = tid + j * kMmaThreads;
        const int o = e / (R * R), c = (e / R) % R, r = e % R;
        const uint32_t off = eoff<ES>(r, c, SBO);
        O::st(bsl + o * SZ_SL + off, vb[j]);
        O::st(asl + o * SZ_SL + off, va[j]);
      }
      async_fence();
      tc_before();
      __syncthreads();
      // ---- MMA1: T for every b
      if (tid == 0) {
        tc_after();
#pragma unroll 1
        for (int b = 0; b < TL; ++b) {
          const uint32_t am = su32(mop + b * SZ_BIG), bm = su32(bsl + b * SZ_SL);
#pragma unroll
          for (int kk = 0; kk < R / O::KI; ++kk)
            mma<KIND>(tmem + (uint32_t)(b * R), sdesc(am + kk * 2 * kLBO, SBO), sdesc(bm + kk * 2 * kLBO, SBO), ID,
                      kk > 0);
        }
        mma_commit(bar);
      }
      failed = __syncthreads_or(!mbar_wait(bar, phase)) != 0;
      phase ^= 1u;
      tc_after();
      if (failed) break;
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
      __syncthreads();
      // ---- MMA2: D_a += T_a A_a,i for every a
      if (tid == 0) {
        tc_after();
#pragma unroll 1
        for (int a = 0; a < TL; ++a) {
          const uint32_t am = su32(top + a * SZ_BIG), bm = su32(asl + a * SZ_SL);
#pragma unroll
          for (int kk = 0; kk < R / O::KI; ++kk)
            mma<KIND>(tmem + 128u + (uint32_t)(a * R), sdesc(am + kk * 2 * kLBO, SBO),
                      sdesc(bm + kk * 2 * kLBO, SBO), ID, (i > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(bar);
      }
      failed = __syncthreads_or(!mbar_wait(bar, phase)) != 0;
      phase ^= 1u;
      tc_after();
      if (failed) break;
    }
    if (failed) break;
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
    __syncthreads();
    tc_after();
  }
  if (failed) {
    // a product did not signal completion: give it one more bounded wait before the
    // tensor memory is released, and report the timeout
    if (tid == 0 && g.err) atomicExch(g.err, (int)T3F_ERR_TIMEOUT);
    mbar_wait(bar, phase);
  }
  tc_before();
  __syncthreads();
  tc_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

int pad_pow2_16(int r) { return r <= 16 ? 16 : (r <= 32 ? 32 : 64); }

template <int KIND>
constexpr uint32_t es_of() { return KIND == 0 ? 4u : 2u; }

// Operand regions for rank R, in this order: B slices (TL x R x R), A slices, M (TL x 128 x R),
// T (TL x 128 x R). The square slice operands come first so that every address a descriptor
// can form -- under either assignment of the two stride fields -- stays inside the allocation.
void mma_layout(int kind, int R, uint32_t* o_as, uint32_t* o_mop, uint32_t* o_top, uint32_t* total) {
  const uint32_t T = 16u / (kind == 0 ? 4u : 2u);
  const uint32_t sbo = (uint32_t)(R / (int)T) * kLBO;
  const uint32_t TL = 128u / (uint32_t)R;
  const uint32_t big = TL * 16u * sbo, sl = TL * (uint32_t)(R / 8) * sbo;
  *o_as = sl;
  *o_mop = 2u * sl;
  *o_top = 2u * sl + big;
  *total = 2u * sl + 2u * big;
}

template <int KIND, int R, typename ST>
t3f_status launch_mma(const GramMmaArgs& g0, cudaStream_t s) {
  GramMmaArgs g = g0;
  mma_layout(KIND, R, &g.o_as, &g.o_mop, &g.o_top, &g.smem_bytes);
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
