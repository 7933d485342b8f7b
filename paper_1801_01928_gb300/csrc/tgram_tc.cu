// Gram matrix of tangent vectors on the tensor cores (paper Section 3.2, tailored operations
// on one tangent space): G[a][b] = sum_k <dA_a,k, dB_b,k> as a split-K TF32 product with FP32
// accumulation in tensor memory.
//
// Core k of a packed batch is a row-major [batch][size_k] FP32 matrix, so the Gram matrix is
// sum_k A_k B_k^T, a dense contraction with K = sum_k size_k (about 2.8e5 per object for a
// rank-32 point with d = 20, n = 16). A CTA owns a 128 x 128 tile of pairs and one K range:
//   * one thread issues 2D TMA loads (cp.async.bulk.tensor, 128-byte swizzle) of 128 rows x
//     32 FP32 columns of A_k and B_k into a ring of stages (B is not loaded when the tile is a
//     diagonal tile of a self Gram matrix: both operands read the same stage);
//   * one thread issues tcgen05.mma kind::tf32 (M = N = 128, K = 8 per instruction, the stage's
//     four K steps advance the descriptor start inside the swizzle span) into a 128-column
//     FP32 accumulator in tensor memory and frees each stage with tcgen05.commit;
//   * four warps read the accumulator back (tcgen05.ld, one lane quarter per warp) and write
//     the CTA's partial tile; a second kernel sums the splits in a fixed order.
// The tensor cores read the FP32 operands as TF32 (the low mantissa bits are ignored).
// Rows past the batch and columns past size_k are zero-filled by the TMA unit. Every
// mbarrier wait is bounded (about one second); a wait that runs out records T3F_ERR_TIMEOUT
// in the error word, the copies still in flight are waited for (bounded) and the tensor
// memory is released before the CTA exits.
#include <cuda.h>  // CUtensorMap and its enums (the encoder is fetched from the driver)
#include <string.h>

#include <algorithm>
#include <mutex>

#include "t3f_internal.cuh"

namespace t3f {

namespace {

constexpr int kStages = 6;
constexpr int kBoxK = 32;                               // FP32 columns per stage (128 bytes)
constexpr int kTile = 128;                              // rows (objects) per tile side
constexpr uint32_t kTileBytes = kTile * kBoxK * 4;      // 16 KB
constexpr int kMaxCoresTc = 32;
constexpr int kTcThreads = 128;
constexpr uint32_t kTmemCols = 128;
constexpr size_t kTcSmem = 2 * kStages * kTileBytes + 1024;  // + alignment slack

struct TGramTcArgs {
  CUtensorMap mapA[kMaxCoresTc];
  CUtensorMap mapB[kMaxCoresTc];
  long long ksz[kMaxCoresTc];
  long long nchunks, cper;  // chunks in all, chunks per split
  int d, bA, bB, nsplit, tilesB, self;
  float* part;  // [nsplit][bA][bB]
  int* err;
};

__device__ __forceinline__ uint32_t su32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait (about one second at 2 GHz); false when it ran out
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity))
    if (clock64() - t0 > (1ll << 31)) return false;
  return true;
}

// SW128 K-major operand: 8-row groups 1024 bytes apart, rows of 128 bytes
__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | (1ull << 16) | ((uint64_t)(1024u >> 4) << 32) | (1ull << 46) |
         (2ull << 61);
}

// D = F32, A = B = TF32, both K-major, M = 128, N = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

// Walk the chunks (core k, column x) with global chunk indices [c0, c1) in order. Core k
// holds ceil(size_k / 32) chunks at columns 0, 32, ...; a chunk never crosses a core or a
// split boundary (columns past size_k are zero-filled by the TMA unit). f(c, k, x) returns
// false to stop; returns the number of chunks visited.
template <typename F>
__device__ __forceinline__ int for_chunks(const TGramTcArgs& g, long long c0, long long c1, F f) {
  int c = 0;
  long long first = 0;  // global index of core k's first chunk
  for (int k = 0; k < g.d && first < c1; ++k) {
    const long long nk = (g.ksz[k] + kBoxK - 1) / kBoxK;
    const long long lo = max(c0, first), hi = min(c1, first + nk);
    for (long long q = lo; q < hi; ++q) {
      if (!f(c, k, (int)((q - first) * kBoxK))) return c;
      ++c;
    }
    first += nk;
  }
  return c;
}

__global__ void __launch_bounds__(kTcThreads, 1) k_tgram_tc(const __grid_constant__ TGramTcArgs g) {
  extern __shared__ char smraw[];
  char* sm = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  char* tA = sm;
  char* tB = sm + kStages * kTileBytes;
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], accb;
  __shared__ uint32_t s_tmem;
  __shared__ int s_bad, s_issued;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int split = blockIdx.x % g.nsplit, tile = blockIdx.x / g.nsplit;
  const int a0 = (tile / g.tilesB) * kTile, b0 = (tile % g.tilesB) * kTile;
  const bool one_operand = g.self && a0 == b0;
  const long long e0 = (long long)split * g.cper, e1 = min(g.nchunks, e0 + g.cper);

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&empty[s])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&accb)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_bad = 0;
    s_issued = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&s_tmem)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  // warp 0 lane 0: producer; warp 1 lane 0: MMA issuer. The other lanes of these two warps
  // park at __syncwarp (not in a divergent spin beside the working lane).
  if (warp == 0 && lane == 0) {
    // ---- producer: TMA loads into the stage ring
    const uint32_t bytes = one_operand ? kTileBytes : 2 * kTileBytes;
    bool ok = true;
    const int issued = for_chunks(g, e0, e1, [&](int c, int k, int x) {
      const int s = c % kStages, u = c / kStages;
      if (u > 0 && !mbar_wait(su32(&empty[s]), (uint32_t)((u - 1) & 1))) {
        ok = false;
        return false;
      }
      const uint32_t fb = su32(&full[s]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(bytes) : "memory");
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
              su32(tA + s * kTileBytes)),
          "l"(reinterpret_cast<uint64_t>(&g.mapA[k])), "r"(x), "r"(a0), "r"(fb)
          : "memory");
      if (!one_operand)
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
                su32(tB + s * kTileBytes)),
            "l"(reinterpret_cast<uint64_t>(&g.mapB[k])), "r"(x), "r"(b0), "r"(fb)
            : "memory");
      return true;
    });
    s_issued = issued;
    if (!ok) atomicExch(&s_bad, 1);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    bool ok = true;
    for_chunks(g, e0, e1, [&](int c, int, int) {
      const int s = c % kStages, u = c / kStages;
      if (!mbar_wait(su32(&full[s]), (uint32_t)(u & 1))) {
        ok = false;
        return false;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t da = desc_sw128(su32(tA + s * kTileBytes));
      const uint64_t db = one_operand ? da : desc_sw128(su32(tB + s * kTileBytes));
#pragma unroll
      for (int kk = 0; kk < kBoxK / 8; ++kk) {
        const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da + (uint64_t)(kk * 2)), "l"(db + (uint64_t)(kk * 2)), "r"(kIdesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       su32(&empty[s]))
                   : "memory");
      return true;
    });
    if (!ok) atomicExch(&s_bad, 1);
    // arrives once every product issued above has completed
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(&accb))
                 : "memory");
  }
  if (warp < 2) __syncwarp();
  // ---- epilogue: all four warps
  const bool acc_ok = mbar_wait(su32(&accb), 0u);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  const bool good = acc_ok && !s_bad && s_issued > 0;
  const int row = warp * 32 + lane;
  const int a = a0 + row;
  float* P = g.part + (long long)split * g.bA * g.bB;
#pragma unroll 1
  for (int c0 = 0; c0 < kTile; c0 += 16) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0)
        : "memory");
    if (a < g.bA) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int b = b0 + c0 + j;
        if (b < g.bB) P[(long long)a * g.bB + b] = good ? __uint_as_float(r[j]) : 0.0f;
      }
    }
  }
  if (tid == 0) {
    if (!good && s_issued > 0 && g.err) atomicExch(g.err, (int)T3F_ERR_TIMEOUT);
    // copies still in flight (a consumer that stopped early): wait for the last fill of
    // every stage before the shared memory is released
    const int issued = s_issued;
    for (int c = max(0, issued - kStages); c < issued; ++c) mbar_wait(su32(&full[c % kStages]), (uint32_t)((c / kStages) & 1));
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                              const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encoder() {
  static std::mutex mu;
  static EncodeFn fn = nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// 2D map over core k of a packed batch: dims {size_k, batch}, box {32, 128}, 128-byte swizzle
bool encode_core(CUtensorMap* m, const TTV& v, int k) {
  EncodeFn enc = encoder();
  if (!enc) return false;
  const long long sz = v.osz[k];
  void* base = static_cast<float*>(v.p) + v.off[k];
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (sz * 4) % 16 != 0) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)sz, (cuuint64_t)v.batch};
  const cuuint64_t strides[1] = {(cuuint64_t)sz * 4};
  const cuuint32_t box[2] = {(cuuint32_t)kBoxK, (cuuint32_t)kTile};
  const cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// SM count of the current device (looked up once per device index).
int dev_sms() {
  static int cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 152;
  }
  if (cache[dev] <= 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      return 152;
    }
    cache[dev] = v;
  }
  return cache[dev];
}

struct TcPlan {
  int tilesA, tilesB, nsplit;
  long long nchunks, cper;
  size_t part_off, mid_off, total;
};

TcPlan tc_plan(const TTV& A, const TTV& B) {
  TcPlan p;
  p.nchunks = 0;
  for (int k = 0; k < A.d; ++k) p.nchunks += (A.osz[k] + kBoxK - 1) / kBoxK;
  p.tilesA = (A.batch + kTile - 1) / kTile;
  p.tilesB = (B.batch + kTile - 1) / kTile;
  const long long tiles = (long long)p.tilesA * p.tilesB;
  long long ns = ((long long)dev_sms() + tiles - 1) / tiles;  // one CTA per SM in all
  ns = std::min(ns, (p.nchunks + 3) / 4);           // at least four chunks per split
  ns = std::max(ns, 1LL);
  p.cper = (p.nchunks + ns - 1) / ns;
  p.nsplit = (int)((p.nchunks + p.cper - 1) / p.cper);
  p.part_off = kWsHeader;
  p.mid_off = p.part_off + align256(sizeof(float) * (size_t)p.nsplit * A.batch * B.batch);
  p.total = p.mid_off + ws_split_reduce((long long)A.batch * B.batch);
  return p;
}

}  // namespace

size_t ws_tangent_gram_tc(const TTV& A, const TTV& B) { return tc_plan(A, B).total; }

// TF32 tensor-core Gram of tangent coordinates; T3F_ERR_UNSUPPORTED when a core block is not
// TMA-addressable (16-byte aligned base, rows a multiple of 16 bytes) or d > 32.
t3f_status run_tangent_gram_tc(const TTV& A, const TTV& B, float* G, void* ws, size_t ws_bytes, cudaStream_t s) {
  if (A.d > kMaxCoresTc) return T3F_ERR_UNSUPPORTED;
  const TcPlan p = tc_plan(A, B);
  T3F_CHECK(check_ws(ws, ws_bytes, p.total));
  // Large (8 KB of tensor maps): built on the host and passed by value. The maps of the last
  // pair of operands are kept, so a repeated call on the same buffers and shapes (the usual
  // case in an iteration) encodes nothing.
  static TGramTcArgs g;
  static struct {
    const void *pA, *pB;
    int d, bA, bB, dev;
    long long osz[kMaxCoresTc];
    bool valid;
  } key;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return T3F_ERR_CUDA;
  }
  bool same = key.valid && key.pA == A.p && key.pB == B.p && key.d == A.d && key.bA == A.batch && key.bB == B.batch &&
              key.dev == dev;
  for (int k = 0; same && k < A.d; ++k) same = key.osz[k] == A.osz[k];
  if (!same) {
    key.valid = false;
    memset(&g, 0, sizeof(g));
    for (int k = 0; k < A.d; ++k) {
      if (!encode_core(&g.mapA[k], A, k) || !encode_core(&g.mapB[k], B, k)) return T3F_ERR_UNSUPPORTED;
      g.ksz[k] = A.osz[k];
      key.osz[k] = A.osz[k];
    }
    key.pA = A.p;
    key.pB = B.p;
    key.d = A.d;
    key.bA = A.batch;
    key.bB = B.batch;
    key.dev = dev;
    key.valid = true;
  }
  g.nchunks = p.nchunks;
  g.cper = p.cper;
  g.d = A.d;
  g.bA = A.batch;
  g.bB = B.batch;
  g.nsplit = p.nsplit;
  g.tilesB = p.tilesB;
  g.self = (A.p == B.p && A.batch == B.batch) ? 1 : 0;
  g.part = reinterpret_cast<float*>(static_cast<char*>(ws) + p.part_off);
  g.err = static_cast<int*>(ws);
  if (cudaMemsetAsync(ws, 0, sizeof(int), s) != cudaSuccess) return T3F_ERR_CUDA;
  if (cudaFuncSetAttribute(k_tgram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem) != cudaSuccess)
    return T3F_ERR_CUDA;
  const long long grid = (long long)p.tilesA * p.tilesB * p.nsplit;
  if (grid > 0x7fffffffLL) return T3F_ERR_UNSUPPORTED;
  k_tgram_tc<<<(unsigned)grid, kTcThreads, kTcSmem, s>>>(g);
  T3F_CHECK(launch_status());
  return run_split_reduce(g.part, p.nsplit, (long long)A.batch * B.batch,
                          reinterpret_cast<float*>(static_cast<char*>(ws) + p.mid_off), G, s);
}

}  // namespace t3f
