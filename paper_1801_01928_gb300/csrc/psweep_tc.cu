// project_sum sweeps on the tensor cores (paper Section 3.2; TF32 operands, FP32 accumulation
// in tensor memory): the left partials L^{(j)}_k of (U, Z_j) and the right partials R^{(j)}_k
// of (V, Z_j) for a batch of Z objects of rank <= 8 at a point X of rank <= 32.
//
// A CTA carries 16 objects through all d cores; its 128 rows are (object j, Z-rank index).
// Left step at core k (rows (j, delta)):
//   T[(j, delta), (alpha, i)] = sum_gamma L^{(j)}[alpha][gamma] Z_j[gamma][i][delta]   CUDA cores
//   L'^{(j)}[beta][delta]     = sum_{(alpha, i)} T[(j, delta), (alpha, i)] U_k[alpha][i][beta]
// the second a product with M = 128, N = 32, K = r_{k} n_k issued by one thread on the tensor
// cores (tcgen05.mma kind::tf32), the shared operand U_k staged once per core in shared memory
// as B[beta][(alpha, i)]. Right step (rows (j, gamma)):
//   T'[(j, gamma), (beta, i)] = sum_delta R^{(j)}[beta][delta] Z_j[gamma][i][delta]
//   R'^{(j)}[alpha][gamma]    = sum_{(beta, i)} T'[(j, gamma), (beta, i)] V_k[alpha][i][beta]
// T is built 4 rank indices (64 K values) at a time into one of two operand buffers while the
// tensor cores consume the other. The Z cores of the CTA's objects arrive by TMA bulk copies
// (one per object and core, rounded out to 16-byte boundaries). The partials are stored in the
// layout of the CUDA-core sweeps ([r_X][r_Z] per object and interface), so the FP32 assembly
// and gauge projection consume them unchanged.
//
// Shared-memory operands are K-major without swizzle: 8-row x 16-byte core matrices, adjacent
// along K (LBO = 128 bytes), 8-row groups SBO = (K / 4) * 128 bytes apart. Every mbarrier wait
// is bounded (about one second); a wait that runs out records T3F_ERR_TIMEOUT in the error
// word, the products in flight are waited for (bounded) and the tensor memory is released.
#include <string.h>

#include <algorithm>

#include "t3f_internal.cuh"

namespace t3f {

namespace {

constexpr int kPtThreads = 256;
constexpr int kPtObj = 16;               // objects per CTA (128 rows of 8)
constexpr int kPtRX = 32;                // X-side rank bound (N of the products)
constexpr int kPtRZ = 8;                 // Z-side rank bound
constexpr int kPtNmax = 16;              // mode bound
constexpr int kPtChunkR = 4;             // rank indices per operand chunk
constexpr int kPtKc = kPtChunkR * kPtNmax;   // K values per chunk (64)
constexpr uint32_t kPtABytes = 128u * kPtKc * 4u;            // 32 KB
constexpr uint32_t kPtBBytes = (uint32_t)kPtRX * kPtRX * kPtNmax * 4u;  // 64 KB (K up to 512)
constexpr int kPtZObj = kPtRZ * kPtNmax * kPtRZ + 8;       // floats per object landing (+ slack)
constexpr uint32_t kPtTmemCols = 32;

struct PtArgs {
  TTV Z;
  const float* X[2];             // U (left sweep) and V (right sweep) cores, packed, batch 1
  long long Xoff[T3F_MAX_D];     // shared by U and V (equal shapes)
  int rx[T3F_MAX_D + 1];
  float* st[2];                  // partial stores of the two sweeps
  long long ioff[2][T3F_MAX_D + 1];
  int nblk;                      // CTAs per direction; blocks [nblk, 2 nblk) run the right sweep
  int* err;
};

__device__ __forceinline__ uint32_t pt_smem(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ bool pt_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > (1ll << 31)) return false;
  }
}

// no-swizzle K-major descriptor: core matrices 128 bytes apart along K, 8-row groups sbo apart
__device__ __forceinline__ uint64_t pt_desc(uint32_t addr, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) |
         (1ull << 46);
}

// byte offset of element (row r, K index k) of a K-major operand with 8-row groups sbo apart
__device__ __forceinline__ uint32_t pt_off(int r, int k, uint32_t sbo) {
  return (uint32_t)(r >> 3) * sbo + (uint32_t)(k >> 2) * 128u + (uint32_t)(r & 7) * 16u + (uint32_t)(k & 3) * 4u;
}

constexpr uint32_t kPtIdesc = (1u << 4) | (2u << 7) | (2u << 10) | (((uint32_t)kPtRX >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t tf32_bits(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}

__global__ void __launch_bounds__(kPtThreads, 1) k_psweep_tc(const __grid_constant__ PtArgs a) {
  extern __shared__ __align__(128) char smem[];
  char* Abuf = smem;                                   // [2][kPtABytes]
  char* Bop = smem + 2 * kPtABytes;                    // [kPtBBytes]
  float* Zl = reinterpret_cast<float*>(Bop + kPtBBytes);          // [16][kPtZObj] landed Z cores
  float* Ls = Zl + kPtObj * kPtZObj;                   // [16][32][8] current partials (x-rank, z-rank)
  __shared__ __align__(8) uint64_t bar_mma[2], bar_z;
  __shared__ uint32_t s_tmem;
  __shared__ int s_bad;
  const TTV& Z = a.Z;
  const int d = Z.d, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int dir = (int)blockIdx.x >= a.nblk ? 1 : 0;
  const int obj0 = ((int)blockIdx.x - dir * a.nblk) * kPtObj;
  const float* Xbase = a.X[dir];
  float* st = a.st[dir];
  const long long* ioff = a.ioff[dir];
  const int nobj = min(kPtObj, Z.batch - obj0);
  const int row = tid & 127, part = tid >> 7;          // operand row (j, z-rank index) and half
  const int jr = row >> 3, zr = row & 7;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(pt_smem(&bar_mma[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(pt_smem(&bar_mma[1])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(pt_smem(&bar_z)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_bad = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(pt_smem(&s_tmem)),
                 "r"(kPtTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // partials at the starting interface: [1] for every object
  for (int e = tid; e < kPtObj * kPtRX * kPtRZ; e += blockDim.x) Ls[e] = (e % (kPtRX * kPtRZ)) == 0 ? 1.0f : 0.0f;
  {
    const int j0 = dir == 0 ? 0 : d;
    if (tid < nobj) st[ioff[j0] + obj0 + tid] = 1.0f;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  uint32_t ph_mma[2] = {0u, 0u}, ph_z = 0u;
  int pend[2] = {0, 0};   // products committed on bar_mma[b] and not yet waited for
  bool bad = false, zpend = false;
  const float* Zp = static_cast<const float*>(Z.p);

  for (int s = 0; s < d; ++s) {
    const int k = dir == 0 ? s : d - 1 - s;
    const int x0 = a.rx[k], x1 = a.rx[k + 1], z0 = Z.r[k], z1 = Z.r[k + 1], n = Z.n[k];
    // the contracted X-side rank (K = cr * n) and the output X-side rank (N)
    const int cr = dir == 0 ? x0 : x1, orr = dir == 0 ? x1 : x0;
    const int lgn = n == 16 ? 4 : 3;  // n is 8 or 16
    const int K = cr * n;
    const uint32_t sboA = (uint32_t)(kPtKc / 4) * 128u, sboB = (uint32_t)(K / 4 + (K & 3 ? 1 : 0)) * 128u;
    // ---- Z cores of the CTA's objects: one bulk copy each (landing at an aligned address)
    const long long zsz = (long long)z0 * n * z1;
    if (tid == 0) {
      uint32_t bytes = 0;
      for (int j = 0; j < nobj; ++j) {
        const float* src = Zp + core_base(Z, k, obj0 + j);
        const uintptr_t s0 = reinterpret_cast<uintptr_t>(src) & ~uintptr_t(15);
        bytes += (uint32_t)(((reinterpret_cast<uintptr_t>(src) - s0) + (uintptr_t)zsz * 4 + 15) & ~uintptr_t(15));
      }
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(pt_smem(&bar_z)), "r"(bytes) : "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      for (int j = 0; j < nobj; ++j) {
        const float* src = Zp + core_base(Z, k, obj0 + j);
        const uintptr_t s0 = reinterpret_cast<uintptr_t>(src) & ~uintptr_t(15);
        const uint32_t b = (uint32_t)(((reinterpret_cast<uintptr_t>(src) - s0) + (uintptr_t)zsz * 4 + 15) & ~uintptr_t(15));
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         pt_smem(Zl + j * kPtZObj)),
                     "l"(s0), "r"(b), "r"(pt_smem(&bar_z))
                     : "memory");
      }
    }
    // ---- shared operand B[o][(c, i)] = X_k (left: U[c][i][o]; right: V[o][i][c]), rows o < 32;
    // K = cr n is a multiple of 8. Left: o varies fastest (U's contiguous index); right: c.
    const float* Xk = Xbase + a.Xoff[k];
    if (dir == 0) {
      for (int e = tid; e < kPtRX * K; e += blockDim.x) {
        const int o = e & (kPtRX - 1), kk = e >> 5;  // kk = c n + i: U[c][i][o] at kk * x1 + o
        const float v = o < orr ? __ldg(Xk + kk * x1 + o) : 0.0f;
        *reinterpret_cast<uint32_t*>(Bop + pt_off(o, kk, sboB)) = tf32_bits(v);
      }
    } else {
      for (int e = tid; e < kPtRX * K; e += blockDim.x) {
        const int c = e % cr, rest = e / cr;  // V[o][i][c] at (o n + i) x1 + c, c fastest
        const int i = rest & (n - 1), o = rest >> lgn;
        const float v = o < orr ? __ldg(Xk + (o * n + i) * x1 + c) : 0.0f;
        *reinterpret_cast<uint32_t*>(Bop + pt_off(o, (c << lgn) + i, sboB)) = tf32_bits(v);
      }
    }
    // one thread polls the barrier, the others wait at the block barrier that follows
    const bool zok = tid == 0 ? pt_wait(pt_smem(&bar_z), ph_z) : true;
    ph_z ^= 1u;
    zpend = !zok;
    if (__syncthreads_or(!zok)) bad = true;  // block-uniform
    if (bad) break;
    // ---- chunks of 4 contracted rank indices
    const int nch = (cr + kPtChunkR - 1) / kPtChunkR;
    const float* zj = Zl + jr * kPtZObj + (int)((reinterpret_cast<uintptr_t>(Zp + core_base(Z, k, obj0 + min(jr, nobj - 1))) & 15) >> 2);
    const bool rvalid = jr < nobj && zr < (dir == 0 ? z1 : z0);
    // this row's Z values: left z[g] = Z[g][i][zr] (g < z0), right z[d] = Z[zr][i][d] (d < z1)
    const int zlen = dir == 0 ? z0 : z1;
    const int zstep = dir == 0 ? n * z1 : 1;                     // stride between the 8 values
    const float* zrow = dir == 0 ? zj + zr : zj + zr * n * z1;  // + i * z1 for slice i
    for (int ch = 0; ch < nch; ++ch) {
      const int buf = ch & 1;
      // the products that read this buffer (chunk ch - 2) must be done
      bool wok = true;
      if (pend[buf]) {
        wok = tid == 0 ? pt_wait(pt_smem(&bar_mma[buf]), ph_mma[buf]) : true;
        ph_mma[buf] ^= 1u;
        pend[buf] = 0;
      }
      char* Ab = Abuf + buf * kPtABytes;
      // T[row][(c - 4 ch) * 16 + i] for this thread's two rank indices c = c0, c0 + 1: the
      // partial rows of both in registers, each slice's Z values loaded once for both
      {
        const int c0 = ch * kPtChunkR + part * 2;
        float l0[kPtRZ], l1[kPtRZ];
#pragma unroll
        for (int g = 0; g < kPtRZ; ++g) {  // left: L[c][gamma]; right: R[c][delta] (zero padded)
          l0[g] = Ls[(jr * kPtRX + c0) * kPtRZ + g];
          l1[g] = Ls[(jr * kPtRX + c0 + 1) * kPtRZ + g];
        }
        const bool v0 = rvalid && c0 < cr, v1 = rvalid && c0 + 1 < cr;
        for (int i4 = 0; i4 < kPtNmax; i4 += 4) {
          float t0[4] = {0.0f, 0.0f, 0.0f, 0.0f}, t1[4] = {0.0f, 0.0f, 0.0f, 0.0f};
          if (v0 && i4 < n) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float* zp = zrow + (i4 + u) * z1;
              float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
              for (int g = 0; g < kPtRZ; ++g) {
                const float zv = g < zlen ? zp[g * zstep] : 0.0f;
                s0 = fmaf(l0[g], zv, s0);
                s1 = fmaf(l1[g], zv, s1);
              }
              t0[u] = s0;
              t1[u] = v1 ? s1 : 0.0f;
            }
          }
          const int kk = part * 2 * kPtNmax + i4;
          *reinterpret_cast<uint4*>(Ab + pt_off(row, kk, sboA)) =
              make_uint4(tf32_bits(t0[0]), tf32_bits(t0[1]), tf32_bits(t0[2]), tf32_bits(t0[3]));
          *reinterpret_cast<uint4*>(Ab + pt_off(row, kk + kPtNmax, sboA)) =
              make_uint4(tf32_bits(t1[0]), tf32_bits(t1[1]), tf32_bits(t1[2]), tf32_bits(t1[3]));
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      if (__syncthreads_or(!wok)) bad = true;  // block-uniform
      if (bad) break;
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // A's K index of (c, i) is (c - 4 ch) * 16 + i (modes padded to 16), B's is c * n + i:
        // one K = 8 product per (c, block of 8 modes)
        const uint32_t aBase = pt_smem(Ab);
        const uint32_t bBase = pt_smem(Bop);
        for (int cc = 0; cc < kPtChunkR; ++cc) {
          const int c = ch * kPtChunkR + cc;
          if (c >= cr) break;
          for (int i8 = 0; i8 < n; i8 += 8) {
            // K = 8: A columns (cc * 16 + i8 .. + 7), B columns (c * n + i8 .. + 7)
            const uint64_t da = pt_desc(aBase + (uint32_t)((cc * kPtNmax + i8) >> 2) * 128u, sboA);
            const uint64_t db = pt_desc(bBase + (uint32_t)((c * n + i8) >> 2) * 128u, sboB);
            const uint32_t acc = (c > 0 || i8 > 0) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                "l"(da), "l"(db), "r"(kPtIdesc), "r"(acc));
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         pt_smem(&bar_mma[buf]))
                     : "memory");
      }
      pend[buf] = 1;
    }
    if (bad) break;
    // ---- accumulator -> partials of the next interface
    bool eok = true;
    for (int b2 = 0; b2 < 2; ++b2)
      if (pend[b2]) {
        eok &= tid == 0 ? pt_wait(pt_smem(&bar_mma[b2]), ph_mma[b2]) : true;
        ph_mma[b2] ^= 1u;
        pend[b2] = 0;
      }
    if (__syncthreads_or(!eok)) {
      bad = true;
      break;
    }
    // thread 0 saw the products complete; the block barrier above orders the reads below
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp < 4) {
      uint32_t r[32];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
          "tcgen05.wait::ld.sync.aligned;\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
            "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(tmem + ((uint32_t)(warp * 32) << 16))
          : "memory");
      // row (j, z) holds the new partial's column z: P[j][o][z] for o < 32
      const int j = (warp * 32 + lane) >> 3, zz = lane & 7;
      const int zlim = dir == 0 ? z1 : z0;
      const int jint = dir == 0 ? k + 1 : k;
#pragma unroll
      for (int o = 0; o < kPtRX; ++o) {
        const float v = (o < orr && zz < zlim && j < nobj) ? __uint_as_float(r[o]) : 0.0f;
        Ls[(j * kPtRX + o) * kPtRZ + zz] = v;
        if (j < nobj && o < orr && zz < zlim)
          st[ioff[jint] + (long long)(obj0 + j) * orr * zlim + o * zlim + zz] = v;
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (bad && tid == 0) {
    if (a.err) atomicExch(a.err, (int)T3F_ERR_TIMEOUT);
    atomicExch(&s_bad, 1);
  }
  __syncthreads();
  if (s_bad && tid == 0) {
    // bounded waits for anything still in flight before the memory is released
    for (int b2 = 0; b2 < 2; ++b2)
      if (pend[b2]) pt_wait(pt_smem(&bar_mma[b2]), ph_mma[b2]);
    if (zpend) pt_wait(pt_smem(&bar_z), ph_z ^ 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kPtTmemCols));
}

}  // namespace

bool psweep_tc_supported(const TTV& X, const TTV& Z) {
  if (X.rmax > kPtRX || Z.rmax > kPtRZ || Z.nmax > kPtNmax) return false;
  for (int k = 0; k < Z.d; ++k)
    if (Z.n[k] != 8 && Z.n[k] != 16) return false;  // K steps of 8 modes, shifts for the index split
  return true;
}

size_t psweep_tc_smem() {
  return 2 * (size_t)kPtABytes + kPtBBytes + sizeof(float) * ((size_t)kPtObj * kPtZObj + (size_t)kPtObj * kPtRX * kPtRZ);
}

// Both sweeps in one launch: the left partials of (U, Z) into stL, the right partials of
// (V, Z) into stR (blocks [0, nblk) and [nblk, 2 nblk)).
t3f_status run_psweep_tc(const TTV& U, const TTV& V, const TTV& Z, float* stL, const long long* ioffL, float* stR,
                         const long long* ioffR, int* err, cudaStream_t s) {
  PtArgs a;
  memset(&a, 0, sizeof(a));
  a.Z = Z;
  a.X[0] = static_cast<const float*>(U.p);
  a.X[1] = static_cast<const float*>(V.p);
  for (int k = 0; k < U.d; ++k) a.Xoff[k] = U.off[k];
  for (int k = 0; k <= U.d; ++k) {
    a.rx[k] = U.r[k];
    a.ioff[0][k] = ioffL[k];
    a.ioff[1][k] = ioffR[k];
  }
  a.st[0] = stL;
  a.st[1] = stR;
  a.err = err;
  a.nblk = (Z.batch + kPtObj - 1) / kPtObj;
  const size_t smem = psweep_tc_smem();
  if (cudaFuncSetAttribute(k_psweep_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return T3F_ERR_CUDA;
  k_psweep_tc<<<(unsigned)(2 * a.nblk), kPtThreads, smem, s>>>(a);
  return launch_status();
}

}  // namespace t3f
