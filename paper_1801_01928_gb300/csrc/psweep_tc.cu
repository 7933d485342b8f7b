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
// tensor cores consume the other; the two threads of a row split the modes (n = 16) or the
// rank indices (n = 8), so each loads its row's Z values once per chunk. The shared operand of
// a core is the same for every CTA: a pre-pass writes it once per (sweep, core) into the
// workspace as the byte image of its shared-memory layout (TF32 values), and each CTA brings
// it in with one bulk copy, beside the Z cores of its objects (one bulk copy per object and
// core, rounded out to 16-byte boundaries). The partials are stored in the layout of the
// CUDA-core sweeps ([r_X][r_Z] per object and interface), so the FP32 assembly and gauge
// projection consume them unchanged.
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
constexpr size_t kPtImgStride = kPtBBytes;       // bytes per (sweep, core) operand image

struct PtArgs {
  TTV Z;
  int rx[T3F_MAX_D + 1];         // X ranks (U and V have equal shapes)
  float* st[2];                  // partial stores of the two sweeps
  long long ioff[2][T3F_MAX_D + 1];
  int nblk;                      // CTAs per direction; blocks [nblk, 2 nblk) run the right sweep
  int* err;
  const char* img;               // [2][d] operand images of kPtImgStride bytes (pre-pass output)
};

struct PtImgArgs {
  const float* X[2];
  long long Xoff[T3F_MAX_D];
  int rx[T3F_MAX_D + 1];
  int n[T3F_MAX_D];
  int d;
  char* img;
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

// Operand image of block (sweep, core): B[o][(c, i)] = U_k[c][i][o] (left) or V_k[o][i][c]
// (right) as TF32 in the K-major layout the sweep kernel reads (rows o < 32, zero past the
// output rank). 16-byte unit u of the image holds row o = 8 (u / 2K) + u % 8 and the four K
// values 4 ((u % 2K) / 8) .. + 3, so consecutive threads write consecutive bytes.
__global__ void __launch_bounds__(256) k_psweep_tc_img(const __grid_constant__ PtImgArgs a) {
  const int dir = (int)blockIdx.x / a.d, k = (int)blockIdx.x % a.d;
  const int x0 = a.rx[k], x1 = a.rx[k + 1], n = a.n[k];
  const int cr = dir == 0 ? x0 : x1, orr = dir == 0 ? x1 : x0;
  const int K = cr * n, lgn = n == 16 ? 4 : 3;
  const float* Xk = a.X[dir] + a.Xoff[k];
  uint4* out = reinterpret_cast<uint4*>(a.img + (size_t)blockIdx.x * kPtImgStride);
  for (int u = threadIdx.x; u < 8 * K; u += blockDim.x) {
    const int g = u / (2 * K), rem = u - g * 2 * K;
    const int o = 8 * g + (rem & 7), kk0 = 4 * (rem >> 3);
    uint32_t v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int kk = kk0 + q, c = kk >> lgn, i = kk & (n - 1);
      float x = 0.0f;
      if (o < orr) x = dir == 0 ? __ldg(Xk + (long long)kk * x1 + o) : __ldg(Xk + ((long long)o * n + i) * x1 + c);
      v[q] = tf32_bits(x);
    }
    out[u] = make_uint4(v[0], v[1], v[2], v[3]);
  }
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
    const int K = cr * n;
    const uint32_t sboA = (uint32_t)(kPtKc / 4) * 128u;
    // ---- Z cores of the CTA's objects: one bulk copy each (landing at an aligned address)
    const long long zsz = (long long)z0 * n * z1;
    const uint32_t sboB = (uint32_t)(K / 4) * 128u, imgb = (uint32_t)K * 128u;  // K is a multiple of 8
    if (tid == 0) {
      uint32_t bytes = imgb;
      for (int j = 0; j < nobj; ++j) {
        const float* src = Zp + core_base(Z, k, obj0 + j);
        const uintptr_t s0 = reinterpret_cast<uintptr_t>(src) & ~uintptr_t(15);
        bytes += (uint32_t)(((reinterpret_cast<uintptr_t>(src) - s0) + (uintptr_t)zsz * 4 + 15) & ~uintptr_t(15));
      }
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(pt_smem(&bar_z)), "r"(bytes) : "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      // the shared operand X_k (no product of the previous core is in flight: they were all
      // waited for before its partials were read out)
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       pt_smem(Bop)),
                   "l"(a.img + (size_t)(dir * d + k) * kPtImgStride), "r"(imgb), "r"(pt_smem(&bar_z))
                   : "memory");
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
    // right sweep: a row's eight values of a slice are contiguous (two 16-byte loads)
    const bool zvec = dir == 1 && z1 == kPtRZ && (reinterpret_cast<uintptr_t>(zrow) & 15) == 0;
    // n = 16: the row's two threads take 8 modes each for all 4 rank indices of a chunk;
    // n = 8: 2 rank indices each for all 8 modes
    const bool nsplit = n == 16;
    const int nc = nsplit ? kPtChunkR : kPtChunkR / 2, iA = nsplit ? part * 8 : 0;
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
      // T[row][(c - 4 ch) * 16 + i] for this thread's rank indices c and modes i: the partial
      // rows in registers, each slice's Z values loaded once for all of them (rows past the
      // rank are zero in Ls)
      {
        const int cA = ch * kPtChunkR + (nsplit ? 0 : part * 2);
        float l[kPtChunkR][kPtRZ];
#pragma unroll
        for (int c = 0; c < kPtChunkR; ++c)
#pragma unroll
          for (int g = 0; g < kPtRZ; ++g)  // left: L[c][gamma]; right: R[c][delta]
            l[c][g] = c < nc ? Ls[(jr * kPtRX + cA + c) * kPtRZ + g] : 0.0f;
#pragma unroll
        for (int ih = 0; ih < 8; ih += 4) {
          const int i4 = iA + ih;
          float t[kPtChunkR][4];
#pragma unroll
          for (int c = 0; c < kPtChunkR; ++c)
#pragma unroll
            for (int u = 0; u < 4; ++u) t[c][u] = 0.0f;
          if (rvalid) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              float z[kPtRZ];
              if (zvec) {
                const float4 p = *reinterpret_cast<const float4*>(zrow + (i4 + u) * kPtRZ);
                const float4 q = *reinterpret_cast<const float4*>(zrow + (i4 + u) * kPtRZ + 4);
                z[0] = p.x; z[1] = p.y; z[2] = p.z; z[3] = p.w;
                z[4] = q.x; z[5] = q.y; z[6] = q.z; z[7] = q.w;
              } else {
                const float* zp = zrow + (i4 + u) * z1;
#pragma unroll
                for (int g = 0; g < kPtRZ; ++g) z[g] = g < zlen ? zp[g * zstep] : 0.0f;
              }
#pragma unroll
              for (int c = 0; c < kPtChunkR; ++c) {
                float sacc = 0.0f;
#pragma unroll
                for (int g = 0; g < kPtRZ; ++g) sacc = fmaf(l[c][g], z[g], sacc);
                t[c][u] = sacc;
              }
            }
          }
#pragma unroll
          for (int c = 0; c < kPtChunkR; ++c)
            if (c < nc)
              *reinterpret_cast<uint4*>(Ab + pt_off(row, (cA - ch * kPtChunkR + c) * kPtNmax + i4, sboA)) =
                  make_uint4(tf32_bits(t[c][0]), tf32_bits(t[c][1]), tf32_bits(t[c][2]), tf32_bits(t[c][3]));
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

size_t psweep_tc_img_bytes(const TTV& X) { return 2 * (size_t)X.d * kPtImgStride; }

size_t psweep_tc_smem() {
  return 2 * (size_t)kPtABytes + kPtBBytes + sizeof(float) * ((size_t)kPtObj * kPtZObj + (size_t)kPtObj * kPtRX * kPtRZ);
}

// The operand images (one launch over the 2 d (sweep, core) pairs), then both sweeps in one
// launch: the left partials of (U, Z) into stL, the right partials of (V, Z) into stR (blocks
// [0, nblk) and [nblk, 2 nblk)). img: psweep_tc_img_bytes(U) bytes, 16-byte aligned.
t3f_status run_psweep_tc(const TTV& U, const TTV& V, const TTV& Z, float* stL, const long long* ioffL, float* stR,
                         const long long* ioffR, void* img, int* err, cudaStream_t s) {
  if (reinterpret_cast<uintptr_t>(img) & 15) return T3F_ERR_WORKSPACE;
  PtImgArgs ia;
  memset(&ia, 0, sizeof(ia));
  ia.X[0] = static_cast<const float*>(U.p);
  ia.X[1] = static_cast<const float*>(V.p);
  ia.d = U.d;
  ia.img = static_cast<char*>(img);
  for (int k = 0; k < U.d; ++k) {
    ia.Xoff[k] = U.off[k];
    ia.n[k] = U.n[k];
  }
  for (int k = 0; k <= U.d; ++k) ia.rx[k] = U.r[k];
  k_psweep_tc_img<<<(unsigned)(2 * U.d), 256, 0, s>>>(ia);
  T3F_CHECK(launch_status());
  PtArgs a;
  memset(&a, 0, sizeof(a));
  a.Z = Z;
  a.img = static_cast<const char*>(img);
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
