// TT-matrix by TT-vector product without rounding (paper Section 4 'matvec'; zip batches
// with broadcasting, Section 3.1) and its adjoint.
//
//   C^k[(a r_x + b), i, (a' r_x + b')] = sum_j A^k[a, i, j, a'] x^k[b, j, b']
//
// One CTA per (pair, core): both cores are staged in shared memory and the product core is
// streamed out row by row; for a fixed output row (a, b) the (i, a', b') block is
// contiguous, so consecutive threads write consecutive addresses.
#include <algorithm>

#include "t3f_internal.cuh"

namespace t3f {

constexpr int kMvRegN = 8;  // column modes n up to this keep A[a, i, :, a'] in registers

struct MatvecArgs {
  TTV A, x, C;
  int bA, bx, P;       // batches; P = number of products
  int maxA, maxX;      // staged floats per core (max over k)
  int* err;            // timeout word of the persistent kernel (nullable)
};


__global__ void __launch_bounds__(256) k_matvec(const __grid_constant__ MatvecArgs a) {
  extern __shared__ float sm[];
  const int p = blockIdx.x / a.A.d, k = blockIdx.x % a.A.d;
  const TTV& A = a.A;
  const TTV& X = a.x;
  const int ra0 = A.r[k], ra1 = A.r[k + 1], rx0 = X.r[k], rx1 = X.r[k + 1];
  const int m = A.m[k], n = A.n[k];
  float* As = sm;             // [ra0][m][n][ra1]
  float* Xs = sm + a.maxA;    // [rx0][n][rx1]
  const float* Ap = static_cast<const float*>(A.p) + core_base(A, k, a.bA == 1 ? 0 : p);
  const float* Xp = static_cast<const float*>(X.p) + core_base(X, k, a.bx == 1 ? 0 : p);
  const int sa = ra0 * m * n * ra1, sx = rx0 * n * rx1;
  for (int e = threadIdx.x; e < sa; e += blockDim.x) As[e] = __ldg(Ap + e);
  for (int e = threadIdx.x; e < sx; e += blockDim.x) Xs[e] = __ldg(Xp + e);
  __syncthreads();
  float* Cp = static_cast<float*>(a.C.p) + core_base(a.C, k, p);
  const int rowlen = m * ra1 * rx1;            // contiguous (i, a', b') block of one row
  // an item is (a, q) with q = (i, a', b') a position of the row block; its thread walks the
  // rows (a, b), b < r_x, so the index split is paid once per r_x outputs; consecutive
  // threads write consecutive addresses
  for (int e = threadIdx.x; e < ra0 * rowlen; e += blockDim.x) {
    const int al = e / rowlen, q = e - al * rowlen;
    const int i = q / (ra1 * rx1), c1 = q - i * (ra1 * rx1);
    const int ap = c1 / rx1, bp = c1 - ap * rx1;
    const float* Ar = As + ((al * m + i) * n) * ra1 + ap;  // A[al, i, j, ap] at j * ra1
    float* cq = Cp + (long long)al * rx0 * rowlen + q;
    if (n <= kMvRegN) {
      float av[kMvRegN];  // A[al, i, :, ap], reused for every row b
#pragma unroll
      for (int j = 0; j < kMvRegN; ++j) av[j] = j < n ? Ar[j * ra1] : 0.0f;
      for (int be = 0; be < rx0; ++be) {
        const float* Xr = Xs + (be * n) * rx1 + bp;        // x[be, j, bp] at j * rx1
        float s = 0.0f;
#pragma unroll
        for (int j = 0; j < kMvRegN; ++j)
          if (j < n) s = fmaf(av[j], Xr[j * rx1], s);
        cq[(long long)be * rowlen] = s;
      }
    } else {
      for (int be = 0; be < rx0; ++be) {
        const float* Xr = Xs + (be * n) * rx1 + bp;
        float s = 0.0f;
        for (int j = 0; j < n; ++j) s = fmaf(Ar[j * ra1], Xr[j * rx1], s);
        cq[(long long)be * rowlen] = s;
      }
    }
  }
}

// Persistent forward for column modes n = N on every core: CTAs take (pair, core) units in
// turn. The next unit's A and x cores arrive by TMA bulk copies -- each core whole, the copy
// rounded out to 16-byte boundaries into a landing zone with slack -- in the other half of a
// double buffer while the current unit's rows are written. A thread item is (position
// q = (i, a', b') of the row block, group of four rows b of x): it keeps x[b, :, b'] of its
// four b in registers and, for every row a, loads A[a, i, :, a'] once to write four outputs
// (consecutive threads write consecutive addresses of four rows).
constexpr int kMvGroup = 4;  // the full-group path below writes exactly four rows

__device__ __forceinline__ uint32_t mv_s32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ const float* mv_floor16(const float* p) {
  return reinterpret_cast<const float*>(reinterpret_cast<uintptr_t>(p) & ~uintptr_t(15));
}
// bytes of the 16-byte-aligned range covering nfl floats from p
__device__ __forceinline__ uint32_t mv_raw_bytes(const float* p, long long nfl) {
  const uintptr_t b = reinterpret_cast<uintptr_t>(p), e = b + (uintptr_t)nfl * 4u;
  return (uint32_t)(((e + 15) & ~uintptr_t(15)) - (b & ~uintptr_t(15)));
}
__device__ __forceinline__ bool mv_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > (1ll << 31)) return false;
  }
}

template <int N>
__global__ void __launch_bounds__(256, 2) k_matvec_p(const __grid_constant__ MatvecArgs a) {
  extern __shared__ __align__(16) float sm[];
  __shared__ __align__(8) uint64_t bar[2];
  const TTV& A = a.A;
  const TTV& X = a.x;
  const int d = A.d, units = a.P * d, tid = threadIdx.x;
  const int lx_off = a.maxA + 8, half = lx_off + a.maxX + 8;  // floats, multiples of 4
  auto a_ptr = [&](int u) {
    return static_cast<const float*>(A.p) + core_base(A, u % d, a.bA == 1 ? 0 : u / d);
  };
  auto x_ptr = [&](int u) {
    return static_cast<const float*>(X.p) + core_base(X, u % d, a.bx == 1 ? 0 : u / d);
  };
  auto issue = [&](int u, int b) {
    const float* Ap = a_ptr(u);
    const float* Xp = x_ptr(u);
    const int k = u % d;
    const uint32_t ba = mv_raw_bytes(Ap, A.osz[k]), bx = mv_raw_bytes(Xp, X.osz[k]);
    const uint32_t bb = mv_s32(&bar[b]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bb), "r"(ba + bx) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     mv_s32(sm + b * half)),
                 "l"(mv_floor16(Ap)), "r"(ba), "r"(bb)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     mv_s32(sm + b * half + lx_off)),
                 "l"(mv_floor16(Xp)), "r"(bx), "r"(bb)
                 : "memory");
  };
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mv_s32(&bar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mv_s32(&bar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if ((int)blockIdx.x < units) issue(blockIdx.x, 0);
  }
  __syncthreads();
  uint32_t ph0 = 0, ph1 = 0;
  int b = 0;
  for (int u = blockIdx.x; u < units; u += gridDim.x, b ^= 1) {
    int good = 1;
    if (tid == 0) good = mv_wait(mv_s32(&bar[b]), b ? ph1 : ph0) ? 1 : 0;
    if (!__syncthreads_and(good)) {
      // the copy did not land: report, wait once more (bounded) for it, and leave
      if (tid == 0) {
        if (a.err) atomicExch(a.err, (int)T3F_ERR_TIMEOUT);
        mv_wait(mv_s32(&bar[b]), b ? ph1 : ph0);
      }
      return;
    }
    if (b) ph1 ^= 1u; else ph0 ^= 1u;
    // prefetch the next unit into the other half (released by the previous iteration's barrier)
    if (tid == 0 && u + (int)gridDim.x < units) issue(u + gridDim.x, b ^ 1);
    const float* Ap = a_ptr(u);
    const float* Xp = x_ptr(u);
    const float* As = sm + b * half + ((reinterpret_cast<uintptr_t>(Ap) & 15) >> 2);
    const float* Xs = sm + b * half + lx_off + ((reinterpret_cast<uintptr_t>(Xp) & 15) >> 2);
    const int p = u / d, k = u % d;
    const int ra0 = A.r[k], ra1 = A.r[k + 1], rx0 = X.r[k], rx1 = X.r[k + 1], m = A.m[k];
    float* Cp = static_cast<float*>(a.C.p) + core_base(a.C, k, p);
    const int L = m * ra1 * rx1, ng = (rx0 + kMvGroup - 1) / kMvGroup, AI = m * N * ra1, rowstep = rx0 * L;
    for (int it = tid; it < L * ng; it += blockDim.x) {
      const int g = it / L, q = it - g * L;
      const int i = q / (ra1 * rx1), c1 = q - i * (ra1 * rx1);
      const int ap = c1 / rx1, bp = c1 - ap * rx1, be0 = g * kMvGroup;
      float xr[kMvGroup][N];
#pragma unroll
      for (int bb = 0; bb < kMvGroup; ++bb)
#pragma unroll
        for (int j = 0; j < N; ++j) xr[bb][j] = be0 + bb < rx0 ? Xs[((be0 + bb) * N + j) * rx1 + bp] : 0.0f;
      const float* Ar = As + (i * N) * ra1 + ap;  // A[al, i, j, ap] at al * AI + j * ra1
      float* cq = Cp + (long long)be0 * L + q;    // rows (al, be0 + bb) at cq + al * rowstep + bb * L
      const long long o1 = L, o2 = 2LL * L, o3 = 3LL * L;
      if (be0 + kMvGroup <= rx0) {
        // a full group of four rows: no predicates in the row loop
#pragma unroll 2
        for (int al = 0; al < ra0; ++al, cq += rowstep, Ar += AI) {
          float av[N];
#pragma unroll
          for (int j = 0; j < N; ++j) av[j] = Ar[j * ra1];
          float sv[kMvGroup];
#pragma unroll
          for (int bb = 0; bb < kMvGroup; ++bb) {
            float t = 0.0f;
#pragma unroll
            for (int j = 0; j < N; ++j) t = fmaf(av[j], xr[bb][j], t);
            sv[bb] = t;
          }
          cq[0] = sv[0];
          cq[o1] = sv[1];
          cq[o2] = sv[2];
          cq[o3] = sv[3];
        }
      } else {
        for (int al = 0; al < ra0; ++al, cq += rowstep, Ar += AI) {
          float av[N];
#pragma unroll
          for (int j = 0; j < N; ++j) av[j] = Ar[j * ra1];
#pragma unroll
          for (int bb = 0; bb < kMvGroup; ++bb) {
            if (be0 + bb < rx0) {
              float t = 0.0f;
#pragma unroll
              for (int j = 0; j < N; ++j) t = fmaf(av[j], xr[bb][j], t);
              cq[(long long)bb * L] = t;
            }
          }
        }
      }
    }
    __syncthreads();
  }
}

// Adjoint: one CTA per (pair, core). Rows a of dC are staged in shared memory in turn.
struct MatvecBwdArgs {
  TTV A, x, dC;
  int bA, bx, P;
  int maxA, maxX, maxRow;
  float* dA;   // packed like A, nullable
  float* dx;   // packed like x, nullable
  int atomicA, atomicX;  // a broadcast side sums over the batch with atomics
};

__global__ void __launch_bounds__(256) k_matvec_bwd(const __grid_constant__ MatvecBwdArgs a) {
  extern __shared__ float sm[];
  const int p = blockIdx.x / a.A.d, k = blockIdx.x % a.A.d;
  const TTV& A = a.A;
  const TTV& X = a.x;
  const int ra0 = A.r[k], ra1 = A.r[k + 1], rx0 = X.r[k], rx1 = X.r[k + 1];
  const int m = A.m[k], n = A.n[k];
  float* As = sm;                     // [ra0][m][n][ra1]
  float* Xs = As + a.maxA;            // [rx0][n][rx1]
  float* Gs = Xs + a.maxX;            // one dC row block a: [rx0][m][ra1][rx1]
  float* dXs = Gs + a.maxRow;         // [rx0][n][rx1] accumulator
  const int oa = a.bA == 1 ? 0 : p, ox = a.bx == 1 ? 0 : p;
  const float* Ap = static_cast<const float*>(A.p) + core_base(A, k, oa);
  const float* Xp = static_cast<const float*>(X.p) + core_base(X, k, ox);
  const float* Gp = static_cast<const float*>(a.dC.p) + core_base(a.dC, k, p);
  const int sa = ra0 * m * n * ra1, sx = rx0 * n * rx1;
  for (int e = threadIdx.x; e < sa; e += blockDim.x) As[e] = __ldg(Ap + e);
  for (int e = threadIdx.x; e < sx; e += blockDim.x) {
    Xs[e] = __ldg(Xp + e);
    dXs[e] = 0.0f;
  }
  const int rowlen = m * ra1 * rx1;
  const int blk = rx0 * rowlen;  // rows (al, 0..rx0-1) are contiguous in dC
  for (int al = 0; al < ra0; ++al) {
    __syncthreads();
    for (int e = threadIdx.x; e < blk; e += blockDim.x) Gs[e] = __ldg(Gp + (long long)al * blk + e);
    __syncthreads();
    if (a.dA) {
      // dA[al, i, j, ap] = sum_{b, bp} G[b][i][ap][bp] x[b][j][bp]
      float* dAp = a.dA + core_base(A, k, oa);
      for (int e = threadIdx.x; e < m * n * ra1; e += blockDim.x) {
        const int ap = e % ra1, j = (e / ra1) % n, i = e / (ra1 * n);
        float s = 0.0f;
        for (int be = 0; be < rx0; ++be) {
          const float* g = Gs + ((be * m + i) * ra1 + ap) * rx1;
          const float* xv = Xs + (be * n + j) * rx1;
          for (int bp = 0; bp < rx1; ++bp) s = fmaf(g[bp], xv[bp], s);
        }
        float* dst = dAp + ((al * m + i) * n + j) * ra1 + ap;
        if (a.atomicA) atomicAdd(dst, s); else *dst = s;
      }
    }
    if (a.dx) {
      // dx[b, j, bp] += sum_{i, ap} G[b][i][ap][bp] A[al, i, j, ap]
      for (int e = threadIdx.x; e < sx; e += blockDim.x) {
        const int bp = e % rx1, j = (e / rx1) % n, be = e / (rx1 * n);
        float s = 0.0f;
        for (int i = 0; i < m; ++i) {
          const float* g = Gs + ((be * m + i) * ra1) * rx1 + bp;
          const float* av = As + ((al * m + i) * n + j) * ra1;
          for (int ap = 0; ap < ra1; ++ap) s = fmaf(g[ap * rx1], av[ap], s);
        }
        dXs[e] += s;
      }
    }
  }
  if (a.dx) {
    float* dXp = a.dx + core_base(X, k, ox);
    for (int e = threadIdx.x; e < sx; e += blockDim.x) {
      if (a.atomicX) atomicAdd(dXp + e, dXs[e]); else dXp[e] = dXs[e];
    }
  }
}

// Adjoint for column modes n = N (2, 4, 8): one CTA per (pair, core). The dC row blocks a
// (rows (a, b), b < r_x: contiguous) are staged by 16-byte asynchronous copies into two
// buffers, one block ahead of the products; A and x are staged with j innermost
// (At[a][i][a'][j], xt[b][b'][j]) so that every K step of the two products reads its N
// values of j with one vector load:
//   dx[b, j, b'] += sum_{i, a'} G[b][i][a'][b'] At[a][i][a'][j]   thread per (b, b'), kept in
//                                                                 registers across all a
//   dA[a, i, j, a'] = sum_{b, b'} G[b][i][a'][b'] xt[b][b'][j]    thread per (i, a') and part of
//                                                                 the b range, parts summed
//                                                                 in shared memory
constexpr int kMvRed = 256 * 8;  // floats of one half of the adjoint's parts buffer

template <int N>
__global__ void __launch_bounds__(256) k_matvec_bwd_n(const __grid_constant__ MatvecBwdArgs a) {
  extern __shared__ __align__(16) float sm[];
  const int p = blockIdx.x / a.A.d, k = blockIdx.x % a.A.d;
  const TTV& A = a.A;
  const TTV& X = a.x;
  const int ra0 = A.r[k], ra1 = A.r[k + 1], rx0 = X.r[k], rx1 = X.r[k + 1];
  const int m = A.m[k];
  const int tid = threadIdx.x;
  float* At = sm;                      // [ra0][m][ra1][N]
  float* Xt = At + a.maxA;             // [rx0][rx1][N]
  float* Gb = Xt + a.maxX;             // [3][maxRow]: a ring of dC row blocks, two ahead
  float* Red = Gb + 3 * a.maxRow;      // [2][kMvRed]: dA partial sums [parts][m * ra1][N]
  const int oa = a.bA == 1 ? 0 : p, ox = a.bx == 1 ? 0 : p;
  const float* Ap = static_cast<const float*>(A.p) + core_base(A, k, oa);
  const float* Xp = static_cast<const float*>(X.p) + core_base(X, k, ox);
  const float* Gp = static_cast<const float*>(a.dC.p) + core_base(a.dC, k, p);
  const int sa = ra0 * m * N * ra1, sx = rx0 * N * rx1;
  for (int e = tid; e < sa; e += blockDim.x) {  // A[al][i][j][ap] -> At[al][i][ap][j]
    const int ap = e % ra1, j = (e / ra1) % N, ali = e / (ra1 * N);
    At[(ali * ra1 + ap) * N + j] = __ldg(Ap + e);
  }
  for (int e = tid; e < sx; e += blockDim.x) {  // x[b][j][bp] -> Xt[b][bp][j]
    const int bp = e % rx1, j = (e / rx1) % N, b = e / (rx1 * N);
    Xt[(b * rx1 + bp) * N + j] = __ldg(Xp + e);
  }
  const int rowlen = m * ra1 * rx1;
  const int blk = rx0 * rowlen;
  const bool vec = ((reinterpret_cast<uintptr_t>(Gp) & 15) == 0) && (blk & 3) == 0;
  auto stage = [&](int al) {
    float* dst = Gb + (al % 3) * a.maxRow;
    const float* src = Gp + (long long)al * blk;
    if (vec) {
      for (int e4 = tid; e4 < blk / 4; e4 += blockDim.x) {
        const unsigned sa_ = (unsigned)__cvta_generic_to_shared(dst + 4 * e4);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa_), "l"(src + 4 * e4));
      }
    } else {
      for (int e = tid; e < blk; e += blockDim.x) {
        const unsigned sa_ = (unsigned)__cvta_generic_to_shared(dst + e);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa_), "l"(src + e));
      }
    }
    asm volatile("cp.async.commit_group;\n" ::);
  };
  // dx: thread per (b, bp) with N accumulators; with at most 256 pairs (b, bp) the sum over
  // q = (i, a') is split into H parts over otherwise idle threads, reduced once at the end
  const int nbb = rx0 * rx1;
  const int H = nbb <= (int)blockDim.x ? max(1, min(8, (int)blockDim.x / max(nbb, 1))) : 1;
  float dxa[2][N];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int j = 0; j < N; ++j) dxa[u][j] = 0.0f;
  // dA: items (i, ap) x parts of the b range
  const int nia = m * ra1;
  const int parts = max(1, min(rx0, (int)blockDim.x / max(nia, 1)));
  // dA[al, i, j, ap] from the parts of row al (written in the iteration of row al)
  float* dAp = a.dA ? a.dA + core_base(A, k, oa) : nullptr;
  auto reduce_dA = [&](int al, const float* R) {
    for (int e = tid; e < nia * N; e += blockDim.x) {
      const int ap = e % ra1, j = (e / ra1) % N, i = e / (ra1 * N);
      const int q = i * ra1 + ap;
      float s = 0.0f;
      for (int pp = 0; pp < parts; ++pp) s += R[(pp * nia + q) * N + j];
      float* dst = dAp + ((al * m + i) * N + j) * ra1 + ap;
      if (a.atomicA) atomicAdd(dst, s); else *dst = s;
    }
  };
  // one barrier per row block: after it, block al has landed, the parts of row al - 1 are
  // complete, and ring slot (al + 2) % 3 (last read for row al - 1) may be restaged
  stage(0);
  if (ra0 > 1) stage(1);
  for (int al = 0; al < ra0; ++al) {
    if (al + 1 < ra0)
      asm volatile("cp.async.wait_group 1;\n" ::);
    else
      asm volatile("cp.async.wait_group 0;\n" ::);
    __syncthreads();
    if (al + 2 < ra0) stage(al + 2);
    if (a.dA && al > 0) reduce_dA(al - 1, Red + ((al - 1) & 1) * kMvRed);
    const float* G = Gb + (al % 3) * a.maxRow;  // [b][i][ap][bp]
    if (a.dx && nbb <= (int)blockDim.x) {
      if (tid < nbb * H) {
        const int bb = tid % nbb, h = tid / nbb;
        const int q0 = h * nia / H, q1 = (h + 1) * nia / H;
        const int b = bb / rx1, bp = bb % rx1;
        const float* g = G + (long long)b * rowlen + bp + q0 * rx1;
        const float* at = At + (long long)al * m * ra1 * N + q0 * N;
#pragma unroll 4
        for (int q = q0; q < q1; ++q, g += rx1, at += N) {
          const float gv = *g;
          if constexpr (N == 4) {
            const float4 v = *reinterpret_cast<const float4*>(at);
            dxa[0][0] = fmaf(gv, v.x, dxa[0][0]);
            dxa[0][1] = fmaf(gv, v.y, dxa[0][1]);
            dxa[0][2] = fmaf(gv, v.z, dxa[0][2]);
            dxa[0][3] = fmaf(gv, v.w, dxa[0][3]);
          } else {
#pragma unroll
            for (int j = 0; j < N; ++j) dxa[0][j] = fmaf(gv, at[j], dxa[0][j]);
          }
        }
      }
    } else if (a.dx) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int e = tid + u * (int)blockDim.x;
        if (e < nbb) {
          const int b = e / rx1, bp = e % rx1;
          const float* g = G + (long long)b * rowlen + bp;
          const float* at = At + (long long)al * m * ra1 * N;
          for (int q = 0; q < nia; ++q) {  // q = i * ra1 + ap
            const float gv = g[q * rx1];
            if constexpr (N == 4) {
              const float4 v = *reinterpret_cast<const float4*>(at + q * 4);
              dxa[u][0] = fmaf(gv, v.x, dxa[u][0]);
              dxa[u][1] = fmaf(gv, v.y, dxa[u][1]);
              dxa[u][2] = fmaf(gv, v.z, dxa[u][2]);
              dxa[u][3] = fmaf(gv, v.w, dxa[u][3]);
            } else {
#pragma unroll
              for (int j = 0; j < N; ++j) dxa[u][j] = fmaf(gv, at[q * N + j], dxa[u][j]);
            }
          }
        }
      }
    }
    if (a.dA) {
      const int it = tid % max(nia, 1), part = tid / max(nia, 1);
      float acc[N];
#pragma unroll
      for (int j = 0; j < N; ++j) acc[j] = 0.0f;
      if (part < parts && it < nia) {
        const int b0 = part * rx0 / parts, b1 = (part + 1) * rx0 / parts;
        for (int b = b0; b < b1; ++b) {
          const float* g = G + (long long)b * rowlen + it * rx1;
          const float* xt = Xt + (long long)b * rx1 * N;
          for (int bp = 0; bp < rx1; ++bp) {
            const float gv = g[bp];
            if constexpr (N == 4) {
              const float4 v = *reinterpret_cast<const float4*>(xt + bp * 4);
              acc[0] = fmaf(gv, v.x, acc[0]);
              acc[1] = fmaf(gv, v.y, acc[1]);
              acc[2] = fmaf(gv, v.z, acc[2]);
              acc[3] = fmaf(gv, v.w, acc[3]);
            } else {
#pragma unroll
              for (int j = 0; j < N; ++j) acc[j] = fmaf(gv, xt[bp * N + j], acc[j]);
            }
          }
        }
#pragma unroll
        for (int j = 0; j < N; ++j) Red[(al & 1) * kMvRed + (part * nia + it) * N + j] = acc[j];
      }
    }
  }
  __syncthreads();
  if (a.dA && ra0 > 0) reduce_dA(ra0 - 1, Red + ((ra0 - 1) & 1) * kMvRed);
  if (a.dx && nbb <= (int)blockDim.x) {
    // the H partial sums of every (b, bp) through the other half of the parts buffer
    float* const Rx = Red + (ra0 & 1) * kMvRed;
    float* dXp = a.dx + core_base(X, k, ox);
    if (tid < nbb * H) {
#pragma unroll
      for (int j = 0; j < N; ++j) Rx[tid * N + j] = dxa[0][j];
    }
    __syncthreads();
    if (tid < nbb) {
      const int b = tid / rx1, bp = tid % rx1;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        float v = 0.0f;
        for (int h = 0; h < H; ++h) v += Rx[(h * nbb + tid) * N + j];
        float* dst = dXp + (b * N + j) * rx1 + bp;
        if (a.atomicX) atomicAdd(dst, v); else *dst = v;
      }
    }
  } else if (a.dx) {
    float* dXp = a.dx + core_base(X, k, ox);
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int e = tid + u * (int)blockDim.x;
      if (e < nbb) {
        const int b = e / rx1, bp = e % rx1;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          float* dst = dXp + (b * N + j) * rx1 + bp;
          if (a.atomicX) atomicAdd(dst, dxa[u][j]); else *dst = dxa[u][j];
        }
      }
    }
  }
}

static t3f_status matvec_views(const t3f_tt* A, const t3f_tt* x, TTV* va, TTV* vx, int* P) {
  T3F_CHECK(make_view(A, va, T3F_F32, true));
  T3F_CHECK(make_view(x, vx, T3F_F32, false));
  if (va->d != vx->d) return T3F_ERR_SHAPE;
  for (int k = 0; k < va->d; ++k)
    if (va->n[k] != vx->n[k]) return T3F_ERR_SHAPE;
  if (va->batch != vx->batch && va->batch != 1 && vx->batch != 1) return T3F_ERR_SHAPE;
  *P = va->batch > vx->batch ? va->batch : vx->batch;
  return T3F_OK;
}

static t3f_status check_product(const TTV& A, const TTV& X, int P, const t3f_tt* C, TTV* vc) {
  T3F_CHECK(make_view(C, vc, T3F_F32, false));
  if (vc->d != A.d || vc->batch != P) return T3F_ERR_SHAPE;
  for (int k = 0; k <= A.d; ++k) {
    if ((long long)vc->r[k] != (long long)A.r[k] * X.r[k]) return T3F_ERR_SHAPE;
    if (k < A.d && vc->n[k] != A.m[k]) return T3F_ERR_SHAPE;
  }
  return T3F_OK;
}

}  // namespace t3f

using namespace t3f;

extern "C" t3f_status t3f_matvec(const t3f_tt* A, const t3f_tt* x, t3f_tt* C, void* ws,
                                 size_t ws_bytes, t3f_stream_t stream) {
  TTV va, vx, vc;
  int P;
  T3F_CHECK(matvec_views(A, x, &va, &vx, &P));
  T3F_CHECK(check_product(va, vx, P, C, &vc));
  MatvecArgs args;
  memset(&args, 0, sizeof(args));
  // the error word of the persistent kernel's bounded waits (optional)
  args.err = (ws && ws_bytes >= kWsHeader) ? static_cast<int*>(ws) : nullptr;
  if (args.err && cudaMemsetAsync(args.err, 0, sizeof(int), (cudaStream_t)stream) != cudaSuccess) return T3F_ERR_CUDA;
  args.A = va;
  args.x = vx;
  args.C = vc;
  args.bA = va.batch;
  args.bx = vx.batch;
  args.P = P;
  args.maxA = 0;
  args.maxX = 0;
  for (int k = 0; k < va.d; ++k) {
    if (va.osz[k] > args.maxA) args.maxA = (int)va.osz[k];
    if (vx.osz[k] > args.maxX) args.maxX = (int)vx.osz[k];
  }
  args.maxA = (args.maxA + 3) & ~3;
  const size_t smem = sizeof(float) * ((size_t)args.maxA + args.maxX);
  if (smem > 200 * 1024) return T3F_ERR_UNSUPPORTED;
  const long long grid = (long long)P * va.d;
  if (grid > 0x7fffffffLL) return T3F_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  int nall = va.n[0];
  for (int k = 0; k < va.d; ++k)
    if (va.n[k] != nall) nall = -1;
  const size_t psm = sizeof(float) * 2 * ((size_t)args.maxA + 8 + ((args.maxX + 3) & ~3) + 8);
  if ((nall == 2 || nall == 4 || nall == 8) && psm <= 200 * 1024) {
    // persistent kernel with TMA-staged cores: as many CTAs as fit on the GPU at once
    args.maxX = (args.maxX + 3) & ~3;
    auto runp = [&](auto kern) -> t3f_status {
      if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm) != cudaSuccess)
        return T3F_ERR_CUDA;
      int dev = 0, sms = 0, per = 0;
      if (cudaGetDevice(&dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, psm) != cudaSuccess)
        return T3F_ERR_CUDA;
      const long long g = std::min<long long>(grid, (long long)sms * std::max(per, 1));
      kern<<<(unsigned)g, 256, psm, s>>>(args);
      return launch_status();
    };
    if (nall == 2) return runp(k_matvec_p<2>);
    if (nall == 4) return runp(k_matvec_p<4>);
    return runp(k_matvec_p<8>);
  }
  auto run = [&](auto kern, long long g) -> t3f_status {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return T3F_ERR_CUDA;
    kern<<<(unsigned)g, 256, smem, s>>>(args);
    return launch_status();
  };
  return run(k_matvec, grid);
}

extern "C" t3f_status t3f_matvec_backward(const t3f_tt* A, const t3f_tt* x, const t3f_tt* dC,
                                          t3f_tt* dA, t3f_tt* dx, void* ws, size_t ws_bytes,
                                          t3f_stream_t stream) {
  TTV va, vx, vg, vda, vdx;
  int P;
  T3F_CHECK(matvec_views(A, x, &va, &vx, &P));
  T3F_CHECK(check_product(va, vx, P, dC, &vg));
  (void)ws;
  (void)ws_bytes;
  cudaStream_t s = (cudaStream_t)stream;
  MatvecBwdArgs args;
  memset(&args, 0, sizeof(args));
  if (dA) {
    T3F_CHECK(make_view(dA, &vda, T3F_F32, true));
    if (vda.batch != va.batch || vda.d != va.d) return T3F_ERR_SHAPE;
    for (int k = 0; k < va.d; ++k)
      if (vda.osz[k] != va.osz[k] || vda.r[k] != va.r[k] || vda.m[k] != va.m[k]) return T3F_ERR_SHAPE;
    args.dA = static_cast<float*>(vda.p);
  }
  if (dx) {
    T3F_CHECK(make_view(dx, &vdx, T3F_F32, false));
    if (vdx.batch != vx.batch || vdx.d != vx.d) return T3F_ERR_SHAPE;
    for (int k = 0; k < vx.d; ++k)
      if (vdx.osz[k] != vx.osz[k] || vdx.r[k] != vx.r[k]) return T3F_ERR_SHAPE;
    args.dx = static_cast<float*>(vdx.p);
  }
  if (!args.dA && !args.dx) return T3F_OK;
  args.A = va;
  args.x = vx;
  args.dC = vg;
  args.bA = va.batch;
  args.bx = vx.batch;
  args.P = P;
  args.atomicA = (va.batch == 1 && P > 1);
  args.atomicX = (vx.batch == 1 && P > 1);
  for (int k = 0; k < va.d; ++k) {
    if (va.osz[k] > args.maxA) args.maxA = (int)va.osz[k];
    if (vx.osz[k] > args.maxX) args.maxX = (int)vx.osz[k];
    const int row = vx.r[k] * va.m[k] * va.r[k + 1] * vx.r[k + 1];
    if (row > args.maxRow) args.maxRow = row;
  }
  const size_t smem = sizeof(float) * ((size_t)args.maxA + 2 * (size_t)args.maxX + args.maxRow);
  if (smem > 200 * 1024) return T3F_ERR_UNSUPPORTED;
  // the specialised adjoint: one column mode for every core, at most 512 (b, b') pairs and
  // 256 (i, a') items per core
  int nall = va.n[0];
  bool spec = true;
  int maxIA = 0;
  for (int k = 0; k < va.d; ++k) {
    if (va.n[k] != nall) nall = -1;
    if (vx.r[k] * vx.r[k + 1] > 512) spec = false;
    maxIA = std::max(maxIA, va.m[k] * va.r[k + 1]);
  }
  if (maxIA > 256) spec = false;
  if (args.atomicA && cudaMemsetAsync(args.dA, 0, sizeof(float) * t3f_packed_size(dA), s) != cudaSuccess)
    return T3F_ERR_CUDA;
  if (args.atomicX && cudaMemsetAsync(args.dx, 0, sizeof(float) * t3f_packed_size(dx), s) != cudaSuccess)
    return T3F_ERR_CUDA;
  const long long grid = (long long)P * va.d;
  if (spec && (nall == 2 || nall == 4 || nall == 8)) {
    MatvecBwdArgs b2 = args;
    b2.maxA = (args.maxA + 3) & ~3;
    b2.maxX = (args.maxX + 3) & ~3;
    b2.maxRow = (args.maxRow + 3) & ~3;
    const size_t sm2 = sizeof(float) * ((size_t)b2.maxA + b2.maxX + 3 * (size_t)b2.maxRow + 2 * (size_t)kMvRed);
    if (sm2 <= 200 * 1024) {
      auto go = [&](auto kern) -> t3f_status {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2) != cudaSuccess)
          return T3F_ERR_CUDA;
        kern<<<(unsigned)grid, 256, sm2, s>>>(b2);
        return launch_status();
      };
      if (nall == 2) return go(k_matvec_bwd_n<2>);
      if (nall == 4) return go(k_matvec_bwd_n<4>);
      return go(k_matvec_bwd_n<8>);
    }
  }
  if (cudaFuncSetAttribute(k_matvec_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return T3F_ERR_CUDA;
  k_matvec_bwd<<<(unsigned)grid, 256, smem, s>>>(args);
  return launch_status();
}
