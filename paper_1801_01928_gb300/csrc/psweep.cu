// Register-tiled sweeps for project_sum and its adjoint (paper Section 3.2): one tangent
// point X (orthogonal forms U, V and the gauge-projected cotangent W; batch 1, ranks <= RU)
// against a batch of TT objects Z (ranks <= 8).
//
// Every step of these sweeps has the form
//     T[m][b]     = sum_K CurT[K][m] Zs[K][b]          (K < 8)       "T-step"
//     Next[m][b] += sum_K As[K][m]   T[K][b]           (K < RU)      "accumulate step"
// with, for the left sweep (interfaces 0 -> d), Zs = Z_k[:, i, :], As = A_k[:, i, :]
// (Next = sum_i A_i^T Cur Z_i), and for the right sweep (d -> 0), Zs = Z_k[:, i, :]^T,
// As = A_k[:, i, :]^T (Next = sum_i A_i Cur Z_i^T). The fused ("mixed") sweeps of the
// adjoint carry a second partial:
//     left :  L' = sum_i U_i^T (L Z_i),   P' = sum_i V_i^T (P Z_i) + W_i^T (L Z_i)
//     right:  R' = sum_i V_i (R Z_i^T),   Q' = sum_i U_i (Q Z_i^T) + W_i (R Z_i^T)
// A CTA holds J objects; each object owns SPLIT groups of G = (RU/4) * 2 threads and group h
// handles the slices i = h (mod SPLIT). A thread accumulates one 4 x 4 block of Next in
// registers; at the end of a core the SPLIT partial blocks are summed in shared memory.
// All operands are zero-padded to RU x 8, so boundary cores need no special cases.
#include "t3f_internal.cuh"

namespace t3f {

constexpr int kRZ = 8;

struct PSweepArgs {
  TTV Z;
  const float* A;
  const float* B1;
  const float* B2;
  long long Aoff[T3F_MAX_D], B1off[T3F_MAX_D], B2off[T3F_MAX_D];
  int ra[T3F_MAX_D + 1];
  int dir;
  float* st1;
  float* st2;
  long long ioff[T3F_MAX_D + 1];
  int J, SPLIT;
  int* err;  // device error word (nullable): a bounded wait that ran out
  int xt;    // right sweep: A / B1 / B2 are transposed copies (r1 x n x r0 cores, see k_xtranspose)
};

__device__ __forceinline__ void fma4x4(float (&acc)[4][4], const float4 a, const float4 b) {
  const float av[4] = {a.x, a.y, a.z, a.w};
  const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
}

// stage slice i of an X-side core (r0 x n x r1) as [K][m] (left: K = row, m = col;
// right: K = col, m = row), zero-padded to RU x RU, with asynchronous copies (the elements
// outside the ranks are zero-filled): 16 bytes at a time when the rows are contiguous and
// aligned (left, r1 a multiple of 4, 16-byte aligned core), else 4 bytes; the caller
// commits and waits
template <int RU>
__device__ __forceinline__ void stage_x_slice_async(float* dst, const float* core, int r0, int n, int r1, int i,
                                                    int dir, bool valid) {
  if (dir == 0 && (r1 & 3) == 0 && (reinterpret_cast<unsigned long long>(core) & 15) == 0) {
    for (int e4 = threadIdx.x; e4 < RU * RU / 4; e4 += blockDim.x) {
      const int K = e4 / (RU / 4), m = 4 * (e4 % (RU / 4));
      const bool ok = valid && K < r0 && m < r1;
      const float* src = ok ? core + ((long long)K * n + i) * r1 + m : core;
      const unsigned sa = (unsigned)__cvta_generic_to_shared(dst + 4 * e4);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(src), "r"(ok ? 16 : 0));
    }
    return;
  }
  for (int e = threadIdx.x; e < RU * RU; e += blockDim.x) {
    const int K = e / RU, m = e % RU;
    const int row = dir == 0 ? K : m, col = dir == 0 ? m : K;
    const bool ok = valid && row < r0 && col < r1;
    const float* src = ok ? core + ((long long)row * n + i) * r1 + col : core;
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst + e);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(src), "r"(ok ? 4 : 0));
  }
}

// Transposed copies Y_k[c][i][r] = X_k[r][i][c] of up to three X-side TTs (batch 1), core k
// at toff[k] (a multiple of 4 floats) of set t's block of tsize floats. A right-style slice
// As[K][m] = X_k[m][i][K] is then the left-style slice Y_k[K][i][m], which the right sweeps and
// the gradient kernel stage with 16-byte copies. kXtParts blocks per (set, core), each a
// contiguous range of the output; writes coalesced.
struct XTransArgs {
  const float* src[3];
  long long soff[T3F_MAX_D], toff[T3F_MAX_D];
  int r[T3F_MAX_D + 1], n[T3F_MAX_D];
  int d;
  long long tsize;
  float* dst;
};

constexpr int kXtParts = 8;

__global__ void __launch_bounds__(256) k_xtranspose(const __grid_constant__ XTransArgs a) {
  const int part = (int)blockIdx.x % kXtParts, tk = (int)blockIdx.x / kXtParts;
  const int t = tk / a.d, k = tk % a.d;
  const int r0 = a.r[k], r1 = a.r[k + 1], n = a.n[k], nr0 = n * r0, sz = r1 * nr0;
  const float* X = a.src[t] + a.soff[k];
  float* Y = a.dst + (long long)t * a.tsize + a.toff[k];
  const int e1 = (int)(((long long)(part + 1) * sz) / kXtParts);
  for (int e = (int)(((long long)part * sz) / kXtParts) + threadIdx.x; e < e1; e += blockDim.x) {
    const int c = e / nr0, rem = e - c * nr0, i = rem / r0, r = rem - i * r0;
    Y[e] = __ldg(X + ((long long)r * n + i) * r1 + c);
  }
}

__device__ __forceinline__ bool ps_bar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > (1ll << 31)) return false;  // about one second
  }
}

template <int RU, bool MIXED>
__global__ void __launch_bounds__(512) k_psweep(const __grid_constant__ PSweepArgs a) {
  extern __shared__ __align__(16) float sm[];
  constexpr int QB = kRZ / 4;        // column blocks
  constexpr int G = (RU / 4) * QB;   // threads per group
  constexpr int TS = RU * kRZ;       // floats of one partial
  const TTV& Z = a.Z;
  const int J = a.J, SP = a.SPLIT, d = Z.d;
  const int nmax = Z.nmax;
  const int tid = threadIdx.x;
  const int ol = tid / (SP * G), h = (tid / G) % SP, lg = tid % G;
  const int qa = lg / QB, qb = lg % QB;
  const int obj = blockIdx.x * J + ol;
  const bool valid = obj < Z.batch;
  constexpr int NX = MIXED ? 3 : 1;
  float* Xs = sm;                                  // [2][NX][SP][RU][RU] (double-buffered)
  float* Zc = Xs + (size_t)2 * NX * SP * RU * RU;  // [J][8][nmax][8]
  float* C1 = Zc + (size_t)J * kRZ * nmax * kRZ;   // [J][8][RU]  (Cur transposed)
  float* C2 = C1 + (size_t)J * TS;                 // mixed only
  float* T1 = C2 + (MIXED ? (size_t)J * TS : 0);   // [J][SP][RU][8]
  float* T2 = T1 + (size_t)J * SP * TS;            // mixed only
  const float* Zp = static_cast<const float*>(Z.p);
  // Z cores whose staged layout [K][i][b] equals their stored one (left sweep, ranks 8 x 8,
  // n_k = nmax, 16-byte aligned blocks) land by one TMA bulk copy per object; the others (and
  // the right sweep, which transposes) keep the zero-filling 4-byte copies
  __shared__ __align__(8) uint64_t zbar;
  uint32_t zph = 0;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((unsigned)__cvta_generic_to_shared(&zbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // initial partials: 1 (and 0) at the starting interface
  for (int e = tid; e < J * TS; e += blockDim.x) {
    C1[e] = (e % TS) == 0 ? 1.0f : 0.0f;
    if (MIXED) C2[e] = 0.0f;
  }
  {
    const int j0 = a.dir == 0 ? 0 : d;
    if (valid && h == 0 && lg == 0) {
      a.st1[a.ioff[j0] + obj] = 1.0f;
      if (MIXED) a.st2[a.ioff[j0] + obj] = 0.0f;
    }
  }
  // X slices of batch ib of core k (sweep step st) into buffer buf, one commit group
  auto issue_batch = [&](int st, int ib, int buf) {
    const int kx = a.dir == 0 ? st : d - 1 - st;
    const int xr0 = a.ra[kx], xr1 = a.ra[kx + 1], xn = Z.n[kx];
    float* X0 = Xs + (size_t)buf * NX * SP * RU * RU;
    // transposed copies (right sweep): the left-style staging of the r1 x n x r0 cores
    const int sr0 = a.xt ? xr1 : xr0, sr1 = a.xt ? xr0 : xr1, sdir = a.xt ? 0 : a.dir;
    for (int hh = 0; hh < SP; ++hh) {
      const int i = ib * SP + hh;
      stage_x_slice_async<RU>(X0 + (size_t)hh * RU * RU, a.A + a.Aoff[kx], sr0, xn, sr1, i, sdir, i < xn);
      if (MIXED) {
        stage_x_slice_async<RU>(X0 + (size_t)(SP + hh) * RU * RU, a.B1 + a.B1off[kx], sr0, xn, sr1, i, sdir, i < xn);
        stage_x_slice_async<RU>(X0 + (size_t)(2 * SP + hh) * RU * RU, a.B2 + a.B2off[kx], sr0, xn, sr1, i, sdir,
                                i < xn);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::);
  };
  int bt = 0;  // running batch index: buffer bt & 1
  issue_batch(0, 0, 0);
  for (int s = 0; s < d; ++s) {
    const int k = a.dir == 0 ? s : d - 1 - s;
    const int r0 = a.ra[k], r1 = a.ra[k + 1], z0 = Z.r[k], z1 = Z.r[k + 1], n = Z.n[k];
    __syncthreads();
    // stage this CTA's Z cores of core k as [K][i][b] (left: K = row, b = col; right: transposed)
    // with 4-byte asynchronous copies (zero-filled outside the ranks), one commit group that
    // the first batch's wait covers; e = ((o * 8 + K) * n + i) * 8 + b, the quotient by n taken
    // through an exact 32-bit reciprocal (indices < 2^13)
    const bool zbulk = a.dir == 0 && z0 == kRZ && z1 == kRZ && n == nmax && (Z.off[k] & 3) == 0 &&
                       (Z.osz[k] & 3) == 0 && (reinterpret_cast<uintptr_t>(Zp) & 15) == 0;
    if (zbulk) {
      if (tid == 0) {
        const int nv = min(J, Z.batch - blockIdx.x * J);
        const uint32_t bytes = (uint32_t)Z.osz[k] * 4u;
        const unsigned zb = (unsigned)__cvta_generic_to_shared(&zbar);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(zb), "r"(bytes * (uint32_t)nv)
                     : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int o = 0; o < nv; ++o)
          asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                           (unsigned)__cvta_generic_to_shared(Zc + (size_t)o * kRZ * nmax * kRZ)),
                       "l"(Zp + core_base(Z, k, blockIdx.x * J + o)), "r"(bytes), "r"(zb)
                       : "memory");
      }
      asm volatile("cp.async.commit_group;\n" ::);  // an empty group keeps the group count
    } else {
      const unsigned mn = 0xffffffffu / (unsigned)n + 1u;
      for (int e = tid; e < J * kRZ * n * kRZ; e += blockDim.x) {
        const unsigned x = (unsigned)e >> 3, q = n == 1 ? x : __umulhi(x, mn);
        const int b = e & 7, i = (int)(x - q * (unsigned)n), K = (int)(q & 7), o = (int)(q >> 3);
        const int row = a.dir == 0 ? K : b, col = a.dir == 0 ? b : K;
        const int ob = blockIdx.x * J + o;
        const bool ok = ob < Z.batch && row < z0 && col < z1;
        const float* src = ok ? Zp + core_base(Z, k, ob) + ((long long)row * n + i) * z1 + col : Zp;
        const unsigned sa = (unsigned)__cvta_generic_to_shared(Zc + (((size_t)o * kRZ + K) * nmax + i) * kRZ + b);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(src), "r"(ok ? 4 : 0));
      }
      asm volatile("cp.async.commit_group;\n" ::);
    }
    float acc1[4][4], acc2[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        acc1[x][y] = 0.0f;
        acc2[x][y] = 0.0f;
      }
    for (int ib = 0; ib * SP < n; ++ib, ++bt) {
      __syncthreads();  // the other buffer's batch has been consumed
      {
        int s2 = s, ib2 = ib + 1;
        if (ib2 * SP >= n) { ++s2; ib2 = 0; }
        if (s2 < d) {
          issue_batch(s2, ib2, (bt + 1) & 1);
          asm volatile("cp.async.wait_group 1;\n" ::);
        } else {
          asm volatile("cp.async.wait_group 0;\n" ::);
        }
      }
      __syncthreads();
      if (ib == 0 && zbulk) {
        if (!ps_bar_wait((unsigned)__cvta_generic_to_shared(&zbar), zph) && tid == 0 && a.err)
          atomicExch(a.err, (int)T3F_ERR_TIMEOUT);
        zph ^= 1u;
      }
      float* const XsB = Xs + (size_t)(bt & 1) * NX * SP * RU * RU;
      const int i = ib * SP + h;
      // T-step: T[m][b] = sum_K CurT[K][m] Zs[K][b]
      if (i < n) {
        float t1[4][4], t2[4][4];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            t1[x][y] = 0.0f;
            t2[x][y] = 0.0f;
          }
#pragma unroll
        for (int K = 0; K < kRZ; ++K) {
          const float4 zv = *reinterpret_cast<const float4*>(Zc + (((size_t)ol * kRZ + K) * nmax + i) * kRZ + 4 * qb);
          const float4 c1 = *reinterpret_cast<const float4*>(C1 + (size_t)ol * TS + K * RU + 4 * qa);
          fma4x4(t1, c1, zv);
          if (MIXED) {
            const float4 c2 = *reinterpret_cast<const float4*>(C2 + (size_t)ol * TS + K * RU + 4 * qa);
            fma4x4(t2, c2, zv);
          }
        }
        float* tb1 = T1 + ((size_t)ol * SP + h) * TS;
#pragma unroll
        for (int x = 0; x < 4; ++x)
          *reinterpret_cast<float4*>(tb1 + (4 * qa + x) * kRZ + 4 * qb) = make_float4(t1[x][0], t1[x][1], t1[x][2], t1[x][3]);
        if (MIXED) {
          float* tb2 = T2 + ((size_t)ol * SP + h) * TS;
#pragma unroll
          for (int x = 0; x < 4; ++x)
            *reinterpret_cast<float4*>(tb2 + (4 * qa + x) * kRZ + 4 * qb) = make_float4(t2[x][0], t2[x][1], t2[x][2], t2[x][3]);
        }
      }
      __syncthreads();
      // accumulate step: Next[m][b] += sum_K As[K][m] T[K][b], K below the contracted X rank
      // (r0 left, r1 right; the staged operands are zero beyond it)
      if (i < n) {
        const float* As = XsB + (size_t)h * RU * RU;
        const float* tb1 = T1 + ((size_t)ol * SP + h) * TS;
        const float* Bs1 = XsB + (size_t)(SP + h) * RU * RU;
        const float* Bs2 = XsB + (size_t)(2 * SP + h) * RU * RU;
        const float* tb2 = T2 + ((size_t)ol * SP + h) * TS;
        const int kr = a.dir == 0 ? r0 : r1;
#pragma unroll 4
        for (int K = 0; K < kr; ++K) {
          const float4 tv1 = *reinterpret_cast<const float4*>(tb1 + K * kRZ + 4 * qb);
          const float4 av = *reinterpret_cast<const float4*>(As + K * RU + 4 * qa);
          fma4x4(acc1, av, tv1);
          if (MIXED) {
            const float4 tv2 = *reinterpret_cast<const float4*>(tb2 + K * kRZ + 4 * qb);
            const float4 b1 = *reinterpret_cast<const float4*>(Bs1 + K * RU + 4 * qa);
            const float4 b2 = *reinterpret_cast<const float4*>(Bs2 + K * RU + 4 * qa);
            fma4x4(acc2, b1, tv2);
            fma4x4(acc2, b2, tv1);
          }
        }
      }
    }
    // sum the SPLIT partial blocks; the new partial becomes CurT and is stored
    __syncthreads();
    {
      float* tb1 = T1 + ((size_t)ol * SP + h) * TS;
#pragma unroll
      for (int x = 0; x < 4; ++x)
        *reinterpret_cast<float4*>(tb1 + (4 * qa + x) * kRZ + 4 * qb) = make_float4(acc1[x][0], acc1[x][1], acc1[x][2], acc1[x][3]);
      if (MIXED) {
        float* tb2 = T2 + ((size_t)ol * SP + h) * TS;
#pragma unroll
        for (int x = 0; x < 4; ++x)
          *reinterpret_cast<float4*>(tb2 + (4 * qa + x) * kRZ + 4 * qb) = make_float4(acc2[x][0], acc2[x][1], acc2[x][2], acc2[x][3]);
      }
    }
    __syncthreads();
    if (h == 0) {
      const int j = a.dir == 0 ? k + 1 : k;
      const int rows = a.dir == 0 ? r1 : r0, cols = a.dir == 0 ? z1 : z0;
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          const int m = 4 * qa + x, b = 4 * qb + y;
          float v1 = 0.0f, v2 = 0.0f;
          for (int hh = 0; hh < SP; ++hh) {
            v1 += T1[((size_t)ol * SP + hh) * TS + m * kRZ + b];
            if (MIXED) v2 += T2[((size_t)ol * SP + hh) * TS + m * kRZ + b];
          }
          C1[(size_t)ol * TS + b * RU + m] = v1;
          if (MIXED) C2[(size_t)ol * TS + b * RU + m] = v2;
          if (valid && m < rows && b < cols) {
            const long long o = a.ioff[j] + (long long)obj * rows * cols + m * cols + b;
            a.st1[o] = v1;
            if (MIXED) a.st2[o] = v2;
          }
        }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Assembly of project_sum: Zhat_k[a][i][a'] = sum_j c_j sum_b L_k^{(j)}[a][b] S_i^{(j)}[a'][b],
// S_i = R_{k+1} Z_k[:, i, :]^T. One CTA per (core k, range of objects) keeps the whole
// RU x n x RU partial in registers (a 4 x 16 block per thread) and writes it to the
// workspace; a second kernel sums the ranges.
// ---------------------------------------------------------------------------------------
struct PAssembleArgs {
  TTV Z;
  int ra[T3F_MAX_D + 1];
  const float* L;
  const float* R;
  long long ioff[T3F_MAX_D + 1];
  const float* c;
  int nranges, range;   // objects per range
  float* part;          // [nranges][compact X-shaped]
  long long xoff[T3F_MAX_D];
  long long xsize;
};

constexpr int kAsmChunk = 4;

template <int RU>
__global__ void __launch_bounds__(512) k_passemble(const __grid_constant__ PAssembleArgs a) {
  extern __shared__ __align__(16) float sm[];
  const TTV& Z = a.Z;
  const int k = blockIdx.x / a.nranges, rg = blockIdx.x % a.nranges;
  const int r0 = a.ra[k], r1 = a.ra[k + 1], z0 = Z.r[k], z1 = Z.r[k + 1], n = Z.n[k];
  const int NC = n * RU;                       // (i, a') columns
  const int NCP = (NC + 15) & ~15;             // row stride of S^T
  const int tid = threadIdx.x;
  const int ta = tid % (RU / 4), tc = tid / (RU / 4);   // 4 rows a, 16 columns (i, a')
  float* LT = sm;                                        // [chunk][8][RU]  c_j L^T
  float* ST = LT + kAsmChunk * kRZ * RU;                 // [chunk][8][NC]  S^T
  float* Rk = ST + (size_t)kAsmChunk * kRZ * ((a.Z.nmax * RU + 15) & ~15);  // [chunk][RU][8]
  float* Zk = Rk + kAsmChunk * RU * kRZ;                 // [chunk][8][n][8]
  const float* Zp = static_cast<const float*>(Z.p);
  float acc[4][16];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 16; ++y) acc[x][y] = 0.0f;
  const int jb = rg * a.range, je = min(Z.batch, jb + a.range);
  const unsigned mn = 0xffffffffu / (unsigned)n + 1u;
  for (int j0 = jb; j0 < je; j0 += kAsmChunk) {
    __syncthreads();
    for (int e = tid; e < kAsmChunk * kRZ * RU; e += blockDim.x) {
      const int m = e % RU, b = (e / RU) % kRZ, o = e / (RU * kRZ), j = j0 + o;
      float v = 0.0f;
      if (j < je && m < r0 && b < z0) v = a.c[j] * a.L[a.ioff[k] + (long long)j * r0 * z0 + m * z0 + b];
      LT[e] = v;
    }
    for (int e = tid; e < kAsmChunk * RU * kRZ; e += blockDim.x) {
      const int b = e % kRZ, m = (e / kRZ) % RU, o = e / (RU * kRZ), j = j0 + o;
      float v = 0.0f;
      if (j < je && m < r1 && b < z1) v = a.R[a.ioff[k + 1] + (long long)j * r1 * z1 + m * z1 + b];
      Rk[e] = v;
    }
    for (int e = tid; e < kAsmChunk * kRZ * n * kRZ; e += blockDim.x) {
      // quotient by n through an exact 32-bit reciprocal (indices < 2^13)
      const unsigned x = (unsigned)e >> 3, q = n == 1 ? x : __umulhi(x, mn);
      const int col = e & 7, i = (int)(x - q * (unsigned)n), row = (int)(q & 7), o = (int)(q >> 3);
      const int j = j0 + o;
      float v = 0.0f;
      if (j < je && row < z0 && col < z1) v = __ldg(Zp + core_base(Z, k, j) + ((long long)row * n + i) * z1 + col);
      Zk[e] = v;
    }
    __syncthreads();
    // S^T[o][b][(i, a')] = sum_delta R[a'][delta] Z[b][i][delta]: a thread item is (o, (i, a'))
    // for all eight b, R's row loaded once; both 8-float rows are 32-byte aligned (two 16-byte
    // loads each) and a warp's lanes share i, so the Z rows are broadcasts
    for (int e = tid; e < kAsmChunk * NC; e += blockDim.x) {
      const int o = e / NC, col = e - o * NC;
      const int i = col / RU, ap = col % RU;
      const float4* rr = reinterpret_cast<const float4*>(Rk + (o * RU + ap) * kRZ);
      const float4 r0 = rr[0], r1 = rr[1];
#pragma unroll
      for (int b = 0; b < kRZ; ++b) {
        const float4* zz = reinterpret_cast<const float4*>(Zk + ((o * kRZ + b) * n + i) * kRZ);
        const float4 q0 = zz[0], q1 = zz[1];
        float s = r0.x * q0.x;
        s = fmaf(r0.y, q0.y, s);
        s = fmaf(r0.z, q0.z, s);
        s = fmaf(r0.w, q0.w, s);
        s = fmaf(r1.x, q1.x, s);
        s = fmaf(r1.y, q1.y, s);
        s = fmaf(r1.z, q1.z, s);
        s = fmaf(r1.w, q1.w, s);
        ST[((size_t)o * kRZ + b) * NCP + col] = s;
      }
    }
    __syncthreads();
    if (tc * 16 < NC) {
#pragma unroll
      for (int o = 0; o < kAsmChunk; ++o)
#pragma unroll
        for (int b = 0; b < kRZ; ++b) {
          const float4 lv = *reinterpret_cast<const float4*>(LT + (o * kRZ + b) * RU + 4 * ta);
          const float* sv = ST + ((size_t)o * kRZ + b) * NCP + 16 * tc;
          const float lvv[4] = {lv.x, lv.y, lv.z, lv.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float4 s4 = *reinterpret_cast<const float4*>(sv + 4 * q);
#pragma unroll
            for (int x = 0; x < 4; ++x) {
              acc[x][4 * q] = fmaf(lvv[x], s4.x, acc[x][4 * q]);
              acc[x][4 * q + 1] = fmaf(lvv[x], s4.y, acc[x][4 * q + 1]);
              acc[x][4 * q + 2] = fmaf(lvv[x], s4.z, acc[x][4 * q + 2]);
              acc[x][4 * q + 3] = fmaf(lvv[x], s4.w, acc[x][4 * q + 3]);
            }
          }
        }
    }
  }
  // write the partial (compact X-shaped layout of core k)
  if (tc * 16 < NC) {
    float* out = a.part + (long long)rg * a.xsize + a.xoff[k];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int m = 4 * ta + x;
      if (m >= r0) continue;
#pragma unroll
      for (int y = 0; y < 16; ++y) {
        const int col = 16 * tc + y;
        const int i = col / RU, ap = col % RU;
        if (i < n && ap < r1) out[((long long)m * n + i) * r1 + ap] = acc[x][y];
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Core gradients of the adjoint: dZ_j^k[:, i, :] = c_j (P_k^T X1_i + L_k^T X2_i) with
// X1_i = V_i R_{k+1}, X2_i = W_i R_{k+1} + U_i Q_{k+1}. Cores are independent, so the grid
// covers (object tile, core); slices are split over SPLIT groups as in the sweeps.
// ---------------------------------------------------------------------------------------
struct PGradFastArgs {
  TTV Z;
  const float *U, *V, *W;
  long long Xoff[T3F_MAX_D];
  int ra[T3F_MAX_D + 1];
  const float *L, *R, *P, *Q;
  long long ioff[T3F_MAX_D + 1];
  const float* c;
  float* dZ;
  float* dc;
  int J, SPLIT, ntiles;
  int xt;  // U / V / W are transposed copies (r1 x n x r0 cores, see k_xtranspose)
};

template <int RU>
__global__ void __launch_bounds__(RU == 32 ? 512 : 256) k_pgrad(const __grid_constant__ PGradFastArgs a) {
  extern __shared__ __align__(16) float sm[];
  constexpr int QB = kRZ / 4, G = (RU / 4) * QB, TS = RU * kRZ;
  const TTV& Z = a.Z;
  const int J = a.J, SP = a.SPLIT;
  const int tile = blockIdx.x % a.ntiles, k = blockIdx.x / a.ntiles;
  const int tid = threadIdx.x;
  const int ol = tid / (SP * G), h = (tid / G) % SP, lg = tid % G;
  const int qa = lg / QB, qb = lg % QB;
  const int obj = tile * J + ol;
  const bool valid = obj < Z.batch;
  const int r0 = a.ra[k], r1 = a.ra[k + 1], z0 = Z.r[k], z1 = Z.r[k + 1], n = Z.n[k];
  float* Xs = sm;                                   // [3][SP][RU][RU]: V^T, W^T, U^T as [K][m]
  float* PL = Xs + (size_t)3 * SP * RU * RU;        // [J][2][RU][8]: P_k, L_k (rows m, cols beta)
  float* RQ = PL + (size_t)J * 2 * TS;              // [J][2][RU][8]: R_{k+1}, Q_{k+1} (rows K, cols b)
  float* XB = RQ + (size_t)J * 2 * TS;              // [J][SP][2][RU][8]: X1, X2
  if (k == Z.d - 1 && a.dc && h == 0 && lg == 0 && valid) a.dc[obj] = a.P[a.ioff[Z.d] + obj];
  if (!a.dZ) return;
  for (int e = tid; e < J * 2 * TS; e += blockDim.x) {
    const int b = e % kRZ, m = (e / kRZ) % RU, w = (e / TS) % 2, o = e / (2 * TS);
    const int ob = tile * J + o;
    float pl = 0.0f, rq = 0.0f;
    if (ob < Z.batch) {
      if (m < r0 && b < z0) pl = (w == 0 ? a.P : a.L)[a.ioff[k] + (long long)ob * r0 * z0 + m * z0 + b];
      if (m < r1 && b < z1) rq = (w == 0 ? a.R : a.Q)[a.ioff[k + 1] + (long long)ob * r1 * z1 + m * z1 + b];
    }
    PL[e] = pl;
    RQ[e] = rq;
  }
  const float cj = valid ? a.c[obj] : 0.0f;
  float* outb = valid ? a.dZ + core_base(Z, k, obj) : nullptr;
  // slices of batch ib, right-style (As[K][m] = X_k[m][i][K]), as one commit group; the next
  // batch is issued once the current one has been consumed, so its copies overlap the dZ step
  auto issue_batch = [&](int ib) {
    const int sr0 = a.xt ? r1 : r0, sr1 = a.xt ? r0 : r1, sdir = a.xt ? 0 : 1;
    for (int hh = 0; hh < SP; ++hh) {
      const int i = ib * SP + hh;
      stage_x_slice_async<RU>(Xs + (size_t)(0 * SP + hh) * RU * RU, a.V + a.Xoff[k], sr0, n, sr1, i, sdir, i < n);
      stage_x_slice_async<RU>(Xs + (size_t)(1 * SP + hh) * RU * RU, a.W + a.Xoff[k], sr0, n, sr1, i, sdir, i < n);
      stage_x_slice_async<RU>(Xs + (size_t)(2 * SP + hh) * RU * RU, a.U + a.Xoff[k], sr0, n, sr1, i, sdir, i < n);
    }
    asm volatile("cp.async.commit_group;\n" ::);
  };
  issue_batch(0);
  for (int ib = 0; ib * SP < n; ++ib) {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    const int i = ib * SP + h;
    if (i < n) {
      float x1[4][4], x2[4][4];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          x1[x][y] = 0.0f;
          x2[x][y] = 0.0f;
        }
      const float* Vs = Xs + (size_t)(0 * SP + h) * RU * RU;
      const float* Ws = Xs + (size_t)(1 * SP + h) * RU * RU;
      const float* Us = Xs + (size_t)(2 * SP + h) * RU * RU;
      const float* Rm = RQ + (size_t)ol * 2 * TS;
      const float* Qm = Rm + TS;
      // K below the X rank r1 (the staged slices and R, Q are zero beyond it)
#pragma unroll 4
      for (int K = 0; K < r1; ++K) {
        const float4 rv = *reinterpret_cast<const float4*>(Rm + K * kRZ + 4 * qb);
        const float4 qv = *reinterpret_cast<const float4*>(Qm + K * kRZ + 4 * qb);
        fma4x4(x1, *reinterpret_cast<const float4*>(Vs + K * RU + 4 * qa), rv);
        fma4x4(x2, *reinterpret_cast<const float4*>(Ws + K * RU + 4 * qa), rv);
        fma4x4(x2, *reinterpret_cast<const float4*>(Us + K * RU + 4 * qa), qv);
      }
      float* xb = XB + ((size_t)ol * SP + h) * 2 * TS;
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        *reinterpret_cast<float4*>(xb + (4 * qa + x) * kRZ + 4 * qb) = make_float4(x1[x][0], x1[x][1], x1[x][2], x1[x][3]);
        *reinterpret_cast<float4*>(xb + TS + (4 * qa + x) * kRZ + 4 * qb) = make_float4(x2[x][0], x2[x][1], x2[x][2], x2[x][3]);
      }
    }
    __syncthreads();
    if ((ib + 1) * SP < n) issue_batch(ib + 1);
    // dZ_i[beta][b] = c_j sum_m (P[m][beta] X1[m][b] + L[m][beta] X2[m][b]); G threads per
    // (object, slice) cover the 8 x 8 block as 16 rows-of-4
    if (i < n && valid) {
      const float* xb = XB + ((size_t)ol * SP + h) * 2 * TS;
      const float* Pm = PL + (size_t)ol * 2 * TS;
      const float* Lm = Pm + TS;
      for (int blk = lg; blk < kRZ * QB; blk += G) {
        const int beta = blk / QB, bq = blk % QB;
        float s[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int m = 0; m < RU; ++m) {
          const float pm = Pm[m * kRZ + beta], lm = Lm[m * kRZ + beta];
          const float4 v1 = *reinterpret_cast<const float4*>(xb + m * kRZ + 4 * bq);
          const float4 v2 = *reinterpret_cast<const float4*>(xb + TS + m * kRZ + 4 * bq);
          s[0] = fmaf(pm, v1.x, fmaf(lm, v2.x, s[0]));
          s[1] = fmaf(pm, v1.y, fmaf(lm, v2.y, s[1]));
          s[2] = fmaf(pm, v1.z, fmaf(lm, v2.z, s[2]));
          s[3] = fmaf(pm, v1.w, fmaf(lm, v2.w, s[3]));
        }
        if (beta < z0)
          for (int y = 0; y < 4; ++y) {
            const int b = 4 * bq + y;
            if (b < z1) outb[((long long)beta * n + i) * z1 + b] = cj * s[y];
          }
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------

static int pick_RU(int r) { return r <= 8 ? 8 : (r <= 16 ? 16 : (r <= 32 ? 32 : 0)); }

bool psweep_supported(const TTV& X, const TTV& Z) {
  return pick_RU(X.rmax) != 0 && Z.rmax <= kRZ && Z.nmax <= 64;
}

static int sm_count() { return device_sm_count(); }

static void plan_tiles(int RU, int batch, int* J, int* SP) {
  const int G = (RU / 4) * (kRZ / 4);
  *SP = 4;
  while (*SP > 1 && G * *SP > 512) *SP /= 2;
  int j = (batch + sm_count() - 1) / sm_count();
  const int jmax = 512 / (G * *SP);
  if (j > jmax) j = jmax;
  if (j < 1) j = 1;
  *J = j;
}

static size_t psweep_smem(int RU, bool mixed, int J, int SP, int nmax) {
  const size_t TS = (size_t)RU * kRZ;
  size_t f = (size_t)2 * (mixed ? 3 : 1) * SP * RU * RU + (size_t)J * kRZ * nmax * kRZ + (size_t)J * TS * (mixed ? 2 : 1) +
             (size_t)J * SP * TS * (mixed ? 2 : 1);
  return f * sizeof(float);
}

template <int RU, bool MIXED>
static t3f_status launch_psweep_t(PSweepArgs& a, cudaStream_t s) {
  const size_t smem = psweep_smem(RU, MIXED, a.J, a.SPLIT, a.Z.nmax);
  if (smem > 227 * 1024) return T3F_ERR_UNSUPPORTED;
  auto kern = k_psweep<RU, MIXED>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return T3F_ERR_CUDA;
  const int G = (RU / 4) * (kRZ / 4);
  const unsigned grid = (unsigned)((a.Z.batch + a.J - 1) / a.J);
  kern<<<grid, a.J * a.SPLIT * G, smem, s>>>(a);
  return launch_status();
}

// dir 0: left sweep (A = U [, B1 = V, B2 = W]); dir 1: right sweep (A = V [, B1 = U, B2 = W]).
t3f_status run_psweep(const TTV& X, const TTV& Z, int dir, const float* A, const float* B1, const float* B2,
                      float* st1, float* st2, const long long* ioff, cudaStream_t s, int* err, const long long* xtoff) {
  PSweepArgs a;
  memset(&a, 0, sizeof(a));
  a.err = err;
  a.Z = Z;
  a.A = A;
  a.B1 = B1;
  a.B2 = B2;
  a.xt = xtoff != nullptr && dir == 1;
  for (int k = 0; k < X.d; ++k) a.Aoff[k] = a.B1off[k] = a.B2off[k] = a.xt ? xtoff[k] : X.off[k];
  for (int k = 0; k <= X.d; ++k) {
    a.ra[k] = X.r[k];
    a.ioff[k] = ioff[k];
  }
  a.dir = dir;
  a.st1 = st1;
  a.st2 = st2;
  const int RU = pick_RU(X.rmax);
  plan_tiles(RU, Z.batch, &a.J, &a.SPLIT);
  const bool mixed = st2 != nullptr;
  switch (RU) {
    case 8: return mixed ? launch_psweep_t<8, true>(a, s) : launch_psweep_t<8, false>(a, s);
    case 16: return mixed ? launch_psweep_t<16, true>(a, s) : launch_psweep_t<16, false>(a, s);
    default: return mixed ? launch_psweep_t<32, true>(a, s) : launch_psweep_t<32, false>(a, s);
  }
}

long long xtranspose_offsets(const TTV& X, long long* toff) {
  long long o = 0;
  for (int k = 0; k < X.d; ++k) {
    if (toff) toff[k] = o;
    o += (X.osz[k] + 3) & ~3LL;
  }
  return o;
}

t3f_status run_xtranspose(const TTV& X, const float* const* srcs, int nsets, float* dst, cudaStream_t s) {
  if (nsets < 1 || nsets > 3 || (reinterpret_cast<uintptr_t>(dst) & 15)) return T3F_ERR_ARG;
  XTransArgs a;
  memset(&a, 0, sizeof(a));
  for (int t = 0; t < nsets; ++t) a.src[t] = srcs[t];
  a.d = X.d;
  a.dst = dst;
  a.tsize = xtranspose_offsets(X, a.toff);
  for (int k = 0; k < X.d; ++k) {
    a.soff[k] = X.off[k];
    a.n[k] = X.n[k];
  }
  for (int k = 0; k <= X.d; ++k) a.r[k] = X.r[k];
  k_xtranspose<<<(unsigned)(nsets * X.d * kXtParts), 256, 0, s>>>(a);
  return launch_status();
}

int passemble_ranges(const TTV& Z) {
  // enough (core, range) CTAs to cover the GPU about twice
  int nr = (2 * sm_count() + Z.d - 1) / Z.d;
  if (nr > Z.batch) nr = Z.batch;
  return nr < 1 ? 1 : nr;
}

template <int RU>
static t3f_status launch_passemble_t(PAssembleArgs& a, cudaStream_t s) {
  const int NC = a.Z.nmax * RU;
  const int NCP = (NC + 15) & ~15;
  const int threads = (RU / 4) * (NCP / 16);
  if (threads > 512) return T3F_ERR_UNSUPPORTED;
  const size_t smem = sizeof(float) * ((size_t)kAsmChunk * kRZ * RU + (size_t)kAsmChunk * kRZ * NCP +
                                       (size_t)kAsmChunk * RU * kRZ + (size_t)kAsmChunk * kRZ * a.Z.nmax * kRZ);
  auto kern = k_passemble<RU>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return T3F_ERR_CUDA;
  kern<<<(unsigned)(a.Z.d * a.nranges), threads, smem, s>>>(a);
  return launch_status();
}

t3f_status run_passemble(const TTV& X, const TTV& Z, const float* L, const float* R, const long long* ioff,
                         const float* c, float* part, int nranges, cudaStream_t s) {
  PAssembleArgs a;
  memset(&a, 0, sizeof(a));
  a.Z = Z;
  for (int k = 0; k <= X.d; ++k) {
    a.ra[k] = X.r[k];
    a.ioff[k] = ioff[k];
  }
  a.L = L;
  a.R = R;
  a.c = c;
  a.nranges = nranges;
  a.range = (Z.batch + nranges - 1) / nranges;
  a.part = part;
  long long o = 0;
  for (int k = 0; k < X.d; ++k) {
    a.xoff[k] = o;
    o += X.osz[k];
  }
  a.xsize = o;
  switch (pick_RU(X.rmax)) {
    case 8: return launch_passemble_t<8>(a, s);
    case 16: return launch_passemble_t<16>(a, s);
    default: return launch_passemble_t<32>(a, s);
  }
}

template <int RU>
static t3f_status launch_pgrad_t(PGradFastArgs& a, cudaStream_t s) {
  const size_t TS = (size_t)RU * kRZ;
  const size_t smem = sizeof(float) * ((size_t)3 * a.SPLIT * RU * RU + (size_t)a.J * 4 * TS + (size_t)a.J * a.SPLIT * 2 * TS);
  const int G = (RU / 4) * (kRZ / 4);
  if (smem > 227 * 1024 || a.J * a.SPLIT * G > (RU == 32 ? 512 : 256)) return T3F_ERR_UNSUPPORTED;
  auto kern = k_pgrad<RU>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return T3F_ERR_CUDA;
  kern<<<(unsigned)(a.ntiles * a.Z.d), a.J * a.SPLIT * G, smem, s>>>(a);
  return launch_status();
}

t3f_status run_pgrad(const TTV& X, const TTV& Z, const float* U, const float* V, const float* W, const float* L,
                     const float* R, const float* P, const float* Q, const long long* ioff, const float* c, float* dZ,
                     float* dc, cudaStream_t s, const long long* xtoff) {
  PGradFastArgs a;
  memset(&a, 0, sizeof(a));
  a.Z = Z;
  a.U = U;
  a.V = V;
  a.W = W;
  a.xt = xtoff != nullptr;
  for (int k = 0; k < X.d; ++k) a.Xoff[k] = a.xt ? xtoff[k] : X.off[k];
  for (int k = 0; k <= X.d; ++k) {
    a.ra[k] = X.r[k];
    a.ioff[k] = ioff[k];
  }
  a.L = L;
  a.R = R;
  a.P = P;
  a.Q = Q;
  a.c = c;
  a.dZ = dZ;
  a.dc = dc;
  const int RU = pick_RU(X.rmax);
  const int G = (RU / 4) * (kRZ / 4);
  a.SPLIT = 4;
  while (a.SPLIT > 1 && G * a.SPLIT > 512) a.SPLIT /= 2;
  a.J = 512 / (G * a.SPLIT);
  // objects per CTA: the X slices a CTA stages serve all of them (8 at RU = 32, where the
  // kernel's registers allow 512 threads)
  if (a.J > (RU == 32 ? 8 : 4)) a.J = RU == 32 ? 8 : 4;
  a.ntiles = (Z.batch + a.J - 1) / a.J;
  switch (RU) {
    case 8: return launch_pgrad_t<8>(a, s);
    case 16: return launch_pgrad_t<16>(a, s);
    default: return launch_pgrad_t<32>(a, s);
  }
}

}  // namespace t3f
