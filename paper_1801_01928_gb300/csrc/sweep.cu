// Generic transfer-matrix sweep over pairs of TT objects (FP32 accumulation).
//
// For a pair (A, B) of TT-vectors with equal modes the left partials are
//   M_0 = 1,  M_k = sum_i A_k[:, i, :]^T M_{k-1} B_k[:, i, :]          (r^A_k x r^B_k)
// and the right partials
//   R_{d+1} = 1,  R_k = sum_i A_k[:, i, :] R_{k+1} B_k[:, i, :]^T      (r^A_{k-1} x r^B_{k-1});
// M_d = R_1 = <A, B>. These sweeps carry the inner products and Gram matrices of the
// paper's Section 4 ('norm', 'gram') and the left/right interfaces of the tangent-space
// projection of Section 3.2.
//
// One CTA owns a tile of TA x TB pairs (or TA diagonal pairs in zip mode). Per core it
// stages one mode slice of each tile object in shared memory, forms the per-pair products
// with the current partial and accumulates the next partial; every partial of the tile
// stays in shared memory for the whole sweep.
#include <algorithm>

#include "t3f_internal.cuh"

namespace t3f {

struct SweepArgs {
  TTV A, B;
  int TA, TB;       // tile objects on each side (zip: TB == TA, pairs on the diagonal)
  int RA, RB;       // max ranks (shared-memory strides)
  int dir;          // 0 = left-to-right, 1 = right-to-left
  int zip;          // 1 = pairs (a, a) only
  float* out;       // [bA * bB] (or [bA] in zip mode), nullable
  float* store;     // partial store, nullable
  long long ioff[T3F_MAX_D + 1];
};

template <typename TAt, typename TBt>
__global__ void __launch_bounds__(256) k_pair_sweep(const __grid_constant__ SweepArgs a) {
  extern __shared__ float sm[];
  const TTV& A = a.A;
  const TTV& B = a.B;
  const int TA = a.TA, TB = a.TB, RA = a.RA, RB = a.RB;
  const int P = a.zip ? TA : TA * TB;
  const int PS = RA * RB;  // per-pair stride of a partial
  float* As = sm;
  float* Bs = As + TA * RA * RA;
  float* Mc = Bs + TB * RB * RB;
  float* Mn = Mc + P * PS;
  float* Tt = Mn + P * PS;
  const TAt* Ap = static_cast<const TAt*>(A.p);
  const TBt* Bp = static_cast<const TBt*>(B.p);
  const int bA = A.batch, bB = B.batch;
  int a0, b0;
  if (a.zip) {
    a0 = blockIdx.x * TA;
    b0 = a0;
  } else {
    const int ntb = (bB + TB - 1) / TB;
    a0 = (blockIdx.x / ntb) * TA;
    b0 = (blockIdx.x % ntb) * TB;
  }
  const int tid = threadIdx.x, nth = blockDim.x;
  const int d = A.d;

  auto pa = [&](int p) { return a.zip ? p : p / TB; };
  auto pb = [&](int p) { return a.zip ? p : p % TB; };
  auto pair_valid = [&](int p) { return a0 + pa(p) < bA && b0 + pb(p) < bB; };
  auto pair_id = [&](int p) -> long long {
    return a.zip ? (long long)(a0 + p) : (long long)(a0 + pa(p)) * bB + (b0 + pb(p));
  };

  for (int p = tid; p < P; p += nth) Mc[p * PS] = 1.0f;
  __syncthreads();
  if (a.store) {
    const int j = a.dir == 0 ? 0 : d;
    for (int p = tid; p < P; p += nth)
      if (pair_valid(p)) a.store[a.ioff[j] + pair_id(p)] = 1.0f;
  }

  for (int s = 0; s < d; ++s) {
    const int k = a.dir == 0 ? s : d - 1 - s;
    const int rA0 = A.r[k], rA1 = A.r[k + 1], rB0 = B.r[k], rB1 = B.r[k + 1];
    const int nk = A.n[k];
    const int nr = a.dir == 0 ? rA1 : rA0;  // rows of the next partial
    const int nc = a.dir == 0 ? rB1 : rB0;  // cols of the next partial
    for (int e = tid; e < P * nr * nc; e += nth) {
      const int p = e / (nr * nc), q = e % (nr * nc);
      Mn[p * PS + q] = 0.0f;
    }
    for (int i = 0; i < nk; ++i) {
      // stage slice i of core k for the tile's objects
      for (int e = tid; e < TA * rA0 * rA1; e += nth) {
        const int t = e / (rA0 * rA1), q = e % (rA0 * rA1);
        const int al = q / rA1, be = q % rA1;
        const int obj = a0 + t;
        As[t * RA * RA + q] =
            obj < bA ? ldf(Ap, core_base(A, k, obj) + ((long long)al * nk + i) * rA1 + be) : 0.0f;
      }
      for (int e = tid; e < TB * rB0 * rB1; e += nth) {
        const int t = e / (rB0 * rB1), q = e % (rB0 * rB1);
        const int al = q / rB1, be = q % rB1;
        const int obj = b0 + t;
        Bs[t * RB * RB + q] =
            obj < bB ? ldf(Bp, core_base(B, k, obj) + ((long long)al * nk + i) * rB1 + be) : 0.0f;
      }
      __syncthreads();
      if (a.dir == 0) {
        // T[p] = M[p] (rA0 x rB0) * Bslice (rB0 x rB1)
        for (int e = tid; e < P * rA0 * rB1; e += nth) {
          const int p = e / (rA0 * rB1), q = e % (rA0 * rB1);
          const int al = q / rB1, bp = q % rB1;
          const float* M = Mc + p * PS + al * rB0;
          const float* Bsl = Bs + pb(p) * RB * RB + bp;
          float acc = 0.0f;
          for (int be = 0; be < rB0; ++be) acc = fmaf(M[be], Bsl[be * rB1], acc);
          Tt[p * PS + q] = acc;
        }
        __syncthreads();
        // Mn[p] += Aslice^T (rA1 x rA0) * T[p] (rA0 x rB1)
        for (int e = tid; e < P * rA1 * rB1; e += nth) {
          const int p = e / (rA1 * rB1), q = e % (rA1 * rB1);
          const int ap = q / rB1, bp = q % rB1;
          const float* Asl = As + pa(p) * RA * RA + ap;
          const float* T = Tt + p * PS + bp;
          float acc = 0.0f;
          for (int al = 0; al < rA0; ++al) acc = fmaf(Asl[al * rA1], T[al * rB1], acc);
          Mn[p * PS + q] += acc;
        }
      } else {
        // T[p] = Aslice (rA0 x rA1) * R[p] (rA1 x rB1)
        for (int e = tid; e < P * rA0 * rB1; e += nth) {
          const int p = e / (rA0 * rB1), q = e % (rA0 * rB1);
          const int al = q / rB1, bp = q % rB1;
          const float* Asl = As + pa(p) * RA * RA + al * rA1;
          const float* R = Mc + p * PS + bp;
          float acc = 0.0f;
          for (int ap = 0; ap < rA1; ++ap) acc = fmaf(Asl[ap], R[ap * rB1], acc);
          Tt[p * PS + q] = acc;
        }
        __syncthreads();
        // Mn[p] += T[p] (rA0 x rB1) * Bslice^T (rB1 x rB0)
        for (int e = tid; e < P * rA0 * rB0; e += nth) {
          const int p = e / (rA0 * rB0), q = e % (rA0 * rB0);
          const int al = q / rB0, be = q % rB0;
          const float* T = Tt + p * PS + al * rB1;
          const float* Bsl = Bs + pb(p) * RB * RB + be * rB1;
          float acc = 0.0f;
          for (int bp = 0; bp < rB1; ++bp) acc = fmaf(T[bp], Bsl[bp], acc);
          Mn[p * PS + q] += acc;
        }
      }
      __syncthreads();
    }
    float* t = Mc;
    Mc = Mn;
    Mn = t;
    if (a.store) {
      const int j = a.dir == 0 ? k + 1 : k;
      const long long sz = (long long)nr * nc;
      for (int e = tid; e < P * nr * nc; e += nth) {
        const int p = e / (nr * nc), q = e % (nr * nc);
        if (pair_valid(p)) a.store[a.ioff[j] + pair_id(p) * sz + q] = Mc[p * PS + q];
      }
    }
  }
  if (a.out) {
    for (int p = tid; p < P; p += nth)
      if (pair_valid(p)) a.out[pair_id(p)] = Mc[p * PS];
  }
}

static size_t sweep_smem(int TA, int TB, int RA, int RB, bool zip) {
  const long long P = zip ? TA : (long long)TA * TB;
  return sizeof(float) * ((size_t)TA * RA * RA + (size_t)TB * RB * RB + 3 * P * RA * RB);
}

static SweepPlan plan_generic(const TTV& A, const TTV& B, bool zip) {
  static const int cand[] = {16, 8, 4, 2, 1};
  const size_t cap = 96 * 1024;
  SweepPlan best{1, 1, sweep_smem(1, 1, A.rmax, B.rmax, zip)};
  long long bestScore = -1;
  for (int ta : cand) {
    if (ta > 1 && ta / 2 >= A.batch) continue;
    for (int tb : cand) {
      if (zip && tb != ta) continue;
      if (!zip && tb > 1 && tb / 2 >= B.batch) continue;
      const size_t smem = sweep_smem(ta, tb, A.rmax, B.rmax, zip);
      if (smem > cap) continue;
      const long long ntiles = zip ? (A.batch + ta - 1) / ta
                                   : (long long)((A.batch + ta - 1) / ta) * ((B.batch + tb - 1) / tb);
      const long long pairs = zip ? ta : (long long)ta * tb;
      // prefer enough CTAs for two per SM, then the largest tile
      const long long score = (ntiles >= 304 ? (1LL << 40) : ntiles << 20) + pairs;
      if (score > bestScore) {
        bestScore = score;
        best = SweepPlan{ta, tb, smem};
      }
    }
  }
  return best;
}

SweepPlan plan_sweep(const TTV& A, const TTV& B, int) { return plan_generic(A, B, false); }

long long partial_offsets(const TTV& A, const TTV& B, long long pairs, long long* ioff) {
  long long o = 0;
  for (int j = 0; j <= A.d; ++j) {
    ioff[j] = o;
    o += pairs * A.r[j] * B.r[j];
  }
  return o;
}

static t3f_status launch_sweep(const TTV& A, const TTV& B, int dir, bool zip, float* out,
                               float* store, const long long* ioff, cudaStream_t s) {
  SweepPlan pl = plan_generic(A, B, zip);
  SweepArgs args;
  args.A = A;
  args.B = B;
  args.TA = pl.TA;
  args.TB = zip ? pl.TA : pl.TB;
  args.RA = A.rmax;
  args.RB = B.rmax;
  args.dir = dir;
  args.zip = zip ? 1 : 0;
  args.out = out;
  args.store = store;
  for (int j = 0; j <= T3F_MAX_D; ++j) args.ioff[j] = (ioff && j <= A.d) ? ioff[j] : 0;
  const long long grid = zip ? (A.batch + pl.TA - 1) / pl.TA
                             : (long long)((A.batch + pl.TA - 1) / pl.TA) * ((B.batch + pl.TB - 1) / pl.TB);
  if (grid > 0x7fffffffLL) return T3F_ERR_UNSUPPORTED;
  if (A.dtype == T3F_F32 && B.dtype == T3F_F32) {
    auto kern = k_pair_sweep<float, float>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem) != cudaSuccess)
      return T3F_ERR_CUDA;
    kern<<<(unsigned)grid, 256, pl.smem, s>>>(args);
  } else if (A.dtype == T3F_BF16 && B.dtype == T3F_BF16) {
    auto kern = k_pair_sweep<__nv_bfloat16, __nv_bfloat16>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem) != cudaSuccess)
      return T3F_ERR_CUDA;
    kern<<<(unsigned)grid, 256, pl.smem, s>>>(args);
  } else {
    return T3F_ERR_DTYPE;
  }
  return launch_status();
}

// Squared norms <A_a, A_a> (paper Section 4, 'norm'): one CTA per object, whole cores staged
// in shared memory (the next core's copies in flight while the current one computes). Per core
// every slice's T_i = M A_i is formed in one pass (n r0 r1 outputs, K = r0) and
// M' = sum_i A_i^T T_i in a second (r1 x r1 outputs, K = n r0): two barrier intervals per
// core instead of a slice-by-slice walk.
struct SelfSweepArgs {
  TTV A;
  float* out;
  int maxcore;  // floats of the largest core, rounded up to 4
};

template <typename ST>
__global__ void __launch_bounds__(256) k_self_sweep(const __grid_constant__ SelfSweepArgs a) {
  extern __shared__ __align__(16) float sm[];
  const TTV& A = a.A;
  const int obj = blockIdx.x, tid = threadIdx.x, nth = blockDim.x, d = A.d;
  float* M = sm + 2 * a.maxcore;     // r0 x r0 (current partial)
  float* T = M + A.rmax * A.rmax;    // [i][al][be]
  const ST* Ap = static_cast<const ST*>(A.p);
  auto stage = [&](int k) {
    float* buf = sm + (k & 1) * a.maxcore;
    const long long base = core_base(A, k, obj), sz = A.osz[k];
    for (long long e = tid; e < sz; e += nth) {
      if (sizeof(ST) == 4) {
        const unsigned sa = (unsigned)__cvta_generic_to_shared(buf + e);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(reinterpret_cast<const float*>(Ap) + base + e));
      } else {
        buf[e] = ldf<ST>(Ap, base + e);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::);
  };
  if (tid == 0) M[0] = 1.0f;
  stage(0);
  for (int k = 0; k < d; ++k) {
    if (k + 1 < d) {
      stage(k + 1);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();
    const float* C = sm + (k & 1) * a.maxcore;  // A_k[al][i][be] at (al n + i) r1 + be
    const int r0 = A.r[k], n = A.n[k], r1 = A.r[k + 1];
    for (int e = tid; e < n * r0 * r1; e += nth) {
      const int i = e / (r0 * r1), q = e - i * r0 * r1, al = q / r1, be = q - al * r1;
      float acc = 0.0f;
      for (int c = 0; c < r0; ++c) acc = fmaf(M[al * r0 + c], C[(c * n + i) * r1 + be], acc);
      T[e] = acc;
    }
    __syncthreads();
    for (int e = tid; e < r1 * r1; e += nth) {
      const int ap = e / r1, bp = e - ap * r1;
      float acc = 0.0f;
      for (int i = 0; i < n; ++i)
        for (int al = 0; al < r0; ++al) acc = fmaf(C[(al * n + i) * r1 + ap], T[(i * r0 + al) * r1 + bp], acc);
      M[e] = acc;
    }
    __syncthreads();
  }
  if (tid == 0) a.out[obj] = M[0];
}

static size_t self_sweep_smem(const TTV& A, int* maxcore) {
  long long mc = 0;
  for (int k = 0; k < A.d; ++k) mc = std::max(mc, A.osz[k]);
  mc = (mc + 3) & ~3LL;
  *maxcore = (int)mc;
  return sizeof(float) * (size_t)(3 * mc + (long long)A.rmax * A.rmax);
}

t3f_status run_self_sweep(const TTV& A, float* out, cudaStream_t s) {
  SelfSweepArgs args;
  args.A = A;
  args.out = out;
  const size_t smem = self_sweep_smem(A, &args.maxcore);
  if (smem > 96 * 1024 || A.batch > 0x7fffffff) return run_zip_sweep(A, A, out, s);
  if (A.batch == 0) return T3F_OK;
  if (A.dtype == T3F_F32) {
    auto kern = k_self_sweep<float>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return T3F_ERR_CUDA;
    kern<<<(unsigned)A.batch, 256, smem, s>>>(args);
  } else if (A.dtype == T3F_BF16) {
    auto kern = k_self_sweep<__nv_bfloat16>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return T3F_ERR_CUDA;
    kern<<<(unsigned)A.batch, 256, smem, s>>>(args);
  } else {
    return T3F_ERR_DTYPE;
  }
  return launch_status();
}

t3f_status run_pair_sweep(const TTV& A, const TTV& B, int dir, float* out, float* store,
                          const long long* ioff, cudaStream_t s) {
  return launch_sweep(A, B, dir, false, out, store, ioff, s);
}

t3f_status run_zip_sweep(const TTV& A, const TTV& B, float* out, cudaStream_t s) {
  return launch_sweep(A, B, 0, true, out, nullptr, nullptr, s);
}

}  // namespace t3f
