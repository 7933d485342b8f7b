// Gram matrices, norms and the Gram adjoint (paper Section 4 'gram' / 'norm', batch
// broadcasting of Section 3.1).
#include <math.h>

#include "t3f_internal.cuh"

namespace t3f {

static t3f_status gram_views(const t3f_tt* A, const t3f_tt* B, TTV* va, TTV* vb) {
  T3F_CHECK(make_view(A, va, -1, false));
  T3F_CHECK(make_view(B, vb, -1, false));
  if (va->dtype == T3F_F64 || va->dtype != vb->dtype) return T3F_ERR_DTYPE;
  if (va->d != vb->d) return T3F_ERR_SHAPE;
  for (int k = 0; k < va->d; ++k)
    if (va->n[k] != vb->n[k]) return T3F_ERR_SHAPE;
  if (va->rmax > T3F_MAX_RANK || vb->rmax > T3F_MAX_RANK) return T3F_ERR_UNSUPPORTED;
  return T3F_OK;
}

// ---------------------------------------------------------------------------------------
// Adjoint: right sweep over the tile's pairs, reading the stored left partials M_k, and
// scattering   dA_k[:, i, :] += g_ab M_k (B_k[:, i, :] R_{k+1}^T)
//              dB_k[:, i, :] += g_ab M_k^T (A_k[:, i, :] R_{k+1})
// ---------------------------------------------------------------------------------------

struct GramBwdArgs {
  TTV A, B;
  int TA, TB, RA, RB;
  const float* dG;
  const float* Mst;                 // stored left partials
  long long ioff[T3F_MAX_D + 1];
  float* dA;                        // packed like A (F32), nullable
  float* dB;                        // packed like B (F32), nullable
};

template <typename Tt>
__global__ void __launch_bounds__(256) k_gram_bwd(const __grid_constant__ GramBwdArgs a) {
  extern __shared__ float sm[];
  const TTV& A = a.A;
  const TTV& B = a.B;
  const int TA = a.TA, TB = a.TB, RA = a.RA, RB = a.RB, P = TA * TB, PS = RA * RB;
  float* As = sm;
  float* Bs = As + TA * RA * RA;
  float* Rc = Bs + TB * RB * RB;
  float* Rn = Rc + P * PS;
  float* X = Rn + P * PS;
  float* Y = X + P * PS;
  float* Mk = Y + P * PS;
  float* gs = Mk + P * PS;  // g_ab for the tile
  const Tt* Ap = static_cast<const Tt*>(A.p);
  const Tt* Bp = static_cast<const Tt*>(B.p);
  const int bA = A.batch, bB = B.batch;
  const int ntb = (bB + TB - 1) / TB;
  const int a0 = (blockIdx.x / ntb) * TA, b0 = (blockIdx.x % ntb) * TB;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int d = A.d;

  for (int p = tid; p < P; p += nth) {
    const int ta = p / TB, tb = p % TB;
    const bool ok = a0 + ta < bA && b0 + tb < bB;
    gs[p] = ok ? a.dG[(long long)(a0 + ta) * bB + (b0 + tb)] : 0.0f;
    Rc[p * PS] = 1.0f;
  }
  __syncthreads();

  for (int k = d - 1; k >= 0; --k) {
    const int rA0 = A.r[k], rA1 = A.r[k + 1], rB0 = B.r[k], rB1 = B.r[k + 1];
    const int nk = A.n[k];
    for (int e = tid; e < P * rA0 * rB0; e += nth) {
      const int p = e / (rA0 * rB0), q = e % (rA0 * rB0);
      const int ta = p / TB, tb = p % TB;
      const bool ok = a0 + ta < bA && b0 + tb < bB;
      const long long pid = (long long)(a0 + ta) * bB + (b0 + tb);
      Mk[p * PS + q] = ok ? a.Mst[a.ioff[k] + pid * rA0 * rB0 + q] : 0.0f;
      Rn[p * PS + q] = 0.0f;
    }
    for (int i = 0; i < nk; ++i) {
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
      // X[p] = A_i (rA0 x rA1) R (rA1 x rB1);  Y[p] = B_i (rB0 x rB1) R^T (rB1 x rA1)
      for (int e = tid; e < P * rA0 * rB1; e += nth) {
        const int p = e / (rA0 * rB1), q = e % (rA0 * rB1);
        const int al = q / rB1, bp = q % rB1;
        const float* Asl = As + (p / TB) * RA * RA + al * rA1;
        const float* R = Rc + p * PS + bp;
        float acc = 0.0f;
        for (int ap = 0; ap < rA1; ++ap) acc = fmaf(Asl[ap], R[ap * rB1], acc);
        X[p * PS + q] = acc;
      }
      for (int e = tid; e < P * rB0 * rA1; e += nth) {
        const int p = e / (rB0 * rA1), q = e % (rB0 * rA1);
        const int be = q / rA1, ap = q % rA1;
        const float* Bsl = Bs + (p % TB) * RB * RB + be * rB1;
        const float* R = Rc + p * PS + ap * rB1;
        float acc = 0.0f;
        for (int bp = 0; bp < rB1; ++bp) acc = fmaf(Bsl[bp], R[bp], acc);
        Y[p * PS + q] = acc;
      }
      __syncthreads();
      // R_next += X B_i^T
      for (int e = tid; e < P * rA0 * rB0; e += nth) {
        const int p = e / (rA0 * rB0), q = e % (rA0 * rB0);
        const int al = q / rB0, be = q % rB0;
        const float* x = X + p * PS + al * rB1;
        const float* Bsl = Bs + (p % TB) * RB * RB + be * rB1;
        float acc = 0.0f;
        for (int bp = 0; bp < rB1; ++bp) acc = fmaf(x[bp], Bsl[bp], acc);
        Rn[p * PS + q] += acc;
      }
      if (a.dA) {
        // dA_a[:, i, :] += sum_b g_ab M_k (rA0 x rB0) Y (rB0 x rA1)
        for (int e = tid; e < TA * rA0 * rA1; e += nth) {
          const int ta = e / (rA0 * rA1), q = e % (rA0 * rA1);
          const int al = q / rA1, ap = q % rA1;
          if (a0 + ta >= bA) continue;
          float acc = 0.0f;
          for (int tb = 0; tb < TB; ++tb) {
            const int p = ta * TB + tb;
            const float g = gs[p];
            if (g == 0.0f) continue;
            const float* M = Mk + p * PS + al * rB0;
            const float* y = Y + p * PS + ap;
            float s = 0.0f;
            for (int be = 0; be < rB0; ++be) s = fmaf(M[be], y[be * rA1], s);
            acc = fmaf(g, s, acc);
          }
          atomicAdd(a.dA + core_base(A, k, a0 + ta) + ((long long)al * nk + i) * rA1 + ap, acc);
        }
      }
      if (a.dB) {
        // dB_b[:, i, :] += sum_a g_ab M_k^T (rB0 x rA0) X (rA0 x rB1)
        for (int e = tid; e < TB * rB0 * rB1; e += nth) {
          const int tb = e / (rB0 * rB1), q = e % (rB0 * rB1);
          const int be = q / rB1, bp = q % rB1;
          if (b0 + tb >= bB) continue;
          float acc = 0.0f;
          for (int ta = 0; ta < TA; ++ta) {
            const int p = ta * TB + tb;
            const float g = gs[p];
            if (g == 0.0f) continue;
            const float* M = Mk + p * PS + be;
            const float* x = X + p * PS + bp;
            float s = 0.0f;
            for (int al = 0; al < rA0; ++al) s = fmaf(M[al * rB0], x[al * rB1], s);
            acc = fmaf(g, s, acc);
          }
          atomicAdd(a.dB + core_base(B, k, b0 + tb) + ((long long)be * nk + i) * rB1 + bp, acc);
        }
      }
      __syncthreads();
    }
    float* t = Rc;
    Rc = Rn;
    Rn = t;
    __syncthreads();
  }
}

static size_t gram_bwd_smem(int TA, int TB, int RA, int RB) {
  const size_t P = (size_t)TA * TB;
  return sizeof(float) * ((size_t)TA * RA * RA + (size_t)TB * RB * RB + 5 * P * RA * RB + P);
}

static void plan_gram_bwd(const TTV& A, const TTV& B, int* TA, int* TB, size_t* smem) {
  static const int cand[] = {8, 4, 2, 1};
  *TA = 1;
  *TB = 1;
  *smem = gram_bwd_smem(1, 1, A.rmax, B.rmax);
  long long best = -1;
  for (int ta : cand)
    for (int tb : cand) {
      if ((ta > 1 && ta / 2 >= A.batch) || (tb > 1 && tb / 2 >= B.batch)) continue;
      const size_t sm = gram_bwd_smem(ta, tb, A.rmax, B.rmax);
      if (sm > 100 * 1024) continue;
      const long long nt = (long long)((A.batch + ta - 1) / ta) * ((B.batch + tb - 1) / tb);
      const long long score = (nt >= 304 ? (1LL << 40) : nt << 20) + ta * tb;
      if (score > best) {
        best = score;
        *TA = ta;
        *TB = tb;
        *smem = sm;
      }
    }
}

static size_t ws_gram_bwd_generic(const TTV& A, const TTV& B) {
  long long ioff[T3F_MAX_D + 1];
  const long long n = partial_offsets(A, B, (long long)A.batch * B.batch, ioff);
  return kWsHeader + align256(sizeof(float) * n);
}

size_t ws_gram_bwd(const TTV& A, const TTV& B) {
  return gram_tile_bwd_supported(A, B) ? ws_gram_tile_bwd(A, B) : ws_gram_bwd_generic(A, B);
}

size_t ws_norm(const TTV& A) { return kWsHeader + align256(sizeof(float) * A.batch); }

__global__ void k_sqrt64(const float* in, double* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = sqrt(fmax((double)in[i], 0.0));
}

// Adds the cotangents of sum_ab dG[a,b] <A_a, B_b> to dA and dB (either may be NULL):
// left partials of every pair are recomputed into the workspace, then the right sweep
// scatters with atomics.
t3f_status gram_bwd_accumulate(const TTV& va, const TTV& vb, const float* dG, float* dA, float* dB, void* ws,
                               size_t ws_bytes, cudaStream_t s) {
  T3F_CHECK(check_ws(ws, ws_bytes, ws_gram_bwd_generic(va, vb)));
  GramBwdArgs args;
  memset(&args, 0, sizeof(args));
  args.dA = dA;
  args.dB = dB;
  if (!dA && !dB) return T3F_OK;
  float* Mst = reinterpret_cast<float*>(static_cast<char*>(ws) + kWsHeader);
  partial_offsets(va, vb, (long long)va.batch * vb.batch, args.ioff);
  T3F_CHECK(run_pair_sweep(va, vb, 0, nullptr, Mst, args.ioff, s));
  args.A = va;
  args.B = vb;
  args.RA = va.rmax;
  args.RB = vb.rmax;
  args.dG = dG;
  args.Mst = Mst;
  size_t smem;
  plan_gram_bwd(va, vb, &args.TA, &args.TB, &smem);
  const long long grid = (long long)((va.batch + args.TA - 1) / args.TA) * ((vb.batch + args.TB - 1) / args.TB);
  if (va.dtype == T3F_F32) {
    auto kern = k_gram_bwd<float>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return T3F_ERR_CUDA;
    kern<<<(unsigned)grid, 256, smem, s>>>(args);
  } else {
    auto kern = k_gram_bwd<__nv_bfloat16>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return T3F_ERR_CUDA;
    kern<<<(unsigned)grid, 256, smem, s>>>(args);
  }
  return launch_status();
}

}  // namespace t3f

using namespace t3f;

extern "C" t3f_status t3f_gram(const t3f_tt* A, const t3f_tt* B, float* G, int32_t math,
                               void* ws, size_t ws_bytes, t3f_stream_t stream) {
  TTV va, vb;
  T3F_CHECK(gram_views(A, B, &va, &vb));
  if (!G) return T3F_ERR_ARG;
  if (math != T3F_MATH_FP32 && math != T3F_MATH_TF32 && math != T3F_MATH_BF16) return T3F_ERR_ARG;
  if (math != T3F_MATH_FP32) {
    if (!gram_mma_supported(va, vb, math)) return T3F_ERR_UNSUPPORTED;
    int* err = (ws && ws_bytes >= kWsHeader) ? static_cast<int*>(ws) : nullptr;
    if (err && cudaMemsetAsync(err, 0, sizeof(int), (cudaStream_t)stream) != cudaSuccess) return T3F_ERR_CUDA;
    return run_gram_mma(va, vb, G, math, err, (cudaStream_t)stream);
  }
  if (gram_tile_supported(va, vb)) return run_gram_tile(va, vb, G, (cudaStream_t)stream);
  return run_pair_sweep(va, vb, 0, G, nullptr, nullptr, (cudaStream_t)stream);
}

extern "C" t3f_status t3f_norm(const t3f_tt* A, double* out, void* ws, size_t ws_bytes,
                               t3f_stream_t stream) {
  TTV va;
  T3F_CHECK(make_view(A, &va, -1, false));
  if (va.dtype == T3F_F64) return T3F_ERR_DTYPE;
  if (va.rmax > T3F_MAX_RANK) return T3F_ERR_UNSUPPORTED;
  if (!out) return T3F_ERR_ARG;
  T3F_CHECK(check_ws(ws, ws_bytes, ws_norm(va)));
  if (va.batch == 0) return T3F_OK;
  float* sq = reinterpret_cast<float*>(static_cast<char*>(ws) + kWsHeader);
  cudaStream_t s = (cudaStream_t)stream;
  T3F_CHECK(run_self_sweep(va, sq, s));
  k_sqrt64<<<(va.batch + 255) / 256, 256, 0, s>>>(sq, out, va.batch);
  return launch_status();
}

extern "C" t3f_status t3f_gram_backward(const t3f_tt* A, const t3f_tt* B, const float* dG,
                                        t3f_tt* dA, t3f_tt* dB, int32_t math, void* ws, size_t ws_bytes,
                                        t3f_stream_t stream) {
  TTV va, vb, vda, vdb;
  T3F_CHECK(gram_views(A, B, &va, &vb));
  if (!dG) return T3F_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  GramBwdArgs args;
  memset(&args, 0, sizeof(args));
  if (dA) {
    T3F_CHECK(make_view(dA, &vda, T3F_F32, false));
    if (vda.batch != va.batch || vda.d != va.d) return T3F_ERR_SHAPE;
    for (int k = 0; k <= va.d; ++k)
      if (vda.r[k] != va.r[k] || (k < va.d && vda.n[k] != va.n[k])) return T3F_ERR_SHAPE;
    args.dA = static_cast<float*>(vda.p);
  }
  if (dB) {
    T3F_CHECK(make_view(dB, &vdb, T3F_F32, false));
    if (vdb.batch != vb.batch || vdb.d != vb.d) return T3F_ERR_SHAPE;
    for (int k = 0; k <= vb.d; ++k)
      if (vdb.r[k] != vb.r[k] || (k < vb.d && vdb.n[k] != vb.n[k])) return T3F_ERR_SHAPE;
    args.dB = static_cast<float*>(vdb.p);
  }
  if (math != T3F_MATH_FP32 && math != T3F_MATH_TF32 && math != T3F_MATH_BF16) return T3F_ERR_ARG;
  if (math != T3F_MATH_FP32) {
    if (!gram_mma_supported(va, vb, math)) return T3F_ERR_UNSUPPORTED;
    T3F_CHECK(check_ws(ws, ws_bytes, ws_gram_bwd_tc(va, vb)));
    int* err = static_cast<int*>(ws);
    if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) return T3F_ERR_CUDA;
    return run_gram_tc_backward(va, vb, dG, args.dA, args.dB, math, static_cast<char*>(ws) + kWsHeader, err, s);
  }
  T3F_CHECK(check_ws(ws, ws_bytes, ws_gram_bwd(va, vb)));
  if (args.dA && cudaMemsetAsync(args.dA, 0, sizeof(float) * t3f_packed_size(dA), s) != cudaSuccess)
    return T3F_ERR_CUDA;
  if (args.dB && cudaMemsetAsync(args.dB, 0, sizeof(float) * t3f_packed_size(dB), s) != cudaSuccess)
    return T3F_ERR_CUDA;
  if (!args.dA && !args.dB) return T3F_OK;
  if (gram_tile_bwd_supported(va, vb)) return run_gram_tile_bwd(va, vb, dG, args.dA, args.dB, ws, ws_bytes, s);
  return gram_bwd_accumulate(va, vb, dG, args.dA, args.dB, ws, ws_bytes, s);
}

