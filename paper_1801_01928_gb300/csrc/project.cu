// Riemannian tangent-space projection (paper Section 3.2): project_sum and its adjoint.
//
// X is given by its orthogonal forms U (left-orthogonal U_1..U_{d-1}) and V
// (right-orthogonal V_2..V_d). For a batch Z_j with weights c_j:
//   L^{(j)} = left partials of (U, Z_j),  R^{(j)} = right partials of (V, Z_j)   (sweep.cu)
//   Zhat_k[:, i, :] = sum_j c_j L^{(j)}_k Z_j^k[:, i, :] (R^{(j)}_{k+1})^T        (assembly)
//   dU_k = (I - U_k U_k^T) Zhat_k (k < d), dU_d = Zhat_d                          (gauge)
// Interfaces are numbered 0..d; core k sits between interfaces k and k+1.
//
// Adjoint of phi = sum_k <dUbar_k, dU_k> (X fixed), with W = gauge projection of dUbar:
//   P_0 = 0, P_{k+1} = sum_i V_k^T P_k Z_k + W_k^T L_k Z_k                (mixed left sweep)
//   Q_d = 0, Q_k = sum_i (U_k Q_{k+1} + W_k R_{k+1}) Z_k^T                (mixed right sweep)
//   dZ_j^k[:, i, :] = c_j (P_k^T V_k R_{k+1} + L_k^T W_k R_{k+1} + L_k^T U_k Q_{k+1})
//   dc_j = P_d
#include <algorithm>

#include "t3f_internal.cuh"

namespace t3f {

// ---------------------------------------------------------------------------------------
// Gauge projection: out_k = Z_k - U_k (U_k^T Z_k) on the (r_{k-1} n_k) x r_k unfoldings.
// One CTA per core: staged in shared memory (gauge_core_staged) when the largest core fits,
// else both steps read global memory.
// ---------------------------------------------------------------------------------------
struct GaugeArgs {
  TTV U;
  const float* Z;   // compact, U's shape
  float* out;       // compact, U's shape
  int staged;       // U_k and Z_k fit in shared memory
};

__global__ void __launch_bounds__(256) k_gauge(const __grid_constant__ GaugeArgs a) {
  extern __shared__ __align__(16) float sm[];
  const int k = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
  const TTV& U = a.U;
  const int r0 = U.r[k], n = U.n[k], r1 = U.r[k + 1];
  const int m = r0 * n;
  const float* Uk = static_cast<const float*>(U.p) + U.off[k];
  const float* Zk = a.Z + U.off[k];
  float* Ok = a.out + U.off[k];
  if (k == U.d - 1) {
    for (int e = tid; e < m * r1; e += nth) Ok[e] = Zk[e];
    return;
  }
  if (a.staged) {
    gauge_core_staged(Uk, Zk, Ok, m, r1, sm);
    return;
  }
  float* G = sm;  // r1 x r1: G = U^T Z
  for (int e = tid; e < r1 * r1; e += nth) {
    const int a1 = e / r1, b1 = e % r1;
    float s = 0.0f;
    for (int q = 0; q < m; ++q) s = fmaf(__ldg(Uk + q * r1 + a1), Zk[q * r1 + b1], s);
    G[e] = s;
  }
  __syncthreads();
  for (int e = tid; e < m * r1; e += nth) {
    const int q = e / r1, b1 = e % r1;
    float s = Zk[e];
    for (int a1 = 0; a1 < r1; ++a1) s = fmaf(-__ldg(Uk + q * r1 + a1), G[a1 * r1 + b1], s);
    Ok[e] = s;
  }
}

t3f_status run_gauge_project(const TTV& U, const float* Z, float* out, cudaStream_t s) {
  GaugeArgs a;
  a.U = U;
  a.Z = Z;
  a.out = out;
  long long full = 0;
  for (int k = 0; k + 1 < U.d; ++k) full = std::max(full, gauge_staged_floats(U.r[k] * U.n[k], U.r[k + 1]));
  const size_t base = sizeof(float) * U.rmax * U.rmax;
  a.staged = sizeof(float) * (size_t)full <= 200 * 1024 ? 1 : 0;
  const size_t smem = a.staged ? std::max(sizeof(float) * (size_t)full, base) : base;
  if (cudaFuncSetAttribute(k_gauge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return T3F_ERR_CUDA;
  k_gauge<<<U.d, 256, smem, s>>>(a);
  return launch_status();
}

// ---------------------------------------------------------------------------------------
// Assembly: one CTA per (core k, slice i, chunk of j), partial sums into the workspace.
// ---------------------------------------------------------------------------------------
struct AssembleArgs {
  TTV U, Z;
  const float* L;                 // left partials, pair = j
  const float* R;                 // right partials
  long long ioffL[T3F_MAX_D + 1];
  long long ioffR[T3F_MAX_D + 1];
  const float* c;
  int jchunk, nchunks;
  float* part;                    // [nchunks][compact U-shaped]
  long long gsize;
  int RU, RZ;                     // max ranks
};

__global__ void __launch_bounds__(256) k_psum_assemble(const __grid_constant__ AssembleArgs a) {
  extern __shared__ float sm[];
  const TTV& U = a.U;
  const TTV& Z = a.Z;
  const int d = U.d;
  int bid = blockIdx.x;
  const int chunk = bid % a.nchunks;
  bid /= a.nchunks;
  // locate (k, i)
  int k = 0, i = bid;
  while (k < d && i >= U.n[k]) {
    i -= U.n[k];
    ++k;
  }
  const int r0 = U.r[k], r1 = U.r[k + 1], s0 = Z.r[k], s1 = Z.r[k + 1], n = U.n[k];
  float* Ls = sm;                       // r0 x s0
  float* Zs = Ls + a.RU * a.RZ;         // s0 x s1
  float* Rs = Zs + a.RZ * a.RZ;         // r1 x s1
  float* Ys = Rs + a.RU * a.RZ;         // r0 x s1
  float* acc = Ys + a.RU * a.RZ;        // r0 x r1
  for (int e = threadIdx.x; e < r0 * r1; e += blockDim.x) acc[e] = 0.0f;
  const int j0 = chunk * a.jchunk;
  const int j1 = min(Z.batch, j0 + a.jchunk);
  const float* Zp = static_cast<const float*>(Z.p);
  for (int j = j0; j < j1; ++j) {
    __syncthreads();
    const float cj = a.c[j];
    for (int e = threadIdx.x; e < r0 * s0; e += blockDim.x)
      Ls[e] = a.L[a.ioffL[k] + (long long)j * r0 * s0 + e];
    for (int e = threadIdx.x; e < s0 * s1; e += blockDim.x) {
      const int g = e / s1, h = e % s1;
      Zs[e] = __ldg(Zp + core_base(Z, k, j) + ((long long)g * n + i) * s1 + h);
    }
    for (int e = threadIdx.x; e < r1 * s1; e += blockDim.x)
      Rs[e] = a.R[a.ioffR[k + 1] + (long long)j * r1 * s1 + e];
    __syncthreads();
    for (int e = threadIdx.x; e < r0 * s1; e += blockDim.x) {
      const int al = e / s1, h = e % s1;
      float s = 0.0f;
      for (int g = 0; g < s0; ++g) s = fmaf(Ls[al * s0 + g], Zs[g * s1 + h], s);
      Ys[e] = cj * s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < r0 * r1; e += blockDim.x) {
      const int al = e / r1, be = e % r1;
      float s = acc[e];
      for (int h = 0; h < s1; ++h) s = fmaf(Ys[al * s1 + h], Rs[be * s1 + h], s);
      acc[e] = s;
    }
  }
  __syncthreads();
  float* out = a.part + (long long)chunk * a.gsize + U.off[k];
  for (int e = threadIdx.x; e < r0 * r1; e += blockDim.x) {
    const int al = e / r1, be = e % r1;
    out[((long long)al * n + i) * r1 + be] = acc[e];
  }
}

// ---------------------------------------------------------------------------------------
// Mixed sweeps of the adjoint. One CTA per tile of TB objects of Z (A side is batch 1).
//   dir 0: Next = sum_i A1_i^T Cur B_i + A2_i^T Aux_k B_i      (Cur_0 = 0; stores 0..d)
//   dir 1: Next = sum_i (A1_i Cur + A2_i Aux_{k+1}) B_i^T       (Cur_d = 0; stores d..0)
// ---------------------------------------------------------------------------------------
struct MixedArgs {
  TTV A1, A2, B;
  const float* aux;
  long long ioff[T3F_MAX_D + 1];  // same interface layout for aux and the store
  float* store;
  int TB, RA, RB, dir;
};

__global__ void __launch_bounds__(256) k_mixed_sweep(const __grid_constant__ MixedArgs a) {
  extern __shared__ float sm[];
  const TTV& B = a.B;
  const int TB = a.TB, RA = a.RA, RB = a.RB, PS = RA * RB, d = B.d;
  float* A1s = sm;                 // RA*RA
  float* A2s = A1s + RA * RA;      // RA*RA
  float* Bs = A2s + RA * RA;       // TB * RB*RB
  float* Cur = Bs + TB * RB * RB;  // TB * PS
  float* Nx = Cur + TB * PS;
  float* Ax = Nx + TB * PS;
  float* T1 = Ax + TB * PS;
  float* T2 = T1 + TB * PS;
  const int b0 = blockIdx.x * TB;
  const int tid = threadIdx.x, nth = blockDim.x;
  const float* A1p = static_cast<const float*>(a.A1.p);
  const float* A2p = static_cast<const float*>(a.A2.p);
  const float* Bp = static_cast<const float*>(B.p);
  for (int p = tid; p < TB; p += nth) Cur[p * PS] = 0.0f;
  __syncthreads();
  {
    const int j = a.dir == 0 ? 0 : d;
    for (int p = tid; p < TB; p += nth)
      if (b0 + p < B.batch) a.store[a.ioff[j] + (b0 + p)] = 0.0f;
  }
  for (int s = 0; s < d; ++s) {
    const int k = a.dir == 0 ? s : d - 1 - s;
    const int rA0 = a.A1.r[k], rA1 = a.A1.r[k + 1], rB0 = B.r[k], rB1 = B.r[k + 1], nk = B.n[k];
    const int nr = a.dir == 0 ? rA1 : rA0, nc = a.dir == 0 ? rB1 : rB0;
    const int ja = a.dir == 0 ? k : k + 1;       // aux interface
    const int ar = a.dir == 0 ? rA0 : rA1, ac = a.dir == 0 ? rB0 : rB1;
    for (int e = tid; e < TB * nr * nc; e += nth) Nx[(e / (nr * nc)) * PS + e % (nr * nc)] = 0.0f;
    for (int e = tid; e < TB * ar * ac; e += nth) {
      const int p = e / (ar * ac), q = e % (ar * ac);
      Ax[p * PS + q] = b0 + p < B.batch ? a.aux[a.ioff[ja] + (long long)(b0 + p) * ar * ac + q] : 0.0f;
    }
    for (int i = 0; i < nk; ++i) {
      for (int e = tid; e < rA0 * rA1; e += nth) {
        const int al = e / rA1, be = e % rA1;
        A1s[e] = __ldg(A1p + a.A1.off[k] + ((long long)al * nk + i) * rA1 + be);
        A2s[e] = __ldg(A2p + a.A2.off[k] + ((long long)al * nk + i) * rA1 + be);
      }
      for (int e = tid; e < TB * rB0 * rB1; e += nth) {
        const int t = e / (rB0 * rB1), q = e % (rB0 * rB1);
        const int al = q / rB1, be = q % rB1;
        Bs[t * RB * RB + q] = b0 + t < B.batch
                                  ? __ldg(Bp + core_base(B, k, b0 + t) + ((long long)al * nk + i) * rB1 + be)
                                  : 0.0f;
      }
      __syncthreads();
      if (a.dir == 0) {
        // T1 = Cur B_i, T2 = Aux B_i   (rA0 x rB1)
        for (int e = tid; e < TB * rA0 * rB1; e += nth) {
          const int p = e / (rA0 * rB1), q = e % (rA0 * rB1);
          const int al = q / rB1, bp = q % rB1;
          const float* c = Cur + p * PS + al * rB0;
          const float* x = Ax + p * PS + al * rB0;
          const float* bs = Bs + p * RB * RB + bp;
          float s1 = 0.0f, s2 = 0.0f;
          for (int be = 0; be < rB0; ++be) {
            s1 = fmaf(c[be], bs[be * rB1], s1);
            s2 = fmaf(x[be], bs[be * rB1], s2);
          }
          T1[p * PS + q] = s1;
          T2[p * PS + q] = s2;
        }
        __syncthreads();
        for (int e = tid; e < TB * rA1 * rB1; e += nth) {
          const int p = e / (rA1 * rB1), q = e % (rA1 * rB1);
          const int ap = q / rB1, bp = q % rB1;
          float s = 0.0f;
          for (int al = 0; al < rA0; ++al)
            s += A1s[al * rA1 + ap] * T1[p * PS + al * rB1 + bp] + A2s[al * rA1 + ap] * T2[p * PS + al * rB1 + bp];
          Nx[p * PS + q] += s;
        }
      } else {
        // T1 = A1_i Cur + A2_i Aux  (rA0 x rB1)
        for (int e = tid; e < TB * rA0 * rB1; e += nth) {
          const int p = e / (rA0 * rB1), q = e % (rA0 * rB1);
          const int al = q / rB1, bp = q % rB1;
          float s = 0.0f;
          for (int ap = 0; ap < rA1; ++ap)
            s += A1s[al * rA1 + ap] * Cur[p * PS + ap * rB1 + bp] + A2s[al * rA1 + ap] * Ax[p * PS + ap * rB1 + bp];
          T1[p * PS + q] = s;
        }
        __syncthreads();
        for (int e = tid; e < TB * rA0 * rB0; e += nth) {
          const int p = e / (rA0 * rB0), q = e % (rA0 * rB0);
          const int al = q / rB0, be = q % rB0;
          float s = 0.0f;
          for (int bp = 0; bp < rB1; ++bp) s = fmaf(T1[p * PS + al * rB1 + bp], Bs[p * RB * RB + be * rB1 + bp], s);
          Nx[p * PS + q] += s;
        }
      }
      __syncthreads();
    }
    float* t = Cur;
    Cur = Nx;
    Nx = t;
    const int j = a.dir == 0 ? k + 1 : k;
    for (int e = tid; e < TB * nr * nc; e += nth) {
      const int p = e / (nr * nc), q = e % (nr * nc);
      if (b0 + p < B.batch) a.store[a.ioff[j] + (long long)(b0 + p) * nr * nc + q] = Cur[p * PS + q];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Core gradients of the adjoint: one CTA per (object j, core k).
// ---------------------------------------------------------------------------------------
struct PGradArgs {
  TTV U, V, W, Z;
  const float *L, *R, *P, *Q;
  long long ioff[T3F_MAX_D + 1];
  const float* c;
  float* dZ;   // packed like Z, nullable
  float* dc;   // nullable
  int RU, RZ;
};

__global__ void __launch_bounds__(256) k_psum_grad(const __grid_constant__ PGradArgs a) {
  extern __shared__ float sm[];
  const int d = a.Z.d;
  const int j = blockIdx.x / d, k = blockIdx.x % d;
  const int r0 = a.U.r[k], r1 = a.U.r[k + 1], s0 = a.Z.r[k], s1 = a.Z.r[k + 1], n = a.Z.n[k];
  const int PS = a.RU * a.RZ;
  float* Ps = sm;          // r0 x s0
  float* Ls = Ps + PS;     // r0 x s0
  float* Rs = Ls + PS;     // r1 x s1
  float* Qs = Rs + PS;     // r1 x s1
  float* Y1 = Qs + PS;     // s0 x r1 : P^T V_i + L^T W_i
  float* Y2 = Y1 + PS;     // s0 x r1 : L^T U_i
  const float cj = a.c[j];
  for (int e = threadIdx.x; e < r0 * s0; e += blockDim.x) {
    Ps[e] = a.P[a.ioff[k] + (long long)j * r0 * s0 + e];
    Ls[e] = a.L[a.ioff[k] + (long long)j * r0 * s0 + e];
  }
  for (int e = threadIdx.x; e < r1 * s1; e += blockDim.x) {
    Rs[e] = a.R[a.ioff[k + 1] + (long long)j * r1 * s1 + e];
    Qs[e] = a.Q[a.ioff[k + 1] + (long long)j * r1 * s1 + e];
  }
  if (k == d - 1 && a.dc && threadIdx.x == 0) a.dc[j] = a.P[a.ioff[d] + j];
  if (!a.dZ) return;
  const float* Up = static_cast<const float*>(a.U.p) + a.U.off[k];
  const float* Vp = static_cast<const float*>(a.V.p) + a.V.off[k];
  const float* Wp = static_cast<const float*>(a.W.p) + a.W.off[k];
  float* out = a.dZ + core_base(a.Z, k, j);
  for (int i = 0; i < n; ++i) {
    __syncthreads();
    for (int e = threadIdx.x; e < s0 * r1; e += blockDim.x) {
      const int g = e / r1, be = e % r1;
      float y1 = 0.0f, y2 = 0.0f;
      for (int al = 0; al < r0; ++al) {
        const long long o = ((long long)al * n + i) * r1 + be;
        y1 += Ps[al * s0 + g] * __ldg(Vp + o) + Ls[al * s0 + g] * __ldg(Wp + o);
        y2 += Ls[al * s0 + g] * __ldg(Up + o);
      }
      Y1[e] = y1;
      Y2[e] = y2;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < s0 * s1; e += blockDim.x) {
      const int g = e / s1, h = e % s1;
      float s = 0.0f;
      for (int be = 0; be < r1; ++be) s += Y1[g * r1 + be] * Rs[be * s1 + h] + Y2[g * r1 + be] * Qs[be * s1 + h];
      out[((long long)g * n + i) * s1 + h] = cj * s;
    }
  }
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------

static t3f_status psum_views(const t3f_tt* U, const t3f_tt* V, const t3f_tt* Z, TTV* vu, TTV* vv,
                             TTV* vz) {
  T3F_CHECK(make_view(U, vu, T3F_F32, false));
  T3F_CHECK(make_view(V, vv, T3F_F32, false));
  T3F_CHECK(make_view(Z, vz, T3F_F32, false));
  if (vu->batch != 1 || vv->batch != 1) return T3F_ERR_SHAPE;
  if (vu->d != vv->d || vu->d != vz->d) return T3F_ERR_SHAPE;
  for (int k = 0; k <= vu->d; ++k) {
    if (vu->r[k] != vv->r[k]) return T3F_ERR_SHAPE;
    if (k < vu->d && (vu->n[k] != vv->n[k] || vu->n[k] != vz->n[k])) return T3F_ERR_SHAPE;
  }
  if (vu->rmax > T3F_MAX_RANK || vz->rmax > T3F_MAX_RANK) return T3F_ERR_UNSUPPORTED;
  return T3F_OK;
}

static t3f_status check_like(const t3f_tt* t, const TTV& ref, TTV* v) {
  T3F_CHECK(make_view(t, v, T3F_F32, false));
  if (v->batch != ref.batch || v->d != ref.d) return T3F_ERR_SHAPE;
  for (int k = 0; k <= ref.d; ++k)
    if (v->r[k] != ref.r[k] || (k < ref.d && v->n[k] != ref.n[k])) return T3F_ERR_SHAPE;
  return T3F_OK;
}

struct PsumLayout {
  long long ioffL[T3F_MAX_D + 1], ioffR[T3F_MAX_D + 1];
  size_t offL, offR, offP, offQ, offW, offPart, offImg, offXT, total;
  int jchunk, nchunks;
  long long gsize;
};

static PsumLayout psum_layout(const TTV& U, const TTV& Z, bool bwd) {
  PsumLayout l;
  l.offImg = 0;
  l.offXT = 0;
  const long long nL = partial_offsets(U, Z, Z.batch, l.ioffL);
  for (int j = 0; j <= U.d; ++j) l.ioffR[j] = l.ioffL[j];
  l.gsize = 0;
  for (int k = 0; k < U.d; ++k) l.gsize += U.osz[k];
  size_t o = kWsHeader;
  l.offL = o;
  o += align256(sizeof(float) * nL);
  l.offR = o;
  o += align256(sizeof(float) * nL);
  if (bwd) {
    l.offP = o;
    o += align256(sizeof(float) * nL);
    l.offQ = o;
    o += align256(sizeof(float) * nL);
    l.offW = o;
    o += align256(sizeof(float) * l.gsize);
    if (psweep_supported(U, Z)) {  // transposed V, U, W for the right sweep and the gradients
      l.offXT = o;
      o += align256(sizeof(float) * 3 * xtranspose_offsets(U, nullptr));
    }
    l.jchunk = 0;
    l.nchunks = 0;
    l.offPart = 0;
  } else if (psweep_supported(U, Z)) {
    l.nchunks = passemble_ranges(Z);
    l.jchunk = (Z.batch + l.nchunks - 1) / l.nchunks;
    l.offPart = o;
    o += align256(sizeof(float) * l.gsize * l.nchunks);
    l.offP = l.offQ = l.offW = 0;
    l.offXT = o;  // transposed V for the right sweep
    o += align256(sizeof(float) * xtranspose_offsets(U, nullptr));
    if (psweep_tc_supported(U, Z)) {  // operand images of the TF32 sweeps
      l.offImg = o;
      o += align256(psweep_tc_img_bytes(U));
    }
  } else {
    // split the batch so that (sum_k n_k) * nchunks CTAs cover the GPU a few times
    long long slices = 0;
    for (int k = 0; k < U.d; ++k) slices += U.n[k];
    int nch = (int)((152LL * 8 + slices - 1) / slices);
    if (nch > Z.batch) nch = Z.batch;
    if (nch < 1) nch = 1;
    l.jchunk = (Z.batch + nch - 1) / nch;
    l.nchunks = (Z.batch + l.jchunk - 1) / l.jchunk;
    l.offPart = o;
    o += align256(sizeof(float) * l.gsize * l.nchunks);
    l.offP = l.offQ = l.offW = 0;
  }
  l.total = o;
  return l;
}

size_t ws_psum(const TTV& U, const TTV& Z, bool bwd) { return psum_layout(U, Z, bwd).total; }

__global__ void k_reduce_chunks(const float* part, int nparts, long long size, float* out) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < size;
       e += (long long)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int p = 0; p < nparts; ++p) s += part[(long long)p * size + e];
    out[e] = s;
  }
}

}  // namespace t3f

using namespace t3f;

extern "C" t3f_status t3f_project_sum(const t3f_tt* U, const t3f_tt* V, const t3f_tt* Z,
                                      const float* c, t3f_tt* dU, int32_t math, void* ws,
                                      size_t ws_bytes, t3f_stream_t stream) {
  TTV vu, vv, vz, vd;
  T3F_CHECK(psum_views(U, V, Z, &vu, &vv, &vz));
  T3F_CHECK(check_like(dU, vu, &vd));
  if (!c) return T3F_ERR_ARG;
  if (math != T3F_MATH_FP32 && math != T3F_MATH_TF32 && math != T3F_MATH_BF16) return T3F_ERR_ARG;
  // TF32: the U- and V-side contractions of both sweeps on the tensor cores; BF16 has no
  // tensor-core form here
  if (math == T3F_MATH_BF16) return T3F_ERR_UNSUPPORTED;
  if (math == T3F_MATH_TF32 && (!psweep_tc_supported(vu, vz) || !psweep_supported(vu, vz))) return T3F_ERR_UNSUPPORTED;
  PsumLayout l = psum_layout(vu, vz, false);
  T3F_CHECK(check_ws(ws, ws_bytes, l.total));
  cudaStream_t s = (cudaStream_t)stream;
  char* w = static_cast<char*>(ws);
  float* Lst = reinterpret_cast<float*>(w + l.offL);
  float* Rst = reinterpret_cast<float*>(w + l.offR);
  float* part = reinterpret_cast<float*>(w + l.offPart);
  if (math == T3F_MATH_TF32) {
    int* err = static_cast<int*>(ws);
    if (cudaMemsetAsync(ws, 0, sizeof(int), s) != cudaSuccess) return T3F_ERR_CUDA;
    T3F_CHECK(run_psweep_tc(vu, vv, vz, Lst, l.ioffL, Rst, l.ioffR, w + l.offImg, err, s));
    T3F_CHECK(run_passemble(vu, vz, Lst, Rst, l.ioffL, c, part, l.nchunks, s));
    k_reduce_chunks<<<256, 256, 0, s>>>(part, l.nchunks, l.gsize, part);
    T3F_CHECK(launch_status());
    return run_gauge_project(vu, part, static_cast<float*>(vd.p), s);
  }
  if (psweep_supported(vu, vz)) {
    int* err = static_cast<int*>(ws);
    if (cudaMemsetAsync(ws, 0, sizeof(int), s) != cudaSuccess) return T3F_ERR_CUDA;
    T3F_CHECK(run_psweep(vu, vz, 0, static_cast<const float*>(vu.p), nullptr, nullptr, Lst, nullptr, l.ioffL, s, err));
    // the right sweep stages its slices from a transposed copy of V (16-byte copies)
    float* VT = reinterpret_cast<float*>(w + l.offXT);
    long long toff[T3F_MAX_D];
    xtranspose_offsets(vv, toff);
    const float* vsrc[1] = {static_cast<const float*>(vv.p)};
    T3F_CHECK(run_xtranspose(vv, vsrc, 1, VT, s));
    T3F_CHECK(run_psweep(vv, vz, 1, VT, nullptr, nullptr, Rst, nullptr, l.ioffR, s, err, toff));
    T3F_CHECK(run_passemble(vu, vz, Lst, Rst, l.ioffL, c, part, l.nchunks, s));
    k_reduce_chunks<<<256, 256, 0, s>>>(part, l.nchunks, l.gsize, part);
    T3F_CHECK(launch_status());
    return run_gauge_project(vu, part, static_cast<float*>(vd.p), s);
  }
  T3F_CHECK(run_pair_sweep(vu, vz, 0, nullptr, Lst, l.ioffL, s));
  T3F_CHECK(run_pair_sweep(vv, vz, 1, nullptr, Rst, l.ioffR, s));
  AssembleArgs a;
  a.U = vu;
  a.Z = vz;
  a.L = Lst;
  a.R = Rst;
  for (int j = 0; j <= T3F_MAX_D; ++j) {
    a.ioffL[j] = j <= vu.d ? l.ioffL[j] : 0;
    a.ioffR[j] = j <= vu.d ? l.ioffR[j] : 0;
  }
  a.c = c;
  a.jchunk = l.jchunk;
  a.nchunks = l.nchunks;
  a.part = part;
  a.gsize = l.gsize;
  a.RU = vu.rmax;
  a.RZ = vz.rmax;
  long long slices = 0;
  for (int k = 0; k < vu.d; ++k) slices += vu.n[k];
  const size_t smem = sizeof(float) * (3 * (size_t)a.RU * a.RZ + (size_t)a.RZ * a.RZ + (size_t)a.RU * a.RU);
  if (cudaFuncSetAttribute(k_psum_assemble, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return T3F_ERR_CUDA;
  k_psum_assemble<<<(unsigned)(slices * l.nchunks), 256, smem, s>>>(a);
  T3F_CHECK(launch_status());
  k_reduce_chunks<<<256, 256, 0, s>>>(part, l.nchunks, l.gsize, part);
  T3F_CHECK(launch_status());
  return run_gauge_project(vu, part, static_cast<float*>(vd.p), s);
}

extern "C" t3f_status t3f_project_sum_backward(const t3f_tt* U, const t3f_tt* V, const t3f_tt* Z,
                                               const float* c, const t3f_tt* dUbar, t3f_tt* dZ,
                                               float* dc, void* ws, size_t ws_bytes,
                                               t3f_stream_t stream) {
  TTV vu, vv, vz, vb, vdz;
  T3F_CHECK(psum_views(U, V, Z, &vu, &vv, &vz));
  T3F_CHECK(check_like(dUbar, vu, &vb));
  if (!c) return T3F_ERR_ARG;
  if (dZ) T3F_CHECK(check_like(dZ, vz, &vdz));
  if (!dZ && !dc) return T3F_OK;
  PsumLayout l = psum_layout(vu, vz, true);
  T3F_CHECK(check_ws(ws, ws_bytes, l.total));
  cudaStream_t s = (cudaStream_t)stream;
  char* w = static_cast<char*>(ws);
  float* Lst = reinterpret_cast<float*>(w + l.offL);
  float* Rst = reinterpret_cast<float*>(w + l.offR);
  float* Pst = reinterpret_cast<float*>(w + l.offP);
  float* Qst = reinterpret_cast<float*>(w + l.offQ);
  float* Wc = reinterpret_cast<float*>(w + l.offW);
  T3F_CHECK(run_gauge_project(vu, static_cast<const float*>(vb.p), Wc, s));
  TTV vw = vu;
  vw.p = Wc;
  if (psweep_supported(vu, vz)) {
    const float* Up = static_cast<const float*>(vu.p);
    const float* Vp = static_cast<const float*>(vv.p);
    int* err = static_cast<int*>(ws);
    if (cudaMemsetAsync(ws, 0, sizeof(int), s) != cudaSuccess) return T3F_ERR_CUDA;
    T3F_CHECK(run_psweep(vu, vz, 0, Up, Vp, Wc, Lst, Pst, l.ioffL, s, err));
    // the right sweep and the gradient kernel stage their slices from transposed copies of
    // V, U and W (16-byte copies)
    float* XT = reinterpret_cast<float*>(w + l.offXT);
    long long toff[T3F_MAX_D];
    const long long tsz = xtranspose_offsets(vu, toff);
    const float* srcs[3] = {Vp, Up, Wc};
    T3F_CHECK(run_xtranspose(vu, srcs, 3, XT, s));
    const float *VT = XT, *UT = XT + tsz, *WT = XT + 2 * tsz;
    T3F_CHECK(run_psweep(vu, vz, 1, VT, UT, WT, Rst, Qst, l.ioffL, s, err, toff));
    return run_pgrad(vu, vz, UT, VT, WT, Lst, Rst, Pst, Qst, l.ioffL, c, dZ ? static_cast<float*>(vdz.p) : nullptr,
                     dc, s, toff);
  }
  T3F_CHECK(run_pair_sweep(vu, vz, 0, nullptr, Lst, l.ioffL, s));
  T3F_CHECK(run_pair_sweep(vv, vz, 1, nullptr, Rst, l.ioffR, s));
  // mixed sweeps
  int TB = 8;
  auto msmem = [&](int tb) {
    return sizeof(float) * (2 * (size_t)vu.rmax * vu.rmax + (size_t)tb * vz.rmax * vz.rmax +
                            5 * (size_t)tb * vu.rmax * vz.rmax);
  };
  while (TB > 1 && (msmem(TB) > 100 * 1024 || (vz.batch + TB - 1) / TB < 304)) TB /= 2;
  MixedArgs m;
  memset(&m, 0, sizeof(m));
  m.B = vz;
  m.TB = TB;
  m.RA = vu.rmax;
  m.RB = vz.rmax;
  for (int j = 0; j <= vu.d; ++j) m.ioff[j] = l.ioffL[j];
  const size_t ms = msmem(TB);
  if (cudaFuncSetAttribute(k_mixed_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ms) != cudaSuccess)
    return T3F_ERR_CUDA;
  const unsigned mg = (unsigned)((vz.batch + TB - 1) / TB);
  m.A1 = vv;
  m.A2 = vw;
  m.aux = Lst;
  m.store = Pst;
  m.dir = 0;
  k_mixed_sweep<<<mg, 256, ms, s>>>(m);
  T3F_CHECK(launch_status());
  m.A1 = vu;
  m.A2 = vw;
  m.aux = Rst;
  m.store = Qst;
  m.dir = 1;
  k_mixed_sweep<<<mg, 256, ms, s>>>(m);
  T3F_CHECK(launch_status());
  PGradArgs g;
  memset(&g, 0, sizeof(g));
  g.U = vu;
  g.V = vv;
  g.W = vw;
  g.Z = vz;
  g.L = Lst;
  g.R = Rst;
  g.P = Pst;
  g.Q = Qst;
  for (int j = 0; j <= vu.d; ++j) g.ioff[j] = l.ioffL[j];
  g.c = c;
  g.dZ = dZ ? static_cast<float*>(vdz.p) : nullptr;
  g.dc = dc;
  g.RU = vu.rmax;
  g.RZ = vz.rmax;
  const size_t gs = sizeof(float) * 6 * (size_t)g.RU * g.RZ;
  if (cudaFuncSetAttribute(k_psum_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gs) != cudaSuccess)
    return T3F_ERR_CUDA;
  k_psum_grad<<<(unsigned)((long long)vz.batch * vz.d), 256, gs, s>>>(g);
  return launch_status();
}
