// TT rounding (paper Section 3, t3f.round: the best approximation of lower TT-rank), the
// TT-SVD recompression of Oseledets (2011) in FP64, one CTA per object:
//   1. right to left, k = d-1..1: Householder QR of the transposed unfolding
//      W_k^T = ((n_k r_k) x r_{k-1}) = Q R with diag(R) >= 0; W_k <- Q^T (right-orthogonal),
//      W_{k-1} <- W_{k-1} R^T;
//   2. left to right, k = 0..d-2: SVD of the (r_{k-1} n_k) x r_k unfolding M = U S V^T through
//      the eigen-decomposition (cyclic Jacobi, FP64, shared memory) of the smaller of M M^T and
//      M^T M, truncated to the leading min(max_rank, rows, cols) triplets; every kept left
//      singular vector has its entry of largest magnitude positive; W_k <- U,
//      W_{k+1} <- (S V^T) W_{k+1}.
// The working cores live in the workspace in FP64 (each core keeps its input capacity; ranks
// only shrink); the output is written in FP32. The eigen-decompositions are limited to
// T3F_ROUND_MAX_SIDE rows (160 KB of shared memory for the matrix and its eigenvectors).
#include <math.h>
#include <string.h>

#include <algorithm>

#include "t3f_internal.cuh"

namespace t3f {

namespace {

constexpr int kRoundThreads = 256;
constexpr int kMaxSide = 100;  // largest eigenproblem (rows of the Gram matrix)

struct RoundArgs {
  TTV X, Y;
  int maxr;
  long long coff[T3F_MAX_D];  // FP64 offset of core k inside an object's working set
  long long maxcore;          // largest core (elements)
  long long per_obj;          // doubles per object: cores + 2 scratch buffers
  double* ws;
  int* err;
};

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

// Householder QR of the column-major m x c matrix A (column a at A + a*m), q = min(m, c)
// reflectors. On return the upper triangle of A's first q rows is R (diag(R) >= 0 after the
// sign fix) and Q (m x q, column-major) is in Qo.
__device__ void householder_qr(double* A, int m, int c, double* Qo, double* sh_v0, double* sh_tau, double* red) {
  const int q = min(m, c);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < q; ++j) {
    double* x = A + (long long)j * m;
    double part = 0.0;
    for (int i = j + tid; i < m; i += blockDim.x) part += x[i] * x[i];
    const double nrm2 = block_sum(part, red);
    const double x0 = x[j];
    const double alpha = -(x0 >= 0.0 ? 1.0 : -1.0) * sqrt(nrm2);
    const double v0 = x0 - alpha;
    const double vn2 = nrm2 - x0 * x0 + v0 * v0;
    const double tau = vn2 > 0.0 ? 2.0 / vn2 : 0.0;
    // apply H_j = I - tau v v^T (v = [v0, x[j+1..m)]) to the columns j+1..c-1, a warp each
    for (int l = j + 1 + warp; l < c; l += nw) {
      double* y = A + (long long)l * m;
      double s = 0.0;
      for (int i = j + 1 + lane; i < m; i += 32) s += x[i] * y[i];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      s = tau * (s + v0 * y[j]);
      if (lane == 0) y[j] -= s * v0;
      for (int i = j + 1 + lane; i < m; i += 32) y[i] -= s * x[i];
    }
    __syncthreads();
    if (tid == 0) {
      sh_v0[j] = v0;
      sh_tau[j] = tau;
      x[j] = alpha;
    }
    __syncthreads();
  }
  // Q = H_0 ... H_{q-1} [I; 0], applied from the last reflector back
  for (int e = tid; e < m * q; e += blockDim.x) Qo[e] = (e % m) == (e / m) ? 1.0 : 0.0;
  __syncthreads();
  for (int j = q - 1; j >= 0; --j) {
    const double* x = A + (long long)j * m;
    const double v0 = sh_v0[j], tau = sh_tau[j];
    for (int l = j + warp; l < q; l += nw) {
      double* y = Qo + (long long)l * m;
      double s = 0.0;
      for (int i = j + 1 + lane; i < m; i += 32) s += x[i] * y[i];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      s = tau * (s + v0 * y[j]);
      if (lane == 0) y[j] -= s * v0;
      for (int i = j + 1 + lane; i < m; i += 32) y[i] -= s * x[i];
    }
    __syncthreads();
  }
  // signs: diag(R) >= 0 (flip column j of Q and row j of R)
  for (int e = tid; e < q * m; e += blockDim.x) {
    const int j = e / m;
    if (A[(long long)j * m + j] < 0.0) Qo[e] = -Qo[e];
  }
  __syncthreads();
  for (int e = tid; e < q * c; e += blockDim.x) {
    const int j = e / c, a = e % c;
    if (a > j && A[(long long)j * m + j] < 0.0) A[(long long)a * m + j] = -A[(long long)a * m + j];
  }
  __syncthreads();
  for (int j = tid; j < q; j += blockDim.x)
    if (A[(long long)j * m + j] < 0.0) A[(long long)j * m + j] = -A[(long long)j * m + j];
  __syncthreads();
}

// Cyclic Jacobi eigen-decomposition of the symmetric s x s matrix S (row-major, shared memory)
// with rotations of s/2 disjoint pairs at a time (round-robin ordering); V receives the
// eigenvectors (columns), diag(S) the eigenvalues.
__device__ void jacobi_eig(double* S, double* V, int s, int* pp, int* pq, double* pc, double* ps, double* red) {
  const int tid = threadIdx.x;
  const int se = s + (s & 1);  // even count; index s is a dummy
  const int np = se / 2;
  for (int e = tid; e < s * s; e += blockDim.x) V[e] = (e / s) == (e % s) ? 1.0 : 0.0;
  __syncthreads();
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int e = tid; e < s * s; e += blockDim.x) {
      const double v = S[e];
      if ((e / s) == (e % s)) dia += v * v; else off += v * v;
    }
    off = block_sum(off, red);
    dia = block_sum(dia, red);
    if (off <= 1e-30 * dia || off == 0.0) break;
    for (int rnd = 0; rnd < se - 1; ++rnd) {
      // round-robin pairs: position 0 fixed, positions 1..se-1 rotate
      for (int t = tid; t < np; t += blockDim.x) {
        auto at = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + rnd) % (se - 1); };
        int p = at(t), q = at(se - 1 - t);
        if (p > q) { const int tmp = p; p = q; q = tmp; }
        double c = 1.0, sn = 0.0;
        if (q < s) {
          const double apq = S[p * s + q];
          if (apq != 0.0) {
            const double tau = (S[q * s + q] - S[p * s + p]) / (2.0 * apq);
            const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + tt * tt);
            sn = tt * c;
          }
        }
        pp[t] = p;
        pq[t] = q;
        pc[t] = c;
        ps[t] = sn;
      }
      __syncthreads();
      // columns: S <- S J, V <- V J
      for (int e = tid; e < s * np; e += blockDim.x) {
        const int i = e / np, t = e % np, p = pp[t], q = pq[t];
        if (q >= s) continue;
        const double c = pc[t], sn = ps[t];
        const double a = S[i * s + p], b = S[i * s + q];
        S[i * s + p] = c * a - sn * b;
        S[i * s + q] = sn * a + c * b;
        const double va = V[i * s + p], vb = V[i * s + q];
        V[i * s + p] = c * va - sn * vb;
        V[i * s + q] = sn * va + c * vb;
      }
      __syncthreads();
      // rows: S <- J^T S
      for (int e = tid; e < s * np; e += blockDim.x) {
        const int j = e / np, t = e % np, p = pp[t], q = pq[t];
        if (q >= s) continue;
        const double c = pc[t], sn = ps[t];
        const double a = S[p * s + j], b = S[q * s + j];
        S[p * s + j] = c * a - sn * b;
        S[q * s + j] = sn * a + c * b;
      }
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(kRoundThreads) k_round(const __grid_constant__ RoundArgs a) {
  extern __shared__ double dsm[];
  double* Sg = dsm;                        // kMaxSide^2
  double* Vg = Sg + kMaxSide * kMaxSide;   // kMaxSide^2
  __shared__ double red[kRoundThreads / 32];
  __shared__ double sh_v0[kMaxSide + T3F_MAX_RANK], sh_tau[kMaxSide + T3F_MAX_RANK];
  __shared__ double pc[kMaxSide / 2 + 1], ps[kMaxSide / 2 + 1], sig[kMaxSide];
  __shared__ int pp[kMaxSide / 2 + 1], pq[kMaxSide / 2 + 1], perm[kMaxSide];
  __shared__ int rk[T3F_MAX_D + 1];
  const int obj = blockIdx.x, tid = threadIdx.x, d = a.X.d;
  double* W = a.ws + (long long)obj * a.per_obj;
  double* S1 = W + a.coff[d - 1] + a.X.osz[d - 1];
  double* S2 = S1 + a.maxcore;
  // FP64 working copy of the object
  const float* Xp = static_cast<const float*>(a.X.p);
  for (int k = 0; k < d; ++k) {
    const float* src = Xp + core_base(a.X, k, obj);
    for (long long e = tid; e < a.X.osz[k]; e += blockDim.x) W[a.coff[k] + e] = (double)src[e];
  }
  if (tid <= d) rk[tid] = a.X.r[tid];
  __syncthreads();
  // 1. right-to-left orthogonalisation
  for (int k = d - 1; k >= 1; --k) {
    const int r0 = rk[k], n = a.X.n[k], r1 = rk[k + 1];
    const int m = n * r1, c = r0, q = min(m, c);
    double* Wk = W + a.coff[k];
    // W_k row-major r0 x (n r1) is W_k^T column-major: factor it in place in S1
    for (long long e = tid; e < (long long)m * c; e += blockDim.x) S1[e] = Wk[e];
    __syncthreads();
    householder_qr(S1, m, c, S2, sh_v0, sh_tau, red);
    for (long long e = tid; e < (long long)m * q; e += blockDim.x) Wk[e] = S2[e];  // Q^T row-major
    __syncthreads();
    // W_{k-1} <- W_{k-1} R^T: rows (r_{k-2} n_{k-1}), c -> q columns
    double* Wp = W + a.coff[k - 1];
    const int rows = rk[k - 1] * a.X.n[k - 1];
    for (long long e = tid; e < (long long)rows * q; e += blockDim.x) {
      const int row = (int)(e / q), j = (int)(e % q);
      double s = 0.0;
      for (int aa = j; aa < c; ++aa) s += Wp[(long long)row * c + aa] * S1[(long long)aa * m + j];
      S2[e] = s;
    }
    __syncthreads();
    for (long long e = tid; e < (long long)rows * q; e += blockDim.x) Wp[e] = S2[e];
    if (tid == 0) rk[k] = q;
    __syncthreads();
  }
  // 2. left-to-right truncated SVDs
  for (int k = 0; k + 1 < d; ++k) {
    const int r0 = rk[k], n = a.X.n[k], c = rk[k + 1];
    const int m = r0 * n;
    const bool rows_side = m <= c;  // eigen-decompose M M^T (else M^T M)
    const int s = rows_side ? m : c;
    const int p = min(a.maxr, s);
    double* M = W + a.coff[k];
    for (int e = tid; e < s * s; e += blockDim.x) {
      const int x = e / s, y = e % s;
      double v = 0.0;
      if (rows_side)
        for (int b = 0; b < c; ++b) v += M[(long long)x * c + b] * M[(long long)y * c + b];
      else
        for (int row = 0; row < m; ++row) v += M[(long long)row * c + x] * M[(long long)row * c + y];
      Sg[e] = v;
    }
    __syncthreads();
    jacobi_eig(Sg, Vg, s, pp, pq, pc, ps, red);
    // order by eigenvalue, largest first (ties by index)
    for (int j = tid; j < s; j += blockDim.x) {
      const double lj = Sg[j * s + j];
      int pos = 0;
      for (int l = 0; l < s; ++l) {
        const double ll = Sg[l * s + l];
        pos += (ll > lj || (ll == lj && l < j)) ? 1 : 0;
      }
      perm[pos] = j;
    }
    __syncthreads();
    for (int j = tid; j < p; j += blockDim.x) sig[j] = sqrt(fmax(Sg[perm[j] * s + perm[j]], 0.0));
    __syncthreads();
    // U (m x p, row-major) in S1, S V^T (p x c, row-major) in S2
    for (long long e = tid; e < (long long)m * p; e += blockDim.x) {
      const int x = (int)(e / p), j = (int)(e % p), col = perm[j];
      double u;
      if (rows_side) {
        u = Vg[x * s + col];
      } else {
        double t = 0.0;
        for (int b = 0; b < c; ++b) t += M[(long long)x * c + b] * Vg[b * s + col];
        u = sig[j] > 0.0 ? t / sig[j] : 0.0;
      }
      S1[e] = u;
    }
    __syncthreads();
    for (long long e = tid; e < (long long)p * c; e += blockDim.x) {
      const int j = (int)(e / c), b = (int)(e % c);
      double v;
      if (rows_side) {
        v = 0.0;
        for (int x = 0; x < m; ++x) v += S1[(long long)x * p + j] * M[(long long)x * c + b];
      } else {
        v = sig[j] * Vg[b * s + perm[j]];
      }
      S2[e] = v;
    }
    __syncthreads();
    // sign convention: the entry of largest magnitude of every kept column of U is positive
    for (int j = tid; j < p; j += blockDim.x) {
      int best = 0;
      double bv = -1.0;
      for (int x = 0; x < m; ++x) {
        const double v = fabs(S1[(long long)x * p + j]);
        if (v > bv) {
          bv = v;
          best = x;
        }
      }
      sig[j] = S1[(long long)best * p + j] < 0.0 ? -1.0 : 1.0;
    }
    __syncthreads();
    for (long long e = tid; e < (long long)m * p; e += blockDim.x) M[e] = S1[e] * sig[e % p];
    for (long long e = tid; e < (long long)p * c; e += blockDim.x) S2[e] *= sig[e / c];
    __syncthreads();
    // W_{k+1} <- (S V^T) W_{k+1}: c x (n_{k+1} r_{k+2}) -> p x (...)
    double* Wn = W + a.coff[k + 1];
    const int cols = a.X.n[k + 1] * rk[k + 2];
    for (long long e = tid; e < (long long)p * cols; e += blockDim.x) {
      const int j = (int)(e / cols), col = (int)(e % cols);
      double t = 0.0;
      for (int b = 0; b < c; ++b) t += S2[(long long)j * c + b] * Wn[(long long)b * cols + col];
      S1[e] = t;
    }
    __syncthreads();
    for (long long e = tid; e < (long long)p * cols; e += blockDim.x) Wn[e] = S1[e];
    if (tid == 0) rk[k + 1] = p;
    __syncthreads();
  }
  // FP32 output with the final ranks
  float* Yp = static_cast<float*>(a.Y.p);
  for (int k = 0; k < d; ++k) {
    float* dst = Yp + core_base(a.Y, k, obj);
    for (long long e = tid; e < a.Y.osz[k]; e += blockDim.x) dst[e] = (float)W[a.coff[k] + e];
  }
}

struct RoundPlan {
  long long coff[T3F_MAX_D];
  long long maxcore, per_obj;
  size_t total;
};

RoundPlan round_plan(const TTV& X) {
  RoundPlan p;
  long long o = 0, mx = 1;
  for (int k = 0; k < X.d; ++k) {
    p.coff[k] = o;
    o += X.osz[k];
    mx = std::max(mx, X.osz[k]);
  }
  p.maxcore = mx;
  p.per_obj = o + 2 * mx;
  p.total = kWsHeader + align256(sizeof(double) * (size_t)p.per_obj * X.batch);
  return p;
}

void round_ranks_host(int d, const int* n, const int* ranks, int maxr, int* out, int* rr) {
  for (int k = 0; k <= d; ++k) rr[k] = ranks[k];
  for (int k = d - 1; k >= 1; --k) rr[k] = (int)std::min<long long>(rr[k], (long long)n[k] * rr[k + 1]);
  out[0] = 1;
  for (int k = 1; k < d; ++k)
    out[k] = (int)std::min<long long>(std::min<long long>((long long)out[k - 1] * n[k - 1], rr[k]), maxr);
  out[d] = 1;
}

}  // namespace

size_t ws_round(const TTV& X) { return round_plan(X).total; }

}  // namespace t3f

using namespace t3f;

extern "C" t3f_status t3f_round_ranks(int32_t d, const int32_t* n, const int32_t* ranks, int32_t max_rank,
                                      int32_t* out_ranks) {
  if (d < 1 || d > T3F_MAX_D || !n || !ranks || !out_ranks || max_rank < 1) return T3F_ERR_ARG;
  if (ranks[0] != 1 || ranks[d] != 1) return T3F_ERR_SHAPE;
  for (int k = 0; k <= d; ++k)
    if (ranks[k] < 1) return T3F_ERR_SHAPE;
  for (int k = 0; k < d; ++k)
    if (n[k] < 1) return T3F_ERR_SHAPE;
  int rr[T3F_MAX_D + 1];
  round_ranks_host(d, n, ranks, max_rank, out_ranks, rr);
  return T3F_OK;
}

extern "C" t3f_status t3f_round(const t3f_tt* X, int32_t max_rank, t3f_tt* Y, void* ws, size_t ws_bytes,
                                t3f_stream_t stream) {
  TTV vx, vy;
  T3F_CHECK(make_view(X, &vx, T3F_F32, false));
  T3F_CHECK(make_view(Y, &vy, T3F_F32, false));
  if (max_rank < 1) return T3F_ERR_ARG;
  if (vy.batch != vx.batch || vy.d != vx.d) return T3F_ERR_SHAPE;
  int want[T3F_MAX_D + 1], rr[T3F_MAX_D + 1];
  round_ranks_host(vx.d, vx.n, vx.r, max_rank, want, rr);
  for (int k = 0; k <= vx.d; ++k)
    if (vy.r[k] != want[k] || (k < vx.d && vy.n[k] != vx.n[k])) return T3F_ERR_SHAPE;
  // limits: the QR reflector count and every eigenproblem side
  for (int k = 1; k < vx.d; ++k)
    if (std::min<long long>((long long)vx.n[k] * rr[k + 1], vx.r[k]) > kMaxSide + T3F_MAX_RANK) return T3F_ERR_UNSUPPORTED;
  for (int k = 0; k + 1 < vx.d; ++k)
    if (std::min<long long>((long long)want[k] * vx.n[k], rr[k + 1]) > kMaxSide) return T3F_ERR_UNSUPPORTED;
  const RoundPlan p = round_plan(vx);
  T3F_CHECK(check_ws(ws, ws_bytes, p.total));
  cudaStream_t s = (cudaStream_t)stream;
  RoundArgs a;
  memset(&a, 0, sizeof(a));
  a.X = vx;
  a.Y = vy;
  a.maxr = max_rank;
  for (int k = 0; k < vx.d; ++k) a.coff[k] = p.coff[k];
  a.maxcore = p.maxcore;
  a.per_obj = p.per_obj;
  a.ws = reinterpret_cast<double*>(static_cast<char*>(ws) + kWsHeader);
  a.err = static_cast<int*>(ws);
  const size_t smem = sizeof(double) * 2 * kMaxSide * kMaxSide;
  if (cudaFuncSetAttribute(k_round, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return T3F_ERR_CUDA;
  k_round<<<(unsigned)vx.batch, kRoundThreads, smem, s>>>(a);
  return launch_status();
}
