// FP64 Householder orthogonalisation of TT-cores (the left- and right-orthogonal forms that
// the tangent-space operations of the paper's Section 3.2 are built on).
//
// One CTA per TT object runs three sweeps on an FP64 copy of the cores in the workspace:
//   right-to-left on X (LQ steps: QR of the transposed r_{k-1} x (n_k r_k) unfolding,
//   R^T pushed into core k-1), left-to-right on the result (QR of the (r_{k-1} n_k) x r_k
//   unfolding, R pushed into core k+1) giving U, and right-to-left on U giving V.
// Every QR is a textbook Householder factorisation (Golub & Van Loan, Algorithm 5.2.1)
// followed by the sign normalisation diag(R) >= 0, which makes Q and R unique for a
// full-rank unfolding.
#include <math.h>

#include "t3f_internal.cuh"

namespace t3f {

constexpr int kOrthThreads = 256;
constexpr int kOrthMaxRows = 4096;

struct OrthArgs {
  TTV X, U, V;
  int ru[T3F_MAX_D + 1];     // ranks after the sweeps
  double* work;              // per object: cores region + scratch
  long long obj_stride;      // doubles per object
  long long coff[T3F_MAX_D]; // offset of working core k within the object region
  long long scratch_off;     // offset of the scratch within the object region
};

__device__ double cta_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

// Householder QR of the column-major m x c matrix W (leading dimension m) in place.
// On exit Q (m x kk, column-major) and R (kk x c, row-major) hold the sign-normalised
// factors, kk = min(m, c). Hv (m x kk) receives the unit Householder vectors.
__device__ void cta_qr(double* W, int m, int c, double* Q, double* R, double* Hv, double* red,
                       double* bcast) {
  const int kk = m < c ? m : c;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nth >> 5;
  for (int j = 0; j < kk; ++j) {
    double* x = W + (long long)j * m;
    double part = 0.0;
    for (int r = j + tid; r < m; r += nth) part += x[r] * x[r];
    const double nrm2 = cta_sum(part, red);
    const double x0 = x[j];
    const double nrm = sqrt(nrm2);
    const double alpha = x0 >= 0.0 ? -nrm : nrm;
    const double v0 = x0 - alpha;
    const double vn2 = nrm2 - x0 * x0 + v0 * v0;
    const double inv = vn2 > 0.0 ? 1.0 / sqrt(vn2) : 0.0;
    double* v = Hv + (long long)j * m;
    for (int r = tid; r < m; r += nth) v[r] = r < j ? 0.0 : (r == j ? v0 : x[r]) * inv;
    __syncthreads();
    // apply H = I - 2 v v^T to columns j..c-1, one warp per column
    for (int l = j + wid; l < c; l += nw) {
      double* col = W + (long long)l * m;
      double s = 0.0;
      for (int r = j + lane; r < m; r += 32) s += v[r] * col[r];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      for (int r = j + lane; r < m; r += 32) col[r] -= 2.0 * v[r] * s;
    }
    __syncthreads();
    (void)bcast;
  }
  // Q = H_0 ... H_{kk-1} [I; 0]
  for (int e = tid; e < m * kk; e += nth) {
    const int r = e % m, l = e / m;
    Q[e] = r == l ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = kk - 1; j >= 0; --j) {
    const double* v = Hv + (long long)j * m;
    for (int l = wid; l < kk; l += nw) {
      double* col = Q + (long long)l * m;
      double s = 0.0;
      for (int r = j + lane; r < m; r += 32) s += v[r] * col[r];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      for (int r = j + lane; r < m; r += 32) col[r] -= 2.0 * v[r] * s;
    }
    __syncthreads();
  }
  // R = upper triangle of W; sign normalisation diag(R) >= 0
  for (int e = tid; e < kk * c; e += nth) {
    const int r = e / c, l = e % c;
    const double sgn = W[(long long)r * m + r] < 0.0 ? -1.0 : 1.0;
    R[e] = l < r ? 0.0 : sgn * W[(long long)l * m + r];
  }
  for (int e = tid; e < m * kk; e += nth) {
    const int l = e / m;
    if (W[(long long)l * m + l] < 0.0) Q[e] = -Q[e];
  }
  __syncthreads();
}

struct CoreDims {
  int r0, n, r1;
};

// Right-to-left sweep over the working cores (dims updated in place).
__device__ void sweep_rl(double* base, const long long* coff, CoreDims* dims, int d,
                         double* Wm, double* Q, double* R, double* Hv, double* red, double* bc) {
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int k = d - 1; k >= 1; --k) {
    const int r0 = dims[k].r0, n = dims[k].n, r1 = dims[k].r1;
    const int m = n * r1, c = r0, kk = m < c ? m : c;
    double* core = base + coff[k];
    // W = core^T, column-major m x c: W[(i r1 + b) + a m] = core[a][i][b]
    for (int e = tid; e < m * c; e += nth) {
      const int a = e / m, q = e % m;
      Wm[e] = core[(long long)a * m + q];
    }
    __syncthreads();
    cta_qr(Wm, m, c, Q, R, Hv, red, bc);
    // new core k (kk x n x r1) = Q^T
    for (int e = tid; e < kk * m; e += nth) {
      const int a = e / m, q = e % m;
      core[e] = Q[(long long)a * m + q];
    }
    // core k-1 (p0 x n' x r0) <- core_{k-1} R^T  -> (p0 x n' x kk)
    double* prev = base + coff[k - 1];
    const int rows = dims[k - 1].r0 * dims[k - 1].n;
    __syncthreads();
    // compute into Wm then copy back (Wm is free now)
    for (int e = tid; e < rows * kk; e += nth) {
      const int row = e / kk, a2 = e % kk;
      double s = 0.0;
      for (int a = 0; a < c; ++a) s += prev[(long long)row * c + a] * R[(long long)a2 * c + a];
      Wm[e] = s;
    }
    __syncthreads();
    for (int e = tid; e < rows * kk; e += nth) prev[e] = Wm[e];
    if (tid == 0) {
      dims[k].r0 = kk;
      dims[k - 1].r1 = kk;
    }
    __syncthreads();
  }
}

// Left-to-right sweep over the working cores.
__device__ void sweep_lr(double* base, const long long* coff, CoreDims* dims, int d,
                         double* Wm, double* Q, double* R, double* Hv, double* red, double* bc) {
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int k = 0; k < d - 1; ++k) {
    const int r0 = dims[k].r0, n = dims[k].n, r1 = dims[k].r1;
    const int m = r0 * n, c = r1, kk = m < c ? m : c;
    double* core = base + coff[k];
    // W column-major m x c: W[q + l m] = core[q * c + l]
    for (int e = tid; e < m * c; e += nth) {
      const int l = e / m, q = e % m;
      Wm[e] = core[(long long)q * c + l];
    }
    __syncthreads();
    cta_qr(Wm, m, c, Q, R, Hv, red, bc);
    for (int e = tid; e < m * kk; e += nth) {
      const int q = e / kk, l = e % kk;
      core[e] = Q[(long long)l * m + q];
    }
    // core k+1 (r1 x n' x r2) <- R (kk x r1) core_{k+1}
    double* next = base + coff[k + 1];
    const int cols = dims[k + 1].n * dims[k + 1].r1;
    __syncthreads();
    for (int e = tid; e < kk * cols; e += nth) {
      const int a2 = e / cols, q = e % cols;
      double s = 0.0;
      for (int a = 0; a < c; ++a) s += R[(long long)a2 * c + a] * next[(long long)a * cols + q];
      Wm[e] = s;
    }
    __syncthreads();
    for (int e = tid; e < kk * cols; e += nth) next[e] = Wm[e];
    if (tid == 0) {
      dims[k].r1 = kk;
      dims[k + 1].r0 = kk;
    }
    __syncthreads();
  }
}

__device__ void write_out(const TTV& O, int obj, const double* base, const long long* coff,
                          const CoreDims* dims, int d) {
  for (int k = 0; k < d; ++k) {
    const long long sz = (long long)dims[k].r0 * dims[k].n * dims[k].r1;
    const long long ob = core_base(O, k, obj);
    if (O.dtype == T3F_F64) {
      double* o = static_cast<double*>(O.p) + ob;
      for (long long e = threadIdx.x; e < sz; e += blockDim.x) o[e] = base[coff[k] + e];
    } else {
      float* o = static_cast<float*>(O.p) + ob;
      for (long long e = threadIdx.x; e < sz; e += blockDim.x) o[e] = (float)base[coff[k] + e];
    }
  }
}

__global__ void __launch_bounds__(kOrthThreads) k_orth(const __grid_constant__ OrthArgs a) {
  __shared__ double red[kOrthThreads / 32];
  __shared__ double bc[2];
  __shared__ CoreDims dims[T3F_MAX_D];
  const int obj = blockIdx.x;
  const TTV& X = a.X;
  const int d = X.d;
  double* base = a.work + (long long)obj * a.obj_stride;
  double* scr = base + a.scratch_off;
  double* Wm = scr;
  double* Q = Wm + (long long)kOrthMaxRows * T3F_MAX_RANK;
  double* Hv = Q + (long long)kOrthMaxRows * T3F_MAX_RANK;
  double* R = Hv + (long long)kOrthMaxRows * T3F_MAX_RANK;
  for (int k = threadIdx.x; k < d; k += blockDim.x) dims[k] = CoreDims{X.r[k], X.n[k], X.r[k + 1]};
  // load X into the FP64 working cores
  for (int k = 0; k < d; ++k) {
    const long long ob = core_base(X, k, obj);
    const long long sz = X.osz[k];
    if (X.dtype == T3F_F64) {
      const double* xp = static_cast<const double*>(X.p) + ob;
      for (long long e = threadIdx.x; e < sz; e += blockDim.x) base[a.coff[k] + e] = xp[e];
    } else {
      const float* xp = static_cast<const float*>(X.p) + ob;
      for (long long e = threadIdx.x; e < sz; e += blockDim.x) base[a.coff[k] + e] = (double)xp[e];
    }
  }
  __syncthreads();
  sweep_rl(base, a.coff, dims, d, Wm, Q, R, Hv, red, bc);
  sweep_lr(base, a.coff, dims, d, Wm, Q, R, Hv, red, bc);
  write_out(a.U, obj, base, a.coff, dims, d);
  __syncthreads();
  sweep_rl(base, a.coff, dims, d, Wm, Q, R, Hv, red, bc);
  write_out(a.V, obj, base, a.coff, dims, d);
}

static long long orth_obj_stride(const TTV& X, long long* coff, long long* scratch_off) {
  long long o = 0;
  for (int k = 0; k < X.d; ++k) {
    if (coff) coff[k] = o;
    o += X.osz[k];
  }
  o = (o + 31) & ~31LL;
  if (scratch_off) *scratch_off = o;
  o += 3LL * kOrthMaxRows * T3F_MAX_RANK + (long long)T3F_MAX_RANK * T3F_MAX_RANK;
  return (o + 31) & ~31LL;
}

size_t ws_orth(const TTV& X) {
  return kWsHeader + align256(sizeof(double) * orth_obj_stride(X, nullptr, nullptr) * X.batch);
}

}  // namespace t3f

using namespace t3f;

extern "C" t3f_status t3f_orthogonalize(const t3f_tt* X, t3f_tt* U, t3f_tt* V, void* ws,
                                        size_t ws_bytes, t3f_stream_t stream) {
  TTV vx, vu, vv;
  T3F_CHECK(make_view(X, &vx, -1, false));
  if (vx.dtype == T3F_BF16) return T3F_ERR_DTYPE;
  T3F_CHECK(make_view(U, &vu, -1, false));
  T3F_CHECK(make_view(V, &vv, -1, false));
  if (vu.dtype == T3F_BF16 || vv.dtype == T3F_BF16) return T3F_ERR_DTYPE;
  if (vx.rmax > T3F_MAX_RANK) return T3F_ERR_UNSUPPORTED;
  for (int k = 0; k < vx.d; ++k) {
    if ((long long)vx.r[k] * vx.n[k] > kOrthMaxRows) return T3F_ERR_UNSUPPORTED;
    if ((long long)vx.n[k] * vx.r[k + 1] > kOrthMaxRows) return T3F_ERR_UNSUPPORTED;
  }
  int ru[T3F_MAX_D + 1];
  int xn[T3F_MAX_D], xr[T3F_MAX_D + 1];
  for (int k = 0; k < vx.d; ++k) xn[k] = vx.n[k];
  for (int k = 0; k <= vx.d; ++k) xr[k] = vx.r[k];
  T3F_CHECK(t3f_orth_ranks(vx.d, xn, xr, ru));
  for (const TTV* o : {&vu, &vv}) {
    if (o->batch != vx.batch || o->d != vx.d) return T3F_ERR_SHAPE;
    for (int k = 0; k <= vx.d; ++k)
      if (o->r[k] != ru[k] || (k < vx.d && o->n[k] != vx.n[k])) return T3F_ERR_SHAPE;
  }
  T3F_CHECK(check_ws(ws, ws_bytes, ws_orth(vx)));
  OrthArgs args;
  memset(&args, 0, sizeof(args));
  args.X = vx;
  args.U = vu;
  args.V = vv;
  for (int k = 0; k <= vx.d; ++k) args.ru[k] = ru[k];
  args.work = reinterpret_cast<double*>(static_cast<char*>(ws) + kWsHeader);
  args.obj_stride = orth_obj_stride(vx, args.coff, &args.scratch_off);
  k_orth<<<vx.batch, kOrthThreads, 0, (cudaStream_t)stream>>>(args);
  return launch_status();
}
