// FP64 Householder orthogonalisation of TT-cores (the left- and right-orthogonal forms that
// the tangent-space operations of the paper's Section 3.2 are built on).
//
// Three sweeps over an FP64 working copy of the cores: right-to-left on X (LQ steps: QR of
// the transposed r_{k-1} x (n_k r_k) unfolding, R^T pushed into core k-1), left-to-right on
// the result (QR of the (r_{k-1} n_k) x r_k unfolding, R pushed into core k+1) giving U, and
// right-to-left on U giving V. Every QR normalises diag(R) >= 0, which makes the factors of a
// full-rank unfolding unique.
//
// GB300 runs FP64 at a small fraction of its FP32 rate, so one QR is spread over a cluster
// of P CTAs (P = 16 when the device allows it, else 8): the m rows of the unfolding W are
// split into P contiguous blocks held in shared memory. Column j's Householder reflector
// (LAPACK dlarfg convention, Golub & Van Loan Algorithm 5.1.1) needs the norm of x = W[j:, j]
// and the products v . W[:, l] with the trailing columns; both follow from one set of
// partial sums per CTA (x.x and x.W[:, l] below the diagonal, plus row j), exchanged through
// distributed shared memory behind a single cluster barrier per column (the publish slots
// alternate between two buffers). R is then broadcast to every CTA and Q = W R^{-1} is
// recovered row by row by a triangular solve that needs no further communication. The
// working cores keep their original row strides so every in-place update touches only the
// rows or columns its CTA owns.
#include <cooperative_groups.h>
#include <math.h>

#include "t3f_internal.cuh"

namespace cg = cooperative_groups;

namespace t3f {

constexpr int kOrthThreads = 256;
constexpr int kOrthMaxRows = 4096;

struct OrthArgs {
  TTV X, U, V;
  int P;                      // CTAs per cluster
  int rows_per;               // max rows of W per CTA (ceil(kOrthMaxRows / P) bound)
  double* work;               // per object: padded working cores
  long long obj_stride;       // doubles per object
  long long coff[T3F_MAX_D];  // offset of working core k
  int R1[T3F_MAX_D];          // padded row stride of core k (= original r_{k+1})
};

struct Dims {
  int r0, n, r1;
};

struct OrthSmem {
  double* W;      // rows_per x c working block (row-major, ld = c)
  double* Rs;     // T3F_MAX_RANK x T3F_MAX_RANK
  double* pub;    // [2][T3F_MAX_RANK] published partial dots (index j holds the squared norm)
  double* rowj;   // [2][T3F_MAX_RANK] published row j (owner only)
  double* gsum;   // T3F_MAX_RANK gathered dots
  double* wj;     // T3F_MAX_RANK row j of W
  double* rinv;   // T3F_MAX_RANK reciprocals of diag(R)
  double* tv;     // rows_per: tau * v_r of the owned rows
  double* refl;   // 4: beta, tau, scale of the current reflector
};

// Address of element (row q, col l) of W inside the padded working core.
//   lr = 1: W = left unfolding, row q = a * n + i, col l = b   -> (a n + i) R1 + l
//   lr = 0: W = transposed right unfolding, row q = i * r1 + b, col l = a
__device__ __forceinline__ long long w_addr(int lr, int q, int l, const Dims& dm, int R1) {
  if (lr) return (long long)q * R1 + l;
  const int i = q / dm.r1, b = q % dm.r1;
  return ((long long)l * dm.n + i) * R1 + b;
}

// One QR step of a sweep on core k (updates dims for core k and its neighbour).
__device__ void qr_step(const OrthArgs& a, double* base, Dims* dims, int k, int lr,
                        const OrthSmem& s, cg::cluster_group& cluster) {
  const int P = a.P;
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, nth = blockDim.x;
  const Dims dm = dims[k];
  const int m = lr ? dm.r0 * dm.n : dm.n * dm.r1;
  const int c = lr ? dm.r1 : dm.r0;
  const int kk = m < c ? m : c;
  const int rp = (m + P - 1) / P;
  const int row0 = rank * rp;
  const int nrow = max(0, min(m, row0 + rp) - row0);
  double* core = base + a.coff[k];
  const int R1 = a.R1[k];

  cluster.sync();  // previous step's global writes are visible; remote smem reads are done
  for (int e = tid; e < nrow * c; e += nth) {
    const int q = e / c, l = e % c;
    s.W[e] = core[w_addr(lr, row0 + q, l, dm, R1)];
  }
  __syncthreads();

  for (int j = 0; j < kk; ++j) {
    const int par = j & 1;
    double* pub = s.pub + par * T3F_MAX_RANK;
    double* rowj = s.rowj + par * T3F_MAX_RANK;
    const bool own_j = j >= row0 && j < row0 + nrow;
    // (1) partials over the owned rows strictly below the diagonal:
    //     pub[j] = sum x_r^2, pub[l] = sum x_r W[r][l] (l > j); the owner publishes row j.
    //     Eight lanes per column split the rows and combine with three shuffles.
    const int q_lo = max(0, j + 1 - row0);
    for (int cb = j; cb < c; cb += nth / 8) {
      const int l = cb + tid / 8, g = tid % 8;
      double acc = 0.0;
      if (l < c)
        for (int q = q_lo + g; q < nrow; q += 8) acc = fma(s.W[q * c + j], s.W[q * c + l], acc);
      acc += __shfl_xor_sync(0xffffffffu, acc, 4, 8);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2, 8);
      acc += __shfl_xor_sync(0xffffffffu, acc, 1, 8);
      if (g == 0 && l < c) pub[l] = acc;
    }
    if (own_j)
      for (int l = j + tid; l < c; l += nth) rowj[l] = s.W[(j - row0) * c + l];
    __syncthreads();
    cluster.sync();
    // (2) gather the cluster sums (8 lanes per column, each reading the partials of ranks g
    //     and g + 8 in one round trip); the lane that owns column j also forms the reflector
    //     (LAPACK dlarfg convention: beta = -sign(w) |x|, tau = (beta - w) / beta,
    //     scale = 1 / (w - beta), with 1 / |x| from one reciprocal square root)
    const int jown = j / rp;
    const int ng = ((c - j) * 8 + 31) & ~31;  // whole warps take part in the shuffles
    for (int e = tid; e < ng; e += nth) {
      const int l = j + e / 8, p = e % 8;
      double v = 0.0, v2 = 0.0, wl = 0.0;
      if (l < c) {
        if (p < P) v = cluster.map_shared_rank(pub, p)[l];
        if (p + 8 < P) v2 = cluster.map_shared_rank(pub, p + 8)[l];
        if (p == 0) wl = cluster.map_shared_rank(rowj, jown)[l];  // issued with v
      }
      v += v2;
      for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, 8);
      if (p == 0 && l < c) {
        s.gsum[l] = v;
        s.wj[l] = wl;
        if (l == j) {
          double beta = wl, tau = 0.0, scale = 0.0;
          if (v != 0.0) {
            const double x2 = wl * wl + v, rn = rsqrt(x2), nrm = x2 * rn;
            const bool pos = wl >= 0.0;
            beta = pos ? -nrm : nrm;
            tau = pos ? 1.0 + wl * rn : 1.0 - wl * rn;  // 1 - wl / beta
            scale = 1.0 / (wl - beta);
          }
          s.refl[0] = beta;
          s.refl[1] = tau;
          s.refl[2] = scale;
        }
      }
    }
    __syncthreads();
    const double beta = s.refl[0], tau = s.refl[1], scale = s.refl[2];
    // (3) w_l = v . W[:, l] for the trailing columns and tau v_r for the owned rows, then the
    //     rank-one update of the owned rows
    for (int l = j + 1 + tid; l < c; l += nth) s.gsum[l] = s.wj[l] + scale * s.gsum[l];
    const int q_j = max(0, j - row0);
    for (int q = q_j + tid; q < nrow; q += nth) s.tv[q] = row0 + q == j ? tau : tau * scale * s.W[q * c + j];
    __syncthreads();
    const int wc = c - j - 1, wr = nrow - q_j;
    for (int e = tid; e < wr * wc; e += nth) {
      const int q = q_j + e / wc, l = j + 1 + e % wc;
      s.W[q * c + l] -= s.tv[q] * s.gsum[l];
    }
    if (own_j && tid == 0) s.W[(j - row0) * c + j] = beta;
    __syncthreads();
  }
  cluster.sync();  // every row of R is final in its owner's shared memory
  // (C) R (kk x c) from the owners of rows 0..kk-1, normalised to diag(R) >= 0
  for (int e = tid; e < kk * c; e += nth) {
    const int j = e / c, l = e % c;
    double v = 0.0;
    if (l >= j) {
      const int own = j / rp;
      v = cluster.map_shared_rank(s.W, own)[(j - own * rp) * c + l];
    }
    s.Rs[j * T3F_MAX_RANK + l] = v;
  }
  __syncthreads();
  for (int e = tid; e < kk * c; e += nth) {
    const int j = e / c, l = e % c;
    if (s.Rs[j * T3F_MAX_RANK + j] < 0.0 && l != j) s.Rs[j * T3F_MAX_RANK + l] = -s.Rs[j * T3F_MAX_RANK + l];
  }
  __syncthreads();
  for (int j = tid; j < kk; j += nth) {
    const double dg = fabs(s.Rs[j * T3F_MAX_RANK + j]);
    s.Rs[j * T3F_MAX_RANK + j] = dg;
    s.rinv[j] = 1.0 / dg;
  }
  cluster.sync();  // all CTAs are done reading remote W before it is reused below
  // (D) Q rows = W rows R[:kk,:kk]^{-1}: reload the original rows, forward substitution
  for (int e = tid; e < nrow * kk; e += nth) {
    const int q = e / kk, l = e % kk;
    s.W[q * c + l] = core[w_addr(lr, row0 + q, l, dm, R1)];
  }
  __syncthreads();
  // right-looking substitution: once q_b is known it is removed from every later column.
  // Eight lanes share a row: lane g keeps the columns l = g (mod 8) of the row in registers
  // and the owner of column b broadcasts q_b with a shuffle.
  if (kk <= 64) {
    const int g = tid % 8;
    const int nq = (nrow + (nth / 8) - 1) / (nth / 8);
    for (int it = 0; it < nq; ++it) {
      const int q = it * (nth / 8) + tid / 8;
      const bool qv = q < nrow;
      double* qr = s.W + (qv ? q : 0) * c;
      double x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int l = g + 8 * u;
        x[u] = (qv && l < kk) ? qr[l] : 0.0;
      }
      const int uend = (kk + 7) / 8;  // register slots holding columns < kk
      // column b = 8 UB + ob lives in slot UB of lane ob; only the slots UB .. uend-1 hold
      // columns l > b, so the loops start at UB at compile time and no update is issued
      // for the slots below it (the FP64 pipe is the scarce one)
#pragma unroll
      for (int UB = 0; UB < 8; ++UB) {
        if (UB >= uend) break;
        for (int ob = 0; ob < 8; ++ob) {
          const int b = 8 * UB + ob;
          if (b >= kk) break;
          double xb = __shfl_sync(0xffffffffu, x[UB] * s.rinv[b], ob, 8);
          if (g == ob) x[UB] = xb;
          const double* rb = s.Rs + b * T3F_MAX_RANK;
#pragma unroll
          for (int u = UB; u < 8; ++u) {
            const int l = g + 8 * u;
            if (u < uend && l > b && l < kk) x[u] = fma(-xb, rb[l], x[u]);
          }
        }
      }
      if (qv) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int l = g + 8 * u;
          if (l < kk) qr[l] = x[u];
        }
      }
    }
  }
  __syncthreads();
  Dims nd = dm;
  if (lr) nd.r1 = kk; else nd.r0 = kk;
  for (int e = tid; e < nrow * kk; e += nth) {
    const int q = e / kk, l = e % kk;
    // L->R: new core (r0, n, kk) row q col l; R->L: new core (kk, n, r1) = Q^T
    core[w_addr(lr, row0 + q, l, nd, R1)] = s.W[q * c + l];
  }
  __syncthreads();
  // (E) push R into the neighbour core, split across the cluster; operands staged in smem
  if (lr) {
    const Dims nx = dims[k + 1];  // (c, n', r2)
    double* nb = base + a.coff[k + 1];
    const int R1n = a.R1[k + 1];
    const int cols = nx.n * nx.r1;
    const int cp = (cols + P - 1) / P, c0 = rank * cp, nc = max(0, min(cols, c0 + cp) - c0);
    for (int e = tid; e < c * nc; e += nth) {
      const int al = e / nc, q = c0 + e % nc;
      const int i = q / nx.r1, b = q % nx.r1;
      s.W[e] = nb[((long long)al * nx.n + i) * R1n + b];
    }
    __syncthreads();
    for (int e = tid; e < kk * nc; e += nth) {
      const int a2 = e / nc, qq = e % nc, q = c0 + qq;
      const int i = q / nx.r1, b = q % nx.r1;
      double acc = 0.0;
      for (int al = a2; al < c; ++al) acc += s.Rs[a2 * T3F_MAX_RANK + al] * s.W[al * nc + qq];
      nb[((long long)a2 * nx.n + i) * R1n + b] = acc;
    }
  } else {
    const Dims pv = dims[k - 1];  // (r0', n', c)
    double* pb = base + a.coff[k - 1];
    const int R1p = a.R1[k - 1];
    const int rows = pv.r0 * pv.n;
    const int rq = (rows + P - 1) / P, q0 = rank * rq, nq = max(0, min(rows, q0 + rq) - q0);
    for (int e = tid; e < nq * c; e += nth) {
      const int q = e / c, b = e % c;
      s.W[e] = pb[(long long)(q0 + q) * R1p + b];
    }
    __syncthreads();
    for (int e = tid; e < nq * kk; e += nth) {
      const int q = e / kk, a2 = e % kk;
      double acc = 0.0;
      for (int b = a2; b < c; ++b) acc += s.W[q * c + b] * s.Rs[a2 * T3F_MAX_RANK + b];
      pb[(long long)(q0 + q) * R1p + a2] = acc;
    }
  }
  __syncthreads();
  __threadfence();
  if (tid == 0) {
    if (lr) {
      dims[k].r1 = kk;
      dims[k + 1].r0 = kk;
    } else {
      dims[k].r0 = kk;
      dims[k - 1].r1 = kk;
    }
  }
  __syncthreads();
}

__device__ void write_out(const OrthArgs& a, const TTV& O, int obj, const double* base,
                          const Dims* dims, cg::cluster_group& cluster) {
  cluster.sync();
  const int P = a.P, rank = (int)cluster.block_rank();
  for (int k = 0; k < O.d; ++k) {
    const Dims dm = dims[k];
    const long long sz = (long long)dm.r0 * dm.n * dm.r1;
    const long long ob = core_base(O, k, obj);
    for (long long e = (long long)rank * blockDim.x + threadIdx.x; e < sz; e += (long long)P * blockDim.x) {
      const int b = (int)(e % dm.r1);
      const long long ai = e / dm.r1;
      const double v = base[a.coff[k] + ai * a.R1[k] + b];
      if (O.dtype == T3F_F64) static_cast<double*>(O.p)[ob + e] = v;
      else static_cast<float*>(O.p)[ob + e] = (float)v;
    }
  }
}

__global__ void __launch_bounds__(kOrthThreads) k_orth(const __grid_constant__ OrthArgs a) {
  extern __shared__ double smd[];
  __shared__ Dims dims[T3F_MAX_D];
  cg::cluster_group cluster = cg::this_cluster();
  const int obj = blockIdx.x / a.P;
  const int rank = (int)cluster.block_rank();
  const TTV& X = a.X;
  const int d = X.d;
  OrthSmem s;
  s.W = smd;
  s.Rs = s.W + (size_t)a.rows_per * T3F_MAX_RANK;
  s.pub = s.Rs + T3F_MAX_RANK * T3F_MAX_RANK;
  s.rowj = s.pub + 2 * T3F_MAX_RANK;
  s.gsum = s.rowj + 2 * T3F_MAX_RANK;
  s.wj = s.gsum + T3F_MAX_RANK;
  s.rinv = s.wj + T3F_MAX_RANK;
  s.tv = s.rinv + T3F_MAX_RANK;
  s.refl = s.tv + a.rows_per;
  double* base = a.work + (long long)obj * a.obj_stride;
  for (int k = threadIdx.x; k < d; k += blockDim.x) dims[k] = Dims{X.r[k], X.n[k], X.r[k + 1]};
  // load X (split across the cluster) into the padded FP64 working cores
  for (int k = 0; k < d; ++k) {
    const long long sz = X.osz[k];
    const long long ob = core_base(X, k, obj);
    for (long long e = (long long)rank * blockDim.x + threadIdx.x; e < sz; e += (long long)a.P * blockDim.x) {
      const double v = X.dtype == T3F_F64 ? static_cast<const double*>(X.p)[ob + e]
                                          : (double)static_cast<const float*>(X.p)[ob + e];
      base[a.coff[k] + e] = v;  // the padded stride equals the original one for X
    }
  }
  __threadfence();
  __syncthreads();
  for (int k = d - 1; k >= 1; --k) qr_step(a, base, dims, k, 0, s, cluster);
  for (int k = 0; k < d - 1; ++k) qr_step(a, base, dims, k, 1, s, cluster);
  __threadfence();
  write_out(a, a.U, obj, base, dims, cluster);
  for (int k = d - 1; k >= 1; --k) qr_step(a, base, dims, k, 0, s, cluster);
  __threadfence();
  write_out(a, a.V, obj, base, dims, cluster);
}

static long long orth_obj_stride(const TTV& X, long long* coff, int* R1) {
  long long o = 0;
  for (int k = 0; k < X.d; ++k) {
    if (coff) coff[k] = o;
    if (R1) R1[k] = X.r[k + 1];
    o += X.osz[k];
  }
  return (o + 31) & ~31LL;
}

static size_t orth_smem(int rows_per) {
  return sizeof(double) * ((size_t)rows_per * T3F_MAX_RANK + T3F_MAX_RANK * T3F_MAX_RANK + 7 * T3F_MAX_RANK + rows_per + 4);
}

// Largest supported cluster size (16 if allowed, else 8), cached per process.
static int orth_cluster_size(size_t* smem_out) {
  static int P = -1;
  static size_t smem = 0;
  if (P >= 0) {
    *smem_out = smem;
    return P;
  }
  P = 0;
  for (int cand : {16, 8}) {
    const int rows_per = (kOrthMaxRows + cand - 1) / cand;
    const size_t sm = orth_smem(rows_per);
    if (cudaFuncSetAttribute(k_orth, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (cand > 8 && cudaFuncSetAttribute(k_orth, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cand;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cand);
    cfg.blockDim = dim3(kOrthThreads);
    cfg.dynamicSmemBytes = sm;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_orth, &cfg) == cudaSuccess && nclusters > 0) {
      P = cand;
      smem = sm;
      break;
    }
    cudaGetLastError();
  }
  *smem_out = smem;
  return P;
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
  size_t smem = 0;
  const int P = orth_cluster_size(&smem);
  if (P == 0) return T3F_ERR_UNSUPPORTED;
  OrthArgs args;
  memset(&args, 0, sizeof(args));
  args.X = vx;
  args.U = vu;
  args.V = vv;
  args.P = P;
  args.rows_per = (kOrthMaxRows + P - 1) / P;
  args.work = reinterpret_cast<double*>(static_cast<char*>(ws) + kWsHeader);
  args.obj_stride = orth_obj_stride(vx, args.coff, args.R1);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = P;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)(P * vx.batch));
  cfg.blockDim = dim3(kOrthThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = (cudaStream_t)stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k_orth, args) != cudaSuccess) {
    cudaGetLastError();
    return T3F_ERR_CUDA;
  }
  return launch_status();
}
