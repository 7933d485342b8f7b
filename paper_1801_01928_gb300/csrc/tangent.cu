// Operations on one tangent space T_X of the fixed-rank TT manifold (paper Section 3.2):
// the per-object projection ('project' of Table 1 applied to every object of a batch), the
// Gram matrix of tangent vectors of one tangent space, the projection of a matrix-by-vector
// product P_X(A c) without forming the rank r_A r_c product, and the linearised Riemannian
// Hessian of the completion loss applied to a tangent vector.
//
// X is given by its orthogonal forms U (left-orthogonal U_1..U_{d-1}) and V (right-orthogonal
// V_2..V_d). A tangent vector is given by gauge coordinates dU (U's shape, U_k^T dU_k = 0 on
// the left unfoldings for k < d); its full tensor is sum_k U_1..U_{k-1} dU_k V_{k+1}..V_d.
// Interfaces are numbered 0..d; core k sits between interfaces k and k+1.
#include <string.h>

#include <algorithm>

#include "t3f_internal.cuh"

namespace t3f {

namespace {

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------------------
// Batched gauge projection, in place: D_j,k <- D_j,k - U_k (U_k^T D_j,k) on the
// (r_{k-1} n_k) x r_k unfoldings, k < d. One CTA per (object j, core k), staged in shared
// memory (gauge_core_staged) when the largest core fits.
// ---------------------------------------------------------------------------------------
struct GaugeBatchArgs {
  TTV U;     // batch 1
  TTV D;     // batch P, U's shape (coordinates, modified in place)
  int staged;
};

__global__ void __launch_bounds__(kThreads) k_gauge_batch(const __grid_constant__ GaugeBatchArgs a) {
  extern __shared__ __align__(16) float G[];  // r1 x r1, or the staged buffers
  const int dm1 = a.U.d - 1;
  const int k = blockIdx.x % dm1, j = blockIdx.x / dm1;
  const int r0 = a.U.r[k], n = a.U.n[k], r1 = a.U.r[k + 1];
  const int m = r0 * n;
  const float* Uk = static_cast<const float*>(a.U.p) + a.U.off[k];
  float* Dk = static_cast<float*>(a.D.p) + core_base(a.D, k, j);
  if (a.staged) {
    gauge_core_staged(Uk, Dk, Dk, m, r1, G);
    return;
  }
  for (int e = threadIdx.x; e < r1 * r1; e += blockDim.x) {
    const int p = e / r1, q = e % r1;
    float s = 0.0f;
    for (int row = 0; row < m; ++row) s = fmaf(__ldg(Uk + row * r1 + p), Dk[row * r1 + q], s);
    G[e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < m * r1; e += blockDim.x) {
    const int row = e / r1, q = e % r1;
    float s = Dk[e];
    for (int p = 0; p < r1; ++p) s = fmaf(-__ldg(Uk + row * r1 + p), G[p * r1 + q], s);
    Dk[e] = s;
  }
}

t3f_status gauge_batch(const TTV& U, const TTV& D, cudaStream_t s) {
  if (U.d < 2) return T3F_OK;
  GaugeBatchArgs a;
  a.U = U;
  a.D = D;
  long long full = 0;
  for (int k = 0; k + 1 < U.d; ++k) full = std::max(full, gauge_staged_floats(U.r[k] * U.n[k], U.r[k + 1]));
  const size_t base = sizeof(float) * U.rmax * U.rmax;
  a.staged = sizeof(float) * (size_t)full <= 200 * 1024 ? 1 : 0;
  const size_t smem = a.staged ? std::max(sizeof(float) * (size_t)full, base) : base;
  if (cudaFuncSetAttribute(k_gauge_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return T3F_ERR_CUDA;
  const long long grid = (long long)(U.d - 1) * D.batch;
  if (grid > 0x7fffffffLL) return T3F_ERR_UNSUPPORTED;
  k_gauge_batch<<<(unsigned)grid, kThreads, smem, s>>>(a);
  return launch_status();
}

// ---------------------------------------------------------------------------------------
// Per-object assembly of the projection: Zhat_j,k[:, i, :] = c_j L_j,k Z_j,k[:, i, :] R_j,k+1^T
// with L, R the left partials of (U, Z_j) and right partials of (V, Z_j) at interfaces k and
// k+1 ([r^U][r^Z] per object). One CTA per (object j, core k).
// ---------------------------------------------------------------------------------------
struct AssembleBatchArgs {
  TTV U, Z, D;                    // D: output coordinates (batch = Z.batch, U's shape)
  const float* L;
  const float* R;
  long long ioff[T3F_MAX_D + 1];  // partial offsets (same for L and R)
  const float* c;                 // nullable: weights
  int RU, RZ;
};

__global__ void __launch_bounds__(kThreads) k_assemble_batch(const __grid_constant__ AssembleBatchArgs a) {
  extern __shared__ float sm[];
  const int d = a.U.d;
  const int k = blockIdx.x % d, j = blockIdx.x / d;
  const int r0 = a.U.r[k], r1 = a.U.r[k + 1], s0 = a.Z.r[k], s1 = a.Z.r[k + 1], n = a.U.n[k];
  float* Ls = sm;                   // r0 x s0
  float* Rs = Ls + a.RU * a.RZ;     // r1 x s1
  float* Zs = Rs + a.RU * a.RZ;     // s0 x s1 (slice i)
  float* Ys = Zs + a.RZ * a.RZ;     // s0 x r1
  const float cj = a.c ? a.c[j] : 1.0f;
  for (int e = threadIdx.x; e < r0 * s0; e += blockDim.x) Ls[e] = a.L[a.ioff[k] + (long long)j * r0 * s0 + e];
  for (int e = threadIdx.x; e < r1 * s1; e += blockDim.x) Rs[e] = a.R[a.ioff[k + 1] + (long long)j * r1 * s1 + e];
  const float* Zp = static_cast<const float*>(a.Z.p) + core_base(a.Z, k, j);
  float* out = static_cast<float*>(a.D.p) + core_base(a.D, k, j);
  for (int i = 0; i < n; ++i) {
    __syncthreads();
    for (int e = threadIdx.x; e < s0 * s1; e += blockDim.x) {
      const int g = e / s1, h = e % s1;
      Zs[e] = __ldg(Zp + ((long long)g * n + i) * s1 + h);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < s0 * r1; e += blockDim.x) {  // Y = Z_i R^T
      const int g = e / r1, b = e % r1;
      float s = 0.0f;
      for (int h = 0; h < s1; ++h) s = fmaf(Zs[g * s1 + h], Rs[b * s1 + h], s);
      Ys[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < r0 * r1; e += blockDim.x) {  // Zhat_i = c L Y
      const int al = e / r1, b = e % r1;
      float s = 0.0f;
      for (int g = 0; g < s0; ++g) s = fmaf(Ls[al * s0 + g], Ys[g * r1 + b], s);
      out[((long long)al * n + i) * r1 + b] = cj * s;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Gather of a tangent vector at index tuples: xi(i) = q_d with the block recurrence
// q_k = q_{k-1} V_k[:, i_k, :] + p_{k-1} dU_k[:, i_k, :], p_k = p_{k-1} U_k[:, i_k, :],
// p_0 = 1, q_0 = 0 (the row vector [q, p] through the rank-2r cores [[V, 0], [dU, U]]).
// Cores are staged in shared memory as zero-padded R x R slices.
// ---------------------------------------------------------------------------------------
struct TGatherArgs {
  int d, nmax;
  long long N;
  int n[T3F_MAX_D];
  int r[T3F_MAX_D + 1];
  const float* U;
  const float* V;
  const float* W;                 // coordinates
  long long off[T3F_MAX_D];       // packed offsets (batch 1), shared by U, V, W
  const int* idx;                 // [d][N]
  float* out;                     // [N]
  int* err;
};

template <int R>
__device__ void stage_slices(float* dst, const float* src, const TGatherArgs& g) {
  constexpr int SS = R * R + 4;  // slice stride: consecutive slices start 4 banks apart
  const int total = g.d * g.nmax * R * R;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int b = e % R, a = (e / R) % R, i = (e / (R * R)) % g.nmax, k = e / (R * R * g.nmax);
    float v = 0.0f;
    if (i < g.n[k] && a < g.r[k] && b < g.r[k + 1]) v = __ldg(src + g.off[k] + ((long long)a * g.n[k] + i) * g.r[k + 1] + b);
    dst[(k * g.nmax + i) * SS + a * R + b] = v;
  }
}

template <int R>
__global__ void __launch_bounds__(256) k_tangent_gather(const __grid_constant__ TGatherArgs g) {
  extern __shared__ __align__(16) float sm[];
  // the tuples of a warp read slices at random indices: a slice stride of R^2 + 4 floats
  // spreads the same offset of different slices over distinct banks
  constexpr int SS = R * R + 4;
  const int SL = g.d * g.nmax * SS;
  float* Us = sm;
  float* Vs = sm + SL;
  float* Ws = sm + 2 * SL;
  stage_slices<R>(Us, g.U, g);
  stage_slices<R>(Vs, g.V, g);
  stage_slices<R>(Ws, g.W, g);
  __syncthreads();
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < g.N; t += (long long)gridDim.x * blockDim.x) {
    float p[R], q[R];
#pragma unroll
    for (int a = 0; a < R; ++a) {
      p[a] = a == 0 ? 1.0f : 0.0f;
      q[a] = 0.0f;
    }
    for (int k = 0; k < g.d; ++k) {
      int i = __ldg(g.idx + (long long)k * g.N + t);
      if (i < 0 || i >= g.n[k]) {
        atomicExch(g.err, (int)T3F_ERR_ARG);
        i = i < 0 ? 0 : g.n[k] - 1;
      }
      const int so = (k * g.nmax + i) * SS;
      float np[R], nq[R];
#pragma unroll
      for (int b = 0; b < R; ++b) np[b] = nq[b] = 0.0f;
#pragma unroll
      for (int a = 0; a < R; ++a) {
#pragma unroll
        for (int b = 0; b < R; b += 4) {
          const float4 u4 = *reinterpret_cast<const float4*>(Us + so + a * R + b);
          const float4 v4 = *reinterpret_cast<const float4*>(Vs + so + a * R + b);
          const float4 w4 = *reinterpret_cast<const float4*>(Ws + so + a * R + b);
          np[b] = fmaf(p[a], u4.x, np[b]);
          np[b + 1] = fmaf(p[a], u4.y, np[b + 1]);
          np[b + 2] = fmaf(p[a], u4.z, np[b + 2]);
          np[b + 3] = fmaf(p[a], u4.w, np[b + 3]);
          nq[b] = fmaf(q[a], v4.x, fmaf(p[a], w4.x, nq[b]));
          nq[b + 1] = fmaf(q[a], v4.y, fmaf(p[a], w4.y, nq[b + 1]));
          nq[b + 2] = fmaf(q[a], v4.z, fmaf(p[a], w4.z, nq[b + 2]));
          nq[b + 3] = fmaf(q[a], v4.w, fmaf(p[a], w4.w, nq[b + 3]));
        }
      }
#pragma unroll
      for (int b = 0; b < R; ++b) {
        p[b] = np[b];
        q[b] = nq[b];
      }
    }
    g.out[t] = q[0];
  }
}

// ---------------------------------------------------------------------------------------
// Gram matrix of tangent vectors (FP32 CUDA cores): G[a][b] = sum_k <dA_a,k, dB_b,k>, a
// split-K product over the concatenated coordinates. A CTA owns a 128 x 128 tile of pairs and
// a range of 16-column chunks (a chunk never crosses a core or a split; columns past a core's
// end are zero); 256 threads hold 8 x 8 accumulators each (rows ty*4 + {0..3} and
// 64 + ty*4 + {0..3}, columns likewise with tx), fed by float4 loads from transposed,
// double-buffered operand tiles. On a diagonal tile of a self Gram matrix one operand is
// staged. The CTA's partial goes to part[split][a][b]; the splits are summed in a fixed order.
// ---------------------------------------------------------------------------------------
constexpr int kTM = 128, kKC = 16, kLD = kTM + 4;

struct TGramArgs {
  TTV A, B;
  long long ksz[T3F_MAX_D];  // coordinates of core k per object
  long long nchunks, cper;   // 16-column chunks in all, per split
  int nsplit, tilesB, self;
  float* part;               // [nsplit][A.batch][B.batch]
};

// chunk c of the concatenated coordinates -> (core k, column of the core)
__device__ __forceinline__ void tg_chunk(const TGramArgs& g, long long c, int* k, long long* col) {
  long long first = 0;
  int kk = 0;
  for (; kk < g.A.d; ++kk) {
    const long long nk = (g.ksz[kk] + kKC - 1) / kKC;
    if (c < first + nk) break;
    first += nk;
  }
  *k = kk;
  *col = (c - first) * kKC;
}

__global__ void __launch_bounds__(kThreads, 2) k_tgram(const __grid_constant__ TGramArgs g) {
  __shared__ __align__(16) float As[2][kKC][kLD];
  __shared__ __align__(16) float Bs[2][kKC][kLD];
  const int split = blockIdx.x % g.nsplit;
  const int tile = blockIdx.x / g.nsplit;
  const int a0 = (tile / g.tilesB) * kTM, b0 = (tile % g.tilesB) * kTM;
  const bool one = g.self && a0 == b0;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const long long c0 = (long long)split * g.cper, c1 = min(g.nchunks, c0 + g.cper);
  const float* Ap = static_cast<const float*>(g.A.p);
  const float* Bp = static_cast<const float*>(g.B.p);
  float acc[8][8];
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int v = 0; v < 8; ++v) acc[u][v] = 0.0f;
  // staging: thread t loads rows t / 4 and 64 + t / 4, columns 4 (t % 4) .. + 3 of a chunk
  const int lr = tid >> 2, lq = (tid & 3) * 4;
  float4 ra[2], rb[2];
  auto load = [&](long long c) {
    int k;
    long long col;
    tg_chunk(g, c, &k, &col);
    const long long sz = g.ksz[k];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = lr + 64 * h;
      float va[4] = {0.0f, 0.0f, 0.0f, 0.0f}, vb[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long cc = col + lq + u;
        if (cc < sz) {
          if (a0 + r < g.A.batch) va[u] = __ldg(Ap + g.A.off[k] + (long long)(a0 + r) * sz + cc);
          if (!one && b0 + r < g.B.batch) vb[u] = __ldg(Bp + g.B.off[k] + (long long)(b0 + r) * sz + cc);
        }
      }
      ra[h] = make_float4(va[0], va[1], va[2], va[3]);
      rb[h] = make_float4(vb[0], vb[1], vb[2], vb[3]);
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = lr + 64 * h;
      As[buf][lq + 0][r] = ra[h].x;
      As[buf][lq + 1][r] = ra[h].y;
      As[buf][lq + 2][r] = ra[h].z;
      As[buf][lq + 3][r] = ra[h].w;
      if (!one) {
        Bs[buf][lq + 0][r] = rb[h].x;
        Bs[buf][lq + 1][r] = rb[h].y;
        Bs[buf][lq + 2][r] = rb[h].z;
        Bs[buf][lq + 3][r] = rb[h].w;
      }
    }
  };
  if (c0 < c1) {
    load(c0);
    store(0);
  }
  __syncthreads();
  for (long long c = c0; c < c1; ++c) {
    const int buf = (int)((c - c0) & 1);
    if (c + 1 < c1) load(c + 1);  // in flight during the products
    const float(*Ab)[kLD] = As[buf];
    const float(*Bb)[kLD] = one ? As[buf] : Bs[buf];
#pragma unroll
    for (int kk = 0; kk < kKC; ++kk) {
      const float4 a_lo = *reinterpret_cast<const float4*>(&Ab[kk][ty * 4]);
      const float4 a_hi = *reinterpret_cast<const float4*>(&Ab[kk][64 + ty * 4]);
      const float4 b_lo = *reinterpret_cast<const float4*>(&Bb[kk][tx * 4]);
      const float4 b_hi = *reinterpret_cast<const float4*>(&Bb[kk][64 + tx * 4]);
      const float av[8] = {a_lo.x, a_lo.y, a_lo.z, a_lo.w, a_hi.x, a_hi.y, a_hi.z, a_hi.w};
      const float bv[8] = {b_lo.x, b_lo.y, b_lo.z, b_lo.w, b_hi.x, b_hi.y, b_hi.z, b_hi.w};
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
    }
    if (c + 1 < c1) store(buf ^ 1);
    __syncthreads();
  }
  float* P = g.part + (long long)split * g.A.batch * g.B.batch;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int a = a0 + (u < 4 ? ty * 4 + u : 64 + ty * 4 + u - 4);
    if (a >= g.A.batch) continue;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const int b = b0 + (v < 4 ? tx * 4 + v : 64 + tx * 4 + v - 4);
      if (b < g.B.batch) P[(long long)a * g.B.batch + b] = acc[u][v];
    }
  }
}

// Sum of split partials in a fixed order, in two levels so that every SM takes part:
// level 1 sums the splits g, g + G1, g + 2 G1, ... of each element into mid[g] (grid
// elements / 256 x G1), level 2 sums the G1 groups.
constexpr int kReduceGroups = 16;

__global__ void k_split_reduce1(const float* part, int nsplit, long long size, float* mid) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int g = blockIdx.y, G1 = gridDim.y;
  if (e >= size) return;
  float s = 0.0f;
#pragma unroll 4
  for (int p = g; p < nsplit; p += G1) s += __ldg(part + (long long)p * size + e);
  mid[(long long)g * size + e] = s;
}

__global__ void k_split_reduce2(const float* mid, int groups, long long size, float* G) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < size; e += (long long)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int g = 0; g < groups; ++g) s += mid[(long long)g * size + e];
    G[e] = s;
  }
}

// SM count of the current device (looked up once per device index).
int dev_sms() {
  static int cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 152;
  }
  if (cache[dev] <= 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      return 152;
    }
    cache[dev] = v;
  }
  return cache[dev];
}

struct TGramPlan {
  int tilesA, tilesB, nsplit;
  long long nchunks, cper;
  size_t part_off, mid_off, total;
};

TGramPlan tgram_plan(const TTV& A, const TTV& B) {
  TGramPlan p;
  p.nchunks = 0;
  for (int k = 0; k < A.d; ++k) p.nchunks += (A.osz[k] + kKC - 1) / kKC;
  p.tilesA = (A.batch + kTM - 1) / kTM;
  p.tilesB = (B.batch + kTM - 1) / kTM;
  const long long tiles = (long long)p.tilesA * p.tilesB;
  long long ns = ((long long)dev_sms() * 2 + tiles - 1) / tiles;  // two CTAs per SM in all
  ns = std::min(ns, (p.nchunks + 7) / 8);                          // at least 8 chunks per split
  ns = std::max(ns, 1LL);
  p.cper = (p.nchunks + ns - 1) / ns;
  p.nsplit = (int)((p.nchunks + p.cper - 1) / p.cper);
  p.part_off = kWsHeader;
  p.mid_off = p.part_off + align256(sizeof(float) * (size_t)p.nsplit * A.batch * B.batch);
  p.total = p.mid_off + align256(sizeof(float) * (size_t)kReduceGroups * A.batch * B.batch);
  return p;
}

// ---------------------------------------------------------------------------------------
// Projected matrix-by-vector product P_X(A c_j): the left partials L_k (U against the
// rank r_A r_c product, [r^U][r^A][r^c]) and the right partials R_k (V against it) are swept
// with the Kronecker structure of the product cores
//   C_k[(a, b), i, (a', b')] = sum_j A_k[a, i, j, a'] c_k[b, j, b'],
// never forming C. One CTA per object and direction; then one CTA per (object, core) for
// Zhat_k = L_k C_k R_{k+1}^T, and the batched gauge.
// ---------------------------------------------------------------------------------------
struct PmvArgs {
  TTV X;                          // U (dir 0, assembly) or V (dir 1)
  TTV A;                          // TT-matrix, batch 1 or P
  TTV c;                          // TT-vectors, batch P
  TTV D;                          // assembly output (batch P, U's shape)
  float* L;                       // left partials store
  float* R;                       // right partials store
  long long ioff[T3F_MAX_D + 1];  // per interface: P * rX rA rc
  int dir;
};

// T1[x][a][j][b'] = sum_b S[x][a][b] c[b][j][b']    (x < rx, a < ra, b < rb0, b' < rb1, j < nn)
__device__ void pmv_c_step(const float* S, const float* cp, float* T1, int rx, int ra, int rb0, int nn, int rb1) {
  const int tot = rx * ra * nn * rb1;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int bp = e % rb1, j = (e / rb1) % nn, xa = e / (rb1 * nn);
    const float* s = S + (long long)xa * rb0;
    float acc = 0.0f;
    for (int b = 0; b < rb0; ++b) acc = fmaf(s[b], __ldg(cp + ((long long)b * nn + j) * rb1 + bp), acc);
    T1[e] = acc;
  }
}

__global__ void __launch_bounds__(kThreads) k_pmv_sweep(const __grid_constant__ PmvArgs g) {
  extern __shared__ float sm[];
  const int obj = blockIdx.x;
  const int d = g.X.d;
  const int aobj = g.A.batch == 1 ? 0 : obj;
  const float* Xp = static_cast<const float*>(g.X.p);
  const float* Ap = static_cast<const float*>(g.A.p);
  const float* Cp = static_cast<const float*>(g.c.p);
  int maxS = 1;
  for (int k = 0; k <= d; ++k) maxS = max(maxS, g.X.r[k] * g.A.r[k] * g.c.r[k]);
  // shared memory (sized by the host): S (current partial), T1, T2 after T1's maximum
  float* S = sm;
  float* T1 = S + maxS;
  int maxT1 = 1;
  for (int k = 0; k < d; ++k) {
    const int t1 = g.dir == 0 ? g.X.r[k] * g.A.r[k] * g.c.n[k] * g.c.r[k + 1]
                              : g.X.r[k + 1] * g.A.r[k + 1] * g.c.n[k] * g.c.r[k];
    maxT1 = max(maxT1, t1);
  }
  float* T2 = T1 + maxT1;
  float* store = g.dir == 0 ? g.L : g.R;
  if (g.dir == 0) {
    if (threadIdx.x == 0) S[0] = 1.0f;
    if (threadIdx.x == 0) store[g.ioff[0] + obj] = 1.0f;
    for (int k = 0; k < d; ++k) {
      const int x0 = g.X.r[k], x1 = g.X.r[k + 1], a0 = g.A.r[k], a1 = g.A.r[k + 1];
      const int b0 = g.c.r[k], b1 = g.c.r[k + 1], m = g.A.m[k], nn = g.A.n[k];
      const float* cp = Cp + core_base(g.c, k, obj);
      const float* ap = Ap + core_base(g.A, k, aobj);
      const float* xp = Xp + g.X.off[k];
      __syncthreads();
      pmv_c_step(S, cp, T1, x0, a0, b0, nn, b1);  // T1[x][a][j][b']
      __syncthreads();
      // T2[x][i][a'][b'] = sum_{a, j} T1[x][a][j][b'] A[a][i][j][a']
      const int t2 = x0 * m * a1 * b1;
      for (int e = threadIdx.x; e < t2; e += blockDim.x) {
        const int bp = e % b1, ap_ = (e / b1) % a1, i = (e / (b1 * a1)) % m, x = e / (b1 * a1 * m);
        float acc = 0.0f;
        for (int a = 0; a < a0; ++a)
          for (int j = 0; j < nn; ++j)
            acc = fmaf(T1[((x * a0 + a) * nn + j) * b1 + bp], __ldg(ap + (((long long)a * m + i) * nn + j) * a1 + ap_), acc);
        T2[e] = acc;
      }
      __syncthreads();
      // S'[x'][a'][b'] = sum_{x, i} U[x][i][x'] T2[x][i][a'][b']
      const int sn = x1 * a1 * b1;
      float* out = store + g.ioff[k + 1] + (long long)obj * sn;
      for (int e = threadIdx.x; e < sn; e += blockDim.x) {
        const int ab = e % (a1 * b1), xp_ = e / (a1 * b1);
        float acc = 0.0f;
        for (int x = 0; x < x0; ++x)
          for (int i = 0; i < m; ++i) acc = fmaf(__ldg(xp + ((long long)x * m + i) * x1 + xp_), T2[(x * m + i) * a1 * b1 + ab], acc);
        out[e] = acc;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < sn; e += blockDim.x) S[e] = out[e];
    }
  } else {
    if (threadIdx.x == 0) S[0] = 1.0f;
    if (threadIdx.x == 0) store[g.ioff[d] + obj] = 1.0f;
    for (int k = d - 1; k >= 0; --k) {
      const int x0 = g.X.r[k], x1 = g.X.r[k + 1], a0 = g.A.r[k], a1 = g.A.r[k + 1];
      const int b0 = g.c.r[k], b1 = g.c.r[k + 1], m = g.A.m[k], nn = g.A.n[k];
      const float* cp = Cp + core_base(g.c, k, obj);
      const float* ap = Ap + core_base(g.A, k, aobj);
      const float* xp = Xp + g.X.off[k];
      __syncthreads();
      // T1[x'][a'][j][b] = sum_{b'} S[x'][a'][b'] c[b][j][b']
      const int t1 = x1 * a1 * nn * b0;
      for (int e = threadIdx.x; e < t1; e += blockDim.x) {
        const int b = e % b0, j = (e / b0) % nn, xa = e / (b0 * nn);
        const float* s = S + (long long)xa * b1;
        float acc = 0.0f;
        for (int bp = 0; bp < b1; ++bp) acc = fmaf(s[bp], __ldg(cp + ((long long)b * nn + j) * b1 + bp), acc);
        T1[e] = acc;
      }
      __syncthreads();
      // T2[x'][i][a][b] = sum_{a', j} T1[x'][a'][j][b] A[a][i][j][a']
      const int t2 = x1 * m * a0 * b0;
      for (int e = threadIdx.x; e < t2; e += blockDim.x) {
        const int b = e % b0, a = (e / b0) % a0, i = (e / (b0 * a0)) % m, x = e / (b0 * a0 * m);
        float acc = 0.0f;
        for (int ap_ = 0; ap_ < a1; ++ap_)
          for (int j = 0; j < nn; ++j)
            acc = fmaf(T1[((x * a1 + ap_) * nn + j) * b0 + b], __ldg(ap + (((long long)a * m + i) * nn + j) * a1 + ap_), acc);
        T2[e] = acc;
      }
      __syncthreads();
      // S'[x][a][b] = sum_{x', i} V[x][i][x'] T2[x'][i][a][b]
      const int sn = x0 * a0 * b0;
      float* out = store + g.ioff[k] + (long long)obj * sn;
      for (int e = threadIdx.x; e < sn; e += blockDim.x) {
        const int ab = e % (a0 * b0), x = e / (a0 * b0);
        float acc = 0.0f;
        for (int xq = 0; xq < x1; ++xq)
          for (int i = 0; i < m; ++i) acc = fmaf(__ldg(xp + ((long long)x * m + i) * x1 + xq), T2[(xq * m + i) * a0 * b0 + ab], acc);
        out[e] = acc;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < sn; e += blockDim.x) S[e] = out[e];
    }
  }
}

// Zhat_k[x][i][x'] = sum_{a', b'} T2[x][i][a'][b'] R_{k+1}[x'][a'][b'], with T2 built from
// L_k as in the left sweep. One CTA per (object, core).
__global__ void __launch_bounds__(kThreads) k_pmv_assemble(const __grid_constant__ PmvArgs g) {
  extern __shared__ float sm[];
  const int d = g.X.d;
  const int k = blockIdx.x % d, obj = blockIdx.x / d;
  const int aobj = g.A.batch == 1 ? 0 : obj;
  const int x0 = g.X.r[k], x1 = g.X.r[k + 1], a0 = g.A.r[k], a1 = g.A.r[k + 1];
  const int b0 = g.c.r[k], b1 = g.c.r[k + 1], m = g.A.m[k], nn = g.A.n[k];
  const float* cp = static_cast<const float*>(g.c.p) + core_base(g.c, k, obj);
  const float* ap = static_cast<const float*>(g.A.p) + core_base(g.A, k, aobj);
  const float* Lk = g.L + g.ioff[k] + (long long)obj * x0 * a0 * b0;
  const float* Rk = g.R + g.ioff[k + 1] + (long long)obj * x1 * a1 * b1;
  float* T1 = sm;                        // x0 a0 nn b1
  float* T2 = T1 + x0 * a0 * nn * b1;    // x0 m a1 b1
  pmv_c_step(Lk, cp, T1, x0, a0, b0, nn, b1);
  __syncthreads();
  const int t2 = x0 * m * a1 * b1;
  for (int e = threadIdx.x; e < t2; e += blockDim.x) {
    const int bp = e % b1, ap_ = (e / b1) % a1, i = (e / (b1 * a1)) % m, x = e / (b1 * a1 * m);
    float acc = 0.0f;
    for (int a = 0; a < a0; ++a)
      for (int j = 0; j < nn; ++j)
        acc = fmaf(T1[((x * a0 + a) * nn + j) * b1 + bp], __ldg(ap + (((long long)a * m + i) * nn + j) * a1 + ap_), acc);
    T2[e] = acc;
  }
  __syncthreads();
  float* out = static_cast<float*>(g.D.p) + core_base(g.D, k, obj);
  const int ab = a1 * b1;
  for (int e = threadIdx.x; e < x0 * m * x1; e += blockDim.x) {
    const int xq = e % x1, xi = e / x1;  // xi = x * m + i
    float acc = 0.0f;
    for (int q = 0; q < ab; ++q) acc = fmaf(T2[xi * ab + q], Rk[(long long)xq * ab + q], acc);
    out[e] = acc;
  }
}

struct PmvPlan {
  long long ioff[T3F_MAX_D + 1];
  size_t offL, offR, total;
  size_t smem_sweep[2], smem_asm;
};

bool pmv_plan(const TTV& U, const TTV& A, const TTV& c, PmvPlan* p) {
  long long o = 0;
  int maxS = 1;
  for (int k = 0; k <= U.d; ++k) {
    p->ioff[k] = o;
    const long long s = (long long)U.r[k] * A.r[k] * c.r[k];
    o += s * c.batch;
    maxS = std::max(maxS, (int)s);
  }
  p->offL = kWsHeader;
  p->offR = p->offL + align256(sizeof(float) * o);
  p->total = p->offR + align256(sizeof(float) * o);
  long long t1l = 1, t1r = 1, t2l = 1, t2r = 1, asmx = 1;
  for (int k = 0; k < U.d; ++k) {
    const long long x0 = U.r[k], x1 = U.r[k + 1], a0 = A.r[k], a1 = A.r[k + 1], b0 = c.r[k], b1 = c.r[k + 1];
    const long long m = A.m[k], nn = A.n[k];
    t1l = std::max(t1l, x0 * a0 * nn * b1);
    t2l = std::max(t2l, x0 * m * a1 * b1);
    t1r = std::max(t1r, x1 * a1 * nn * b0);
    t2r = std::max(t2r, x1 * m * a0 * b0);
    asmx = std::max(asmx, x0 * a0 * nn * b1 + x0 * m * a1 * b1);
  }
  p->smem_sweep[0] = sizeof(float) * (size_t)(maxS + t1l + t2l);
  p->smem_sweep[1] = sizeof(float) * (size_t)(maxS + t1r + t2r);
  p->smem_asm = sizeof(float) * (size_t)asmx;
  const size_t cap = 200 * 1024;
  return p->smem_sweep[0] <= cap && p->smem_sweep[1] <= cap && p->smem_asm <= cap;
}

// Common view checks: U, V orthogonal forms (batch 1, equal ranks and modes); D like U.
t3f_status uv_views(const t3f_tt* U, const t3f_tt* V, TTV* vu, TTV* vv) {
  T3F_CHECK(make_view(U, vu, T3F_F32, false));
  T3F_CHECK(make_view(V, vv, T3F_F32, false));
  if (vu->batch != 1 || vv->batch != 1 || vu->d != vv->d) return T3F_ERR_SHAPE;
  for (int k = 0; k <= vu->d; ++k) {
    if (vu->r[k] != vv->r[k]) return T3F_ERR_SHAPE;
    if (k < vu->d && vu->n[k] != vv->n[k]) return T3F_ERR_SHAPE;
  }
  if (vu->rmax > T3F_MAX_RANK) return T3F_ERR_UNSUPPORTED;
  return T3F_OK;
}

t3f_status coords_view(const t3f_tt* t, const TTV& U, int batch, TTV* v) {
  T3F_CHECK(make_view(t, v, T3F_F32, false));
  if ((batch > 0 && v->batch != batch) || v->d != U.d) return T3F_ERR_SHAPE;
  for (int k = 0; k <= U.d; ++k)
    if (v->r[k] != U.r[k] || (k < U.d && v->n[k] != U.n[k])) return T3F_ERR_SHAPE;
  return T3F_OK;
}

struct ProjectLayout {
  long long ioff[T3F_MAX_D + 1];
  size_t offL, offR, offXT, total;
};

ProjectLayout project_layout(const TTV& U, const TTV& Z) {
  ProjectLayout l;
  const long long nL = partial_offsets(U, Z, Z.batch, l.ioff);
  l.offL = kWsHeader;
  l.offR = l.offL + align256(sizeof(float) * nL);
  l.offXT = l.offR + align256(sizeof(float) * nL);  // transposed V for the right sweep
  l.total = l.offXT + align256(sizeof(float) * xtranspose_offsets(U, nullptr));
  return l;
}

}  // namespace

t3f_status run_split_reduce(const float* part, int nsplit, long long size, float* mid, float* G, cudaStream_t s) {
  const int G1 = std::min(nsplit, kReduceGroups);
  const long long bx = (size + 255) / 256;
  if (bx > 0x7fffffffLL) return T3F_ERR_UNSUPPORTED;
  k_split_reduce1<<<dim3((unsigned)bx, (unsigned)G1), 256, 0, s>>>(part, nsplit, size, mid);
  T3F_CHECK(launch_status());
  k_split_reduce2<<<(unsigned)std::min<long long>(std::max<long long>(bx, 1), 1024), 256, 0, s>>>(mid, G1, size, G);
  return launch_status();
}

size_t ws_split_reduce(long long size) { return align256(sizeof(float) * (size_t)kReduceGroups * size); }

size_t ws_project(const TTV& U, const TTV& Z) { return project_layout(U, Z).total; }
size_t ws_tangent_gram(const TTV& A, const TTV& B) {
  return std::max(tgram_plan(A, B).total, ws_tangent_gram_tc(A, B));
}
size_t ws_completion_hvp(const TTV& U, const TTV& V, long long N) {
  return align256(ws_rgather(U, V, N)) + align256(sizeof(float) * (size_t)std::max(N, 1LL));
}

}  // namespace t3f

using namespace t3f;

extern "C" t3f_status t3f_project(const t3f_tt* U, const t3f_tt* V, const t3f_tt* Z, const float* c,
                                  t3f_tt* dU, void* ws, size_t ws_bytes, t3f_stream_t stream) {
  TTV vu, vv, vz, vd;
  T3F_CHECK(uv_views(U, V, &vu, &vv));
  T3F_CHECK(make_view(Z, &vz, T3F_F32, false));
  if (vz.d != vu.d) return T3F_ERR_SHAPE;
  for (int k = 0; k < vu.d; ++k)
    if (vz.n[k] != vu.n[k]) return T3F_ERR_SHAPE;
  if (vz.rmax > T3F_MAX_RANK) return T3F_ERR_UNSUPPORTED;
  T3F_CHECK(coords_view(dU, vu, vz.batch, &vd));
  const ProjectLayout l = project_layout(vu, vz);
  T3F_CHECK(check_ws(ws, ws_bytes, l.total));
  cudaStream_t s = (cudaStream_t)stream;
  char* w = static_cast<char*>(ws);
  float* Lst = reinterpret_cast<float*>(w + l.offL);
  float* Rst = reinterpret_cast<float*>(w + l.offR);
  if (psweep_supported(vu, vz)) {
    T3F_CHECK(run_psweep(vu, vz, 0, static_cast<const float*>(vu.p), nullptr, nullptr, Lst, nullptr, l.ioff, s));
    // the right sweep stages its slices from a transposed copy of V (16-byte copies)
    float* VT = reinterpret_cast<float*>(w + l.offXT);
    long long toff[T3F_MAX_D];
    xtranspose_offsets(vv, toff);
    const float* vsrc[1] = {static_cast<const float*>(vv.p)};
    T3F_CHECK(run_xtranspose(vv, vsrc, 1, VT, s));
    T3F_CHECK(run_psweep(vv, vz, 1, VT, nullptr, nullptr, Rst, nullptr, l.ioff, s, nullptr, toff));
  } else {
    T3F_CHECK(run_pair_sweep(vu, vz, 0, nullptr, Lst, l.ioff, s));
    T3F_CHECK(run_pair_sweep(vv, vz, 1, nullptr, Rst, l.ioff, s));
  }
  AssembleBatchArgs a;
  memset(&a, 0, sizeof(a));
  a.U = vu;
  a.Z = vz;
  a.D = vd;
  a.L = Lst;
  a.R = Rst;
  for (int j = 0; j <= vu.d; ++j) a.ioff[j] = l.ioff[j];
  a.c = c;
  a.RU = vu.rmax;
  a.RZ = vz.rmax;
  const size_t smem = sizeof(float) * (2 * (size_t)a.RU * a.RZ + 2 * (size_t)a.RZ * std::max(a.RZ, a.RU));
  const long long grid = (long long)vz.batch * vu.d;
  if (grid > 0x7fffffffLL) return T3F_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(k_assemble_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return T3F_ERR_CUDA;
  k_assemble_batch<<<(unsigned)grid, kThreads, smem, s>>>(a);
  T3F_CHECK(launch_status());
  return gauge_batch(vu, vd, s);
}

extern "C" t3f_status t3f_tangent_gram(const t3f_tt* dA, const t3f_tt* dB, float* G, int32_t math, void* ws,
                                       size_t ws_bytes, t3f_stream_t stream) {
  TTV va, vb;
  T3F_CHECK(make_view(dA, &va, T3F_F32, false));
  T3F_CHECK(make_view(dB, &vb, T3F_F32, false));
  if (!G) return T3F_ERR_ARG;
  if (va.d != vb.d) return T3F_ERR_SHAPE;
  for (int k = 0; k <= va.d; ++k)
    if (va.r[k] != vb.r[k] || (k < va.d && va.n[k] != vb.n[k])) return T3F_ERR_SHAPE;
  if (math == T3F_MATH_TF32) return run_tangent_gram_tc(va, vb, G, ws, ws_bytes, (cudaStream_t)stream);
  if (math != T3F_MATH_FP32) return T3F_ERR_UNSUPPORTED;
  const TGramPlan p = tgram_plan(va, vb);
  T3F_CHECK(check_ws(ws, ws_bytes, p.total));
  cudaStream_t s = (cudaStream_t)stream;
  TGramArgs g;
  memset(&g, 0, sizeof(g));
  g.A = va;
  g.B = vb;
  for (int k = 0; k < va.d; ++k) g.ksz[k] = va.osz[k];
  g.nchunks = p.nchunks;
  g.cper = p.cper;
  g.nsplit = p.nsplit;
  g.tilesB = p.tilesB;
  g.self = (va.p == vb.p && va.batch == vb.batch) ? 1 : 0;
  g.part = reinterpret_cast<float*>(static_cast<char*>(ws) + p.part_off);
  const long long grid = (long long)p.tilesA * p.tilesB * p.nsplit;
  if (grid > 0x7fffffffLL) return T3F_ERR_UNSUPPORTED;
  k_tgram<<<(unsigned)grid, kThreads, 0, s>>>(g);
  T3F_CHECK(launch_status());
  const long long size = (long long)va.batch * vb.batch;
  return run_split_reduce(g.part, p.nsplit, size, reinterpret_cast<float*>(static_cast<char*>(ws) + p.mid_off), G, s);
}

extern "C" size_t t3f_project_matvec_workspace_size(const t3f_tt* U, const t3f_tt* A, const t3f_tt* x) {
  TTV vu, va, vx;
  if (make_view(U, &vu, T3F_F32, false) != T3F_OK || make_view(A, &va, T3F_F32, true) != T3F_OK ||
      make_view(x, &vx, T3F_F32, false) != T3F_OK)
    return 0;
  if (vu.d != va.d || vu.d != vx.d) return 0;
  PmvPlan p;
  pmv_plan(vu, va, vx, &p);
  return p.total;
}

extern "C" t3f_status t3f_project_matvec(const t3f_tt* U, const t3f_tt* V, const t3f_tt* A, const t3f_tt* x,
                                         t3f_tt* dU, void* ws, size_t ws_bytes, t3f_stream_t stream) {
  TTV vu, vv, va, vx, vd;
  T3F_CHECK(uv_views(U, V, &vu, &vv));
  T3F_CHECK(make_view(A, &va, T3F_F32, true));
  T3F_CHECK(make_view(x, &vx, T3F_F32, false));
  if (va.d != vu.d || vx.d != vu.d) return T3F_ERR_SHAPE;
  if (va.batch != 1 && va.batch != vx.batch) return T3F_ERR_SHAPE;
  for (int k = 0; k < vu.d; ++k)
    if (va.m[k] != vu.n[k] || va.n[k] != vx.n[k]) return T3F_ERR_SHAPE;
  T3F_CHECK(coords_view(dU, vu, vx.batch, &vd));
  PmvPlan p;
  if (!pmv_plan(vu, va, vx, &p)) return T3F_ERR_UNSUPPORTED;
  T3F_CHECK(check_ws(ws, ws_bytes, p.total));
  cudaStream_t s = (cudaStream_t)stream;
  char* w = static_cast<char*>(ws);
  PmvArgs g;
  memset(&g, 0, sizeof(g));
  g.A = va;
  g.c = vx;
  g.D = vd;
  g.L = reinterpret_cast<float*>(w + p.offL);
  g.R = reinterpret_cast<float*>(w + p.offR);
  for (int k = 0; k <= vu.d; ++k) g.ioff[k] = p.ioff[k];
  for (int dir = 0; dir < 2; ++dir) {
    g.X = dir == 0 ? vu : vv;
    g.dir = dir;
    if (cudaFuncSetAttribute(k_pmv_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem_sweep[dir]) !=
        cudaSuccess)
      return T3F_ERR_CUDA;
    k_pmv_sweep<<<(unsigned)vx.batch, kThreads, p.smem_sweep[dir], s>>>(g);
    T3F_CHECK(launch_status());
  }
  g.X = vu;
  if (cudaFuncSetAttribute(k_pmv_assemble, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem_asm) != cudaSuccess)
    return T3F_ERR_CUDA;
  const long long grid = (long long)vx.batch * vu.d;
  if (grid > 0x7fffffffLL) return T3F_ERR_UNSUPPORTED;
  k_pmv_assemble<<<(unsigned)grid, kThreads, p.smem_asm, s>>>(g);
  T3F_CHECK(launch_status());
  return gauge_batch(vu, vd, s);
}

extern "C" t3f_status t3f_completion_hvp(const t3f_tt* U, const t3f_tt* V, const int32_t* idx, int64_t N,
                                         const t3f_tt* dZ, t3f_tt* out, void* ws, size_t ws_bytes,
                                         t3f_stream_t stream) {
  TTV vu, vv, vz, vo;
  T3F_CHECK(uv_views(U, V, &vu, &vv));
  T3F_CHECK(coords_view(dZ, vu, 1, &vz));
  T3F_CHECK(coords_view(out, vu, 1, &vo));
  if (N < 0 || (N > 0 && !idx)) return T3F_ERR_ARG;
  const size_t rg = ws_rgather(vu, vv, N);
  const size_t need = ws_completion_hvp(vu, vv, N);
  T3F_CHECK(check_ws(ws, ws_bytes, need));
  int R = vu.rmax <= 4 ? 4 : (vu.rmax <= 8 ? 8 : (vu.rmax <= 16 ? 16 : 0));
  if (!R) return T3F_ERR_UNSUPPORTED;
  const size_t smem = sizeof(float) * 3 * (size_t)vu.d * vu.nmax * (R * R + 4);
  if (smem > 200 * 1024) return T3F_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  float* wv = reinterpret_cast<float*>(static_cast<char*>(ws) + align256(rg));
  if (cudaMemsetAsync(ws, 0, sizeof(int), s) != cudaSuccess) return T3F_ERR_CUDA;
  if (N > 0) {
    TGatherArgs g;
    memset(&g, 0, sizeof(g));
    g.d = vu.d;
    g.nmax = vu.nmax;
    g.N = N;
    for (int k = 0; k < vu.d; ++k) {
      g.n[k] = vu.n[k];
      g.off[k] = vu.off[k];
    }
    for (int k = 0; k <= vu.d; ++k) g.r[k] = vu.r[k];
    g.U = static_cast<const float*>(vu.p);
    g.V = static_cast<const float*>(vv.p);
    g.W = static_cast<const float*>(vz.p);
    g.idx = idx;
    g.out = wv;
    g.err = static_cast<int*>(ws);
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)std::min<long long>((N + 255) / 256, (long long)sms * 4);
    switch (R) {
      case 4:
        cudaFuncSetAttribute(k_tangent_gather<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_tangent_gather<4><<<grid, 256, smem, s>>>(g);
        break;
      case 8:
        cudaFuncSetAttribute(k_tangent_gather<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_tangent_gather<8><<<grid, 256, smem, s>>>(g);
        break;
      default:
        cudaFuncSetAttribute(k_tangent_gather<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_tangent_gather<16><<<grid, 256, smem, s>>>(g);
        break;
    }
    T3F_CHECK(launch_status());
  }
  // P_X (sum_t w_t e_{i_t}) with w_t = xi(i_t): the Riemannian adjoint scatter with weights
  return t3f_gather_backward(nullptr, idx, N, wv, nullptr, nullptr, out, 1, U, V, ws, rg, stream);
}
