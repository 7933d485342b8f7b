// Element gather, completion loss and its adjoint (paper Section 1's completion example;
// Section 3.2's Riemannian gradient of that loss).
//
// For a tuple t with indices i_{t,1..d}:
//   prefix  l_{t,0} = 1,          l_{t,k} = l_{t,k-1} G^k[:, i_{t,k}, :]
//   suffix  rho_{t,d+1} = 1,      rho_{t,k} = G^k[:, i_{t,k}, :] rho_{t,k+1}
//   X(i_t) = l_{t,d} = rho_{t,1}
//   cotangent of sum_t w_t X(i_t):  dG^k[:, i, :] = sum_{t: i_{t,k} = i} w_t l_{t,k-1} rho_{t,k+1}^T
// One thread owns one tuple. The cores are staged in shared memory as zero-padded R x R
// mode slices, so the chains run fully unrolled in registers. The adjoint stores the
// suffix vectors of its tuple in shared memory, evaluates the residual, then walks the
// prefix and scatters the outer products into a per-CTA shared accumulator; a second
// kernel reduces the per-CTA partials in a fixed order.
#include <mutex>

#include "t3f_internal.cuh"

namespace t3f {

constexpr int kGatherThreads = 128;

struct GatherArgs {
  int d;
  long long N;
  int nmax;
  int rl[T3F_MAX_D + 1];     // ranks of the prefix cores (X or U)
  int rr[T3F_MAX_D + 1];     // ranks of the suffix cores (X or V)
  int n[T3F_MAX_D];
  const float* L;            // prefix cores, packed, batch 1
  long long Loff[T3F_MAX_D];
  const float* Rg;           // suffix cores, packed, batch 1
  long long Roff[T3F_MAX_D];
  int same;                  // L and R are the same cores
  const int* idx;            // [d][N]
  const float* y;            // nullable
  const float* w;            // nullable
  float* vals;               // nullable
  double* loss_part;         // [gridDim.x] nullable
  float* grad_part;          // [gridDim.x][gsize] nullable
  long long goff[T3F_MAX_D]; // compact per-core offsets of the gradient (r^L_k x n_k x r^R_{k+1})
  long long gsize;
  int* err;                  // device error word
};

template <int R>
__device__ __forceinline__ void stage_padded(float* dst, const float* src, const long long* off,
                                             const int* r, const int* n, int d, int nmax) {
  const int total = d * nmax * R * R;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int b = e % R, a = (e / R) % R, i = (e / (R * R)) % nmax, k = e / (R * R * nmax);
    float v = 0.0f;
    if (i < n[k] && a < r[k] && b < r[k + 1])
      v = __ldg(src + off[k] + ((long long)a * n[k] + i) * r[k + 1] + b);
    dst[e] = v;
  }
}

__device__ __forceinline__ int load_index(const GatherArgs& g, int k, long long t) {
  int i = __ldg(g.idx + (long long)k * g.N + t);
  if (i < 0 || i >= g.n[k]) {
    atomicExch(g.err, (int)T3F_ERR_ARG);
    i = i < 0 ? 0 : g.n[k] - 1;
  }
  return i;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  __syncthreads();
  return s;
}

// Forward: values and / or loss partials.
template <int R>
__global__ void __launch_bounds__(kGatherThreads) k_gather_fwd(const __grid_constant__ GatherArgs g) {
  extern __shared__ float sm[];
  __shared__ double red[kGatherThreads / 32];
  float* Ls = sm;
  stage_padded<R>(Ls, g.L, g.Loff, g.rl, g.n, g.d, g.nmax);
  __syncthreads();
  double lsum = 0.0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < g.N;
       t += (long long)gridDim.x * blockDim.x) {
    float l[R];
#pragma unroll
    for (int a = 0; a < R; ++a) l[a] = a == 0 ? 1.0f : 0.0f;
    for (int k = 0; k < g.d; ++k) {
      const int i = load_index(g, k, t);
      const float* S = Ls + (k * g.nmax + i) * R * R;
      float nl[R];
#pragma unroll
      for (int b = 0; b < R; ++b) nl[b] = 0.0f;
#pragma unroll
      for (int a = 0; a < R; ++a) {
#pragma unroll
        for (int b = 0; b < R; b += 4) {
          const float4 s4 = *reinterpret_cast<const float4*>(S + a * R + b);
          nl[b] = fmaf(l[a], s4.x, nl[b]);
          nl[b + 1] = fmaf(l[a], s4.y, nl[b + 1]);
          nl[b + 2] = fmaf(l[a], s4.z, nl[b + 2]);
          nl[b + 3] = fmaf(l[a], s4.w, nl[b + 3]);
        }
      }
#pragma unroll
      for (int b = 0; b < R; ++b) l[b] = nl[b];
    }
    const float x = l[0];
    if (g.vals) g.vals[t] = x;
    if (g.loss_part) {
      const double res = (double)x - (double)g.y[t];
      lsum += 0.5 * res * res;
    }
  }
  if (g.loss_part) {
    const double s = block_sum(lsum, red);
    if (threadIdx.x == 0) g.loss_part[blockIdx.x] = s;
  }
}

// Adjoint (Euclidean or Riemannian): per-CTA partial gradients (+ loss partials).
template <int R>
__global__ void __launch_bounds__(kGatherThreads) k_gather_bwd(const __grid_constant__ GatherArgs g) {
  extern __shared__ float sm[];
  __shared__ double red[kGatherThreads / 32];
  const int SL = g.d * g.nmax * R * R;   // staged floats per core set
  const int GS = R * R + 1;              // odd slice stride of the accumulator
  float* Ls = sm;
  float* Rs = g.same ? Ls : Ls + SL;
  float* acc = Ls + (g.same ? SL : 2 * SL);  // d * nmax * GS
  float* sfx = acc + g.d * g.nmax * GS;      // [d][R][blockDim]: suffix at interface k+1
  stage_padded<R>(Ls, g.L, g.Loff, g.rl, g.n, g.d, g.nmax);
  if (!g.same) stage_padded<R>(Rs, g.Rg, g.Roff, g.rr, g.n, g.d, g.nmax);
  for (int e = threadIdx.x; e < g.d * g.nmax * GS; e += blockDim.x) acc[e] = 0.0f;
  __syncthreads();
  const int tid = threadIdx.x, nth = blockDim.x;
  double lsum = 0.0;
  for (long long t0 = (long long)blockIdx.x * nth; t0 < g.N; t0 += (long long)gridDim.x * nth) {
    const long long t = t0 + tid;
    const bool active = t < g.N;
    if (active) {
      // suffix chain through the right cores
      float rho[R];
#pragma unroll
      for (int a = 0; a < R; ++a) rho[a] = a == 0 ? 1.0f : 0.0f;
      for (int k = g.d - 1; k >= 1; --k) {
#pragma unroll
        for (int a = 0; a < R; ++a) sfx[(k * R + a) * nth + tid] = rho[a];
        const int i = load_index(g, k, t);
        const float* S = Rs + (k * g.nmax + i) * R * R;
        float nr[R];
#pragma unroll
        for (int a = 0; a < R; ++a) {
          float s = 0.0f;
#pragma unroll
          for (int b = 0; b < R; b += 4) {
            const float4 s4 = *reinterpret_cast<const float4*>(S + a * R + b);
            s = fmaf(s4.x, rho[b], s);
            s = fmaf(s4.y, rho[b + 1], s);
            s = fmaf(s4.z, rho[b + 2], s);
            s = fmaf(s4.w, rho[b + 3], s);
          }
          nr[a] = s;
        }
#pragma unroll
        for (int a = 0; a < R; ++a) rho[a] = nr[a];
      }
#pragma unroll
      for (int a = 0; a < R; ++a) sfx[a * nth + tid] = rho[a];
      const int i0 = load_index(g, 0, t);
      // X(i_t) = row 0 of the first suffix core's slice times the suffix at interface 1
      const float* S0 = Rs + i0 * R * R;
      float x = 0.0f;
#pragma unroll
      for (int b = 0; b < R; ++b) x = fmaf(S0[b], rho[b], x);
      float wt;
      if (g.w) {
        wt = g.w[t];
      } else {
        const double res = (double)x - (double)g.y[t];
        lsum += 0.5 * res * res;
        wt = (float)res;
      }
      // prefix walk with the scatter of w l_k rho_{k+1}^T into slice i_k of core k
      float l[R];
#pragma unroll
      for (int a = 0; a < R; ++a) l[a] = a == 0 ? wt : 0.0f;  // carries the weight
      for (int k = 0; k < g.d; ++k) {
        const int i = (k == 0) ? i0 : load_index(g, k, t);
        float r1[R];
#pragma unroll
        for (int b = 0; b < R; ++b) r1[b] = sfx[(k * R + b) * nth + tid];
        const int ra = g.rl[k], rb = g.rr[k + 1];
        float* A = acc + (k * g.nmax + i) * GS;
#pragma unroll
        for (int a = 0; a < R; ++a) {
          if (a < ra) {
#pragma unroll
            for (int b = 0; b < R; ++b)
              if (b < rb) atomicAdd(A + a * R + b, l[a] * r1[b]);
          }
        }
        if (k + 1 < g.d) {
          const float* S = Ls + (k * g.nmax + i) * R * R;
          float nl[R];
#pragma unroll
          for (int b = 0; b < R; ++b) nl[b] = 0.0f;
#pragma unroll
          for (int a = 0; a < R; ++a) {
#pragma unroll
            for (int b = 0; b < R; b += 4) {
              const float4 s4 = *reinterpret_cast<const float4*>(S + a * R + b);
              nl[b] = fmaf(l[a], s4.x, nl[b]);
              nl[b + 1] = fmaf(l[a], s4.y, nl[b + 1]);
              nl[b + 2] = fmaf(l[a], s4.z, nl[b + 2]);
              nl[b + 3] = fmaf(l[a], s4.w, nl[b + 3]);
            }
          }
#pragma unroll
          for (int b = 0; b < R; ++b) l[b] = nl[b];
        }
      }
    }
  }
  __syncthreads();
  // write this CTA's partial gradient in the compact layout
  float* out = g.grad_part + (long long)blockIdx.x * g.gsize;
  for (int k = 0; k < g.d; ++k) {
    const int ra = g.rl[k], rb = g.rr[k + 1], nk = g.n[k];
    for (int e = tid; e < ra * nk * rb; e += nth) {
      const int b = e % rb, i = (e / rb) % nk, a = e / (rb * nk);
      out[g.goff[k] + e] = acc[(k * g.nmax + i) * GS + a * R + b];
    }
  }
  if (g.loss_part) {
    const double s = block_sum(lsum, red);
    if (threadIdx.x == 0) g.loss_part[blockIdx.x] = s;
  }
}

__global__ void k_reduce_partials(const float* part, int nparts, long long size, float* out) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < size;
       e += (long long)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int p = 0; p < nparts; ++p) s += part[(long long)p * size + e];
    out[e] = s;
  }
}

__global__ void k_reduce_loss(const double* part, int nparts, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int p = threadIdx.x; p < nparts; p += blockDim.x) s += part[p];
  s = block_sum(s, red);
  if (threadIdx.x == 0) *out = s;
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------

static int pick_R(int rmax) {
  if (rmax <= 4) return 4;
  if (rmax <= 8) return 8;
  if (rmax <= 16) return 16;
  return 0;
}

static int gather_grid(long long N, int maxCtas) {
  long long g = (N + kGatherThreads - 1) / kGatherThreads;
  if (g > maxCtas) g = maxCtas;
  return (int)(g < 1 ? 1 : g);
}

static int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  return sms;
}

struct GatherLayout {
  int R;
  int grid;
  size_t smem;
  size_t loss_off, grad_off, total;
};

static GatherLayout gather_layout(const TTV& L, const TTV& Rv, long long N, bool bwd, bool same) {
  GatherLayout lay{};
  lay.R = pick_R(L.rmax > Rv.rmax ? L.rmax : Rv.rmax);
  const int R = lay.R ? lay.R : 16;
  const int nmax = L.nmax;
  const size_t SL = (size_t)L.d * nmax * R * R;
  if (!bwd) {
    lay.smem = sizeof(float) * SL;
    lay.grid = gather_grid(N, num_sms() * 8);
  } else {
    lay.smem = sizeof(float) * ((same ? 1 : 2) * SL + (size_t)L.d * nmax * (R * R + 1) +
                                (size_t)L.d * R * kGatherThreads);
    lay.grid = gather_grid(N, num_sms() * 2);
  }
  long long gsize = 0;
  for (int k = 0; k < L.d; ++k) gsize += (long long)L.r[k] * L.n[k] * Rv.r[k + 1];
  lay.loss_off = kWsHeader;
  lay.grad_off = lay.loss_off + align256(sizeof(double) * lay.grid);
  lay.total = lay.grad_off + (bwd ? align256(sizeof(float) * gsize * lay.grid) : 0);
  return lay;
}

size_t ws_gather(const TTV& X, long long N, bool bwd) {
  return gather_layout(X, X, N, bwd, true).total;
}
size_t ws_rgather(const TTV& U, const TTV& V, long long N) {
  return gather_layout(U, V, N, true, false).total;
}

static void fill_args(GatherArgs* g, const TTV& L, const TTV& Rv) {
  g->d = L.d;
  g->nmax = L.nmax;
  for (int k = 0; k <= L.d; ++k) {
    g->rl[k] = L.r[k];
    g->rr[k] = Rv.r[k];
  }
  long long go = 0;
  for (int k = 0; k < L.d; ++k) {
    g->n[k] = L.n[k];
    g->Loff[k] = L.off[k];
    g->Roff[k] = Rv.off[k];
    g->goff[k] = go;
    go += (long long)L.r[k] * L.n[k] * Rv.r[k + 1];
  }
  g->gsize = go;
  g->L = static_cast<const float*>(L.p);
  g->Rg = static_cast<const float*>(Rv.p);
}

template <int R>
static t3f_status launch_fwd(const GatherArgs& g, const GatherLayout& lay, cudaStream_t s) {
  auto kern = k_gather_fwd<R>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.smem) != cudaSuccess)
    return T3F_ERR_CUDA;
  kern<<<lay.grid, kGatherThreads, lay.smem, s>>>(g);
  return launch_status();
}

template <int R>
static t3f_status launch_bwd(const GatherArgs& g, const GatherLayout& lay, cudaStream_t s) {
  auto kern = k_gather_bwd<R>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.smem) != cudaSuccess)
    return T3F_ERR_CUDA;
  kern<<<lay.grid, kGatherThreads, lay.smem, s>>>(g);
  return launch_status();
}

}  // namespace t3f

using namespace t3f;

extern "C" t3f_status t3f_gather(const t3f_tt* X, const int32_t* idx, int64_t N, const float* y,
                                 float* vals, double* loss, void* ws, size_t ws_bytes,
                                 t3f_stream_t stream) {
  TTV vx;
  T3F_CHECK(make_view(X, &vx, T3F_F32, false));
  if (vx.batch != 1) return T3F_ERR_SHAPE;
  if (N < 0 || (N > 0 && !idx) || (loss && !y && N > 0)) return T3F_ERR_ARG;
  GatherLayout lay = gather_layout(vx, vx, N, false, true);
  if (!lay.R || lay.smem > 200 * 1024) return T3F_ERR_UNSUPPORTED;
  T3F_CHECK(check_ws(ws, ws_bytes, lay.total));
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(ws, 0, sizeof(int32_t), s) != cudaSuccess) return T3F_ERR_CUDA;
  if (N == 0) {
    if (loss && cudaMemsetAsync(loss, 0, sizeof(double), s) != cudaSuccess) return T3F_ERR_CUDA;
    return T3F_OK;
  }
  GatherArgs g;
  memset(&g, 0, sizeof(g));
  fill_args(&g, vx, vx);
  g.same = 1;
  g.N = N;
  g.idx = idx;
  g.y = y;
  g.vals = vals;
  g.err = static_cast<int*>(ws);
  double* lp = reinterpret_cast<double*>(static_cast<char*>(ws) + lay.loss_off);
  g.loss_part = loss ? lp : nullptr;
  t3f_status st;
  switch (lay.R) {
    case 4: st = launch_fwd<4>(g, lay, s); break;
    case 8: st = launch_fwd<8>(g, lay, s); break;
    default: st = launch_fwd<16>(g, lay, s); break;
  }
  T3F_CHECK(st);
  if (loss) {
    k_reduce_loss<<<1, 1024, 0, s>>>(lp, lay.grid, loss);
    T3F_CHECK(launch_status());
  }
  return T3F_OK;
}

extern "C" t3f_status t3f_gather_backward(const t3f_tt* X, const int32_t* idx, int64_t N,
                                          const float* w, const float* y, double* loss,
                                          t3f_tt* dX, int32_t riemannian, const t3f_tt* U,
                                          const t3f_tt* V, void* ws, size_t ws_bytes,
                                          t3f_stream_t stream) {
  TTV vl, vr, vd;
  if (riemannian != 0 && riemannian != 1) return T3F_ERR_ARG;
  if (riemannian) {
    T3F_CHECK(make_view(U, &vl, T3F_F32, false));
    T3F_CHECK(make_view(V, &vr, T3F_F32, false));
    if (vl.batch != 1 || vr.batch != 1 || vl.d != vr.d) return T3F_ERR_SHAPE;
    for (int k = 0; k <= vl.d; ++k)
      if (vl.r[k] != vr.r[k] || (k < vl.d && vl.n[k] != vr.n[k])) return T3F_ERR_SHAPE;
  } else {
    T3F_CHECK(make_view(X, &vl, T3F_F32, false));
    if (vl.batch != 1) return T3F_ERR_SHAPE;
    vr = vl;
  }
  T3F_CHECK(make_view(dX, &vd, T3F_F32, false));
  if (vd.batch != 1 || vd.d != vl.d) return T3F_ERR_SHAPE;
  for (int k = 0; k <= vl.d; ++k)
    if (vd.r[k] != vl.r[k] || (k < vl.d && vd.n[k] != vl.n[k])) return T3F_ERR_SHAPE;
  if (N < 0 || (N > 0 && !idx)) return T3F_ERR_ARG;
  if (N > 0 && !w && !y) return T3F_ERR_ARG;
  if (w && loss) return T3F_ERR_ARG;
  const bool same = !riemannian;
  GatherLayout lay = gather_layout(vl, vr, N, true, same);
  if (!lay.R || lay.smem > 200 * 1024) return T3F_ERR_UNSUPPORTED;
  T3F_CHECK(check_ws(ws, ws_bytes, lay.total));
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(ws, 0, sizeof(int32_t), s) != cudaSuccess) return T3F_ERR_CUDA;
  float* out = static_cast<float*>(vd.p);
  const long long gsize = t3f_packed_size(dX);
  if (N == 0) {
    if (cudaMemsetAsync(out, 0, sizeof(float) * gsize, s) != cudaSuccess) return T3F_ERR_CUDA;
    if (loss && cudaMemsetAsync(loss, 0, sizeof(double), s) != cudaSuccess) return T3F_ERR_CUDA;
    return T3F_OK;
  }
  GatherArgs g;
  memset(&g, 0, sizeof(g));
  fill_args(&g, vl, vr);
  g.same = same ? 1 : 0;
  g.N = N;
  g.idx = idx;
  g.y = y;
  g.w = w;
  g.err = static_cast<int*>(ws);
  double* lp = reinterpret_cast<double*>(static_cast<char*>(ws) + lay.loss_off);
  g.loss_part = (!w && loss) ? lp : nullptr;
  float* gp = reinterpret_cast<float*>(static_cast<char*>(ws) + lay.grad_off);
  g.grad_part = gp;
  t3f_status st;
  switch (lay.R) {
    case 4: st = launch_bwd<4>(g, lay, s); break;
    case 8: st = launch_bwd<8>(g, lay, s); break;
    default: st = launch_bwd<16>(g, lay, s); break;
  }
  T3F_CHECK(st);
  // the compact gradient layout equals the packed layout of a batch-1 descriptor
  float* target = out;
  if (riemannian) {
    // reduce into the tail of the workspace region? reuse the first partial slot instead
    target = gp;  // partial 0 is overwritten by the sum (read before write per element)
  }
  k_reduce_partials<<<num_sms() * 4, 256, 0, s>>>(gp, lay.grid, g.gsize, target);
  T3F_CHECK(launch_status());
  if (loss && !w) {
    k_reduce_loss<<<1, 1024, 0, s>>>(lp, lay.grid, loss);
    T3F_CHECK(launch_status());
  }
  if (riemannian) T3F_CHECK(run_gauge_project(vl, gp, out, s));
  return T3F_OK;
}

// ---------------------------------------------------------------------------------------
// Allocation-free variant of t3f_gather.
//
// Some callers cannot allocate device memory for the workspace: a plugin whose host
// framework owns every byte of device memory through its own pool or a hard memory cap
// (a cudaMalloc there either fails or escapes the host's accounting), or code that must
// not risk the implicit device synchronisation that cudaMalloc/cudaFree can cause. This
// entry point needs no workspace: its scratch (the device error word and the per-CTA loss
// partials) lives in one file-scope device array of T3F_NOALLOC_SCRATCH_BYTES that every
// GPU which loads the library keeps until the process exits.
// ---------------------------------------------------------------------------------------

namespace t3f {

static __device__ __align__(256) unsigned char g_noalloc_scratch[T3F_NOALLOC_SCRATCH_BYTES];

constexpr int kNoAllocMaxDevices = 64;
static std::once_flag g_noalloc_once[kNoAllocMaxDevices];
static void* g_noalloc_ptr[kNoAllocMaxDevices];
static cudaError_t g_noalloc_err[kNoAllocMaxDevices];

// Device address of the scratch array on the current device. The array's name in host
// code is only a host-side stand-in, so the address is looked up once per device (with
// that device current) and cached.
static t3f_status noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return T3F_ERR_CUDA;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return T3F_ERR_UNSUPPORTED;
  std::call_once(g_noalloc_once[dev], [dev]() {
    g_noalloc_err[dev] = cudaGetSymbolAddress(&g_noalloc_ptr[dev], g_noalloc_scratch);
  });
  if (g_noalloc_err[dev] != cudaSuccess || !g_noalloc_ptr[dev]) return T3F_ERR_CUDA;
  *out = g_noalloc_ptr[dev];
  return T3F_OK;
}

}  // namespace t3f

extern "C" t3f_status t3f_gather_noalloc(const t3f_tt* X, const int32_t* idx, int64_t N,
                                         const float* y, float* vals, double* loss,
                                         t3f_stream_t stream) {
  TTV vx;
  T3F_CHECK(make_view(X, &vx, T3F_F32, false));
  if (N < 0) return T3F_ERR_ARG;
  if (gather_layout(vx, vx, N, false, true).total > (size_t)T3F_NOALLOC_SCRATCH_BYTES)
    return T3F_ERR_WORKSPACE;
  void* scratch = nullptr;
  T3F_CHECK(noalloc_scratch(&scratch));
  // the existing entry point clears the error word and overwrites every partial it reads
  return t3f_gather(X, idx, N, y, vals, loss, scratch, T3F_NOALLOC_SCRATCH_BYTES, stream);
}
