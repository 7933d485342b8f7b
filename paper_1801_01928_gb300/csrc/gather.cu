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
#include <atomic>
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
  long long Lnfl, Rnfl;      // floats of the packed prefix / suffix object
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

// ---- whole-object staging through the TMA unit -------------------------------------------
// One cp.async.bulk copies the packed cores of a batch-1 TT (rounded out to 16-byte
// boundaries: the copy may start up to 12 bytes before the object and end up to 15 bytes
// after it, always inside the same 16-byte block, hence the same page) into a landing zone
// of shared memory; stage_from_raw then lays the slices out on chip. The landing zone is
// the first core rounded down by delta floats: raw[delta + element offset].

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
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

__device__ __forceinline__ void bar_init(uint64_t* bar) {
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
}

__host__ __device__ __forceinline__ uint32_t raw_bytes(const float* src, long long nfl) {
  const uintptr_t s = reinterpret_cast<uintptr_t>(src);
  return (uint32_t)(((s & 15) + (uintptr_t)nfl * 4 + 15) & ~uintptr_t(15));
}

__device__ __forceinline__ int raw_delta(const float* src) { return (int)((reinterpret_cast<uintptr_t>(src) & 15) >> 2); }

// thread 0: one bulk copy of [src, src + nfl) (rounded out) into raw, completing on bar
__device__ __forceinline__ void tma_copy(float* raw, const float* src, long long nfl, uint64_t* bar) {
  const uintptr_t s0 = reinterpret_cast<uintptr_t>(src) & ~uintptr_t(15);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(raw)),
               "l"(s0), "r"(raw_bytes(src, nfl)), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tma_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// zero-padded R x R slices with slice stride SS from the landed object
template <int R>
__device__ __forceinline__ void stage_from_raw(float* dst, int SS, const float* raw, const long long* off,
                                               const int* r, const int* n, int d, int nmax) {
  const int total = d * nmax * SS;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int q = e % SS, i = (e / SS) % nmax, k = e / (SS * nmax);
    const int a = q / R, b = q % R;
    float v = 0.0f;
    if (q < R * R && i < n[k] && a < r[k] && b < r[k + 1]) v = raw[off[k] + ((long long)a * n[k] + i) * r[k + 1] + b];
    dst[e] = v;
  }
}

// land one object and stage it (every thread; bar used at `parity`); false on a timeout
template <int R>
__device__ bool stage_object_tma(float* dst, int SS, float* landing, const float* src, long long nfl,
                                 const long long* off, const int* r, const int* n, int d, int nmax, uint64_t* bar,
                                 uint32_t parity) {
  if (threadIdx.x == 0) {
    tma_expect(bar, raw_bytes(src, nfl));
    tma_copy(landing, src, nfl, bar);
  }
  const bool ok = bar_wait(smem_u32(bar), parity);
  stage_from_raw<R>(dst, SS, landing + raw_delta(src), off, r, n, d, nmax);
  return ok;
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
  extern __shared__ __align__(16) float sm[];
  __shared__ double red[kGatherThreads / 32];
  __shared__ __align__(8) uint64_t bar;
  float* Ls = sm;
  // slices R^2 + 4 floats apart: the random slice indices of a warp's tuples fall on
  // different banks
  constexpr int SS = R * R + 4;
  float* landing = sm + g.d * g.nmax * SS;  // 16-byte aligned (SS is a multiple of 4)
  bar_init(&bar);
  if (!stage_object_tma<R>(Ls, SS, landing, g.L, g.Lnfl, g.Loff, g.rl, g.n, g.d, g.nmax, &bar, 0u) &&
      threadIdx.x == 0)
    atomicExch(g.err, (int)T3F_ERR_TIMEOUT);
  __syncthreads();
  double lsum = 0.0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < g.N;
       t += (long long)gridDim.x * blockDim.x) {
    float l[R];
#pragma unroll
    for (int a = 0; a < R; ++a) l[a] = a == 0 ? 1.0f : 0.0f;
    for (int k = 0; k < g.d; ++k) {
      const int i = load_index(g, k, t);
      const float* S = Ls + (k * g.nmax + i) * SS;
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
  constexpr int SS = R * R + 4;          // slice stride (distinct banks for random slices)
  const int SL = g.d * g.nmax * SS;      // staged floats per core set
  const int GS = R * R + 1;              // odd slice stride of the accumulator
  float* Ls = sm;
  float* Rs = g.same ? Ls : Ls + SL;
  float* acc = Ls + (g.same ? SL : 2 * SL);  // d * nmax * GS
  float* sfx = acc + g.d * g.nmax * GS;      // [d][R][blockDim]: suffix at interface k+1
  // both objects land in the accumulator region (zeroed afterwards), one after the other
  __shared__ __align__(8) uint64_t bar;
  bar_init(&bar);
  bool ok = stage_object_tma<R>(Ls, SS, acc, g.L, g.Lnfl, g.Loff, g.rl, g.n, g.d, g.nmax, &bar, 0u);
  __syncthreads();
  if (!g.same) {
    ok &= stage_object_tma<R>(Rs, SS, acc, g.Rg, g.Rnfl, g.Roff, g.rr, g.n, g.d, g.nmax, &bar, 1u);
    __syncthreads();
  }
  if (!ok && threadIdx.x == 0) atomicExch(g.err, (int)T3F_ERR_TIMEOUT);
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
        const float* S = Rs + (k * g.nmax + i) * SS;
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
      const float* S0 = Rs + i0 * SS;
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
          const float* S = Ls + (k * g.nmax + i) * SS;
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

// Bucketed adjoint (the main path for ranks <= 8). Per chunk of T = blockDim tuples:
//  (1) a deterministic counting sort of the chunk's tuples by slice, for every core (warp
//      match + per-warp prefix sums), giving each tuple its bucket position at core k;
//  (2) thread per tuple: suffix chain storing rho_{k+1} and prefix chain (scaled by the
//      weight) storing w l_k, both written into the bucket order of core k;
//  (3) thread per item (core k, slice s, part): a persistent R x R register accumulator
//      adds w l_k rho_{k+1}^T over the item's share of the bucket; consecutive lanes read
//      consecutive bucket rows.
// No atomics in the loop; the per-CTA partial is summed in a fixed order by a second kernel.
struct CompletionArgs {
  GatherArgs g;
  int T;                      // tuples per chunk (= blockDim.x)
  int NB;                     // buckets per core (nmax + 1; the last holds invalid tuples)
  int parts[T3F_MAX_D];       // items per slice at core k
  int item0[T3F_MAX_D + 1];   // first item of core k
};

template <int R>
__global__ void __launch_bounds__(256, 1) k_completion(const __grid_constant__ CompletionArgs ca) {
  extern __shared__ __align__(16) float sm[];
  __shared__ double red[8];
  const GatherArgs& g = ca.g;
  const int d = g.d, nmax = g.nmax, T = ca.T, NB = ca.NB;
  constexpr int SS = R * R + 4;  // padded slice stride (breaks same-bank slices)
  constexpr int H = R / 4;       // float4 planes of a rank vector
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, NW = (T + 31) >> 5;
  const int SL = d * nmax * SS;
  float* Ls = sm;
  float* Rs = g.same ? Ls : Ls + SL;
  float4* RH = reinterpret_cast<float4*>(Ls + (g.same ? SL : 2 * SL));  // [d][H][T]
  float4* LW = RH + (size_t)d * H * T;                                     // [d][H][T]
  unsigned short* POS = reinterpret_cast<unsigned short*>(LW + (size_t)d * H * T);  // [d][T]
  unsigned char* IDX = reinterpret_cast<unsigned char*>(POS + (size_t)d * T);       // [d][T]
  unsigned short* WC = reinterpret_cast<unsigned short*>(IDX + (((size_t)d * T + 15) & ~(size_t)15));  // [d][NB][NW]
  int* CNT = reinterpret_cast<int*>(WC + (((size_t)d * NB * NW + 1) & ~(size_t)1));                      // [d][NB]
  int* BO = CNT + (size_t)d * NB;                                                   // [d][NB+1]

  // stage the cores as zero-padded R x R slices with stride SS: the whole object(s) land in
  // the RH / LW region (not used before the first chunk) through one TMA bulk copy each
  __shared__ __align__(8) uint64_t bar;
  bar_init(&bar);
  float* landL = reinterpret_cast<float*>(RH);
  float* landR = landL + ((raw_bytes(g.L, g.Lnfl) + 15) / 16) * 4;
  if (tid == 0) {
    tma_expect(&bar, raw_bytes(g.L, g.Lnfl) + (g.same ? 0u : raw_bytes(g.Rg, g.Rnfl)));
    tma_copy(landL, g.L, g.Lnfl, &bar);
    if (!g.same) tma_copy(landR, g.Rg, g.Rnfl, &bar);
  }
  if (!bar_wait(smem_u32(&bar), 0u) && tid == 0) atomicExch(g.err, (int)T3F_ERR_TIMEOUT);
  stage_from_raw<R>(Ls, SS, landL + raw_delta(g.L), g.Loff, g.rl, g.n, d, nmax);
  if (!g.same) stage_from_raw<R>(Rs, SS, landR + raw_delta(g.Rg), g.Roff, g.rr, g.n, d, nmax);
  __syncthreads();
  // this thread's item (core ik, slice is, part ip) of the accumulation phase
  int ik = -1, is = 0, ip = 0, np = 1;
  for (int k = 0; k < d; ++k)
    if (tid >= ca.item0[k] && tid < ca.item0[k + 1]) {
      ik = k;
      is = (tid - ca.item0[k]) / ca.parts[k];
      ip = (tid - ca.item0[k]) % ca.parts[k];
      np = ca.parts[k];
    }
  float acc[R][R];
#pragma unroll
  for (int a = 0; a < R; ++a)
#pragma unroll
    for (int b = 0; b < R; ++b) acc[a][b] = 0.0f;
  double lsum = 0.0;
  __syncthreads();

  for (long long base = (long long)blockIdx.x * T; base < g.N; base += (long long)gridDim.x * T) {
    const long long t = base + tid;
    const bool valid = tid < T && t < g.N;
    // (1) counting sort by slice, per core
    for (int e = tid; e < d * NB * NW; e += blockDim.x) WC[e] = 0;
    __syncthreads();
    for (int k = 0; k < d; ++k) {
      const int sl = valid ? load_index(g, k, t) : nmax;
      const unsigned m = __match_any_sync(0xffffffffu, sl);
      const int rank = __popc(m & ((1u << lane) - 1u));
      if (tid < T) {
        IDX[k * T + tid] = (unsigned char)sl;
        POS[k * T + tid] = (unsigned short)rank;
        if (rank == 0) WC[(k * NB + sl) * NW + warp] = (unsigned short)__popc(m);
      }
    }
    __syncthreads();
    for (int e = tid; e < d * NB; e += blockDim.x) {
      int run = 0;
      for (int w = 0; w < NW; ++w) {
        const int c = WC[e * NW + w];
        WC[e * NW + w] = (unsigned short)run;
        run += c;
      }
      CNT[e] = run;
    }
    __syncthreads();
    for (int k = tid; k < d; k += blockDim.x) {
      int run = 0;
      for (int sl = 0; sl < NB; ++sl) {
        BO[k * (NB + 1) + sl] = run;
        run += CNT[k * NB + sl];
      }
      BO[k * (NB + 1) + NB] = run;
    }
    __syncthreads();
    if (tid < T)
      for (int k = 0; k < d; ++k) {
        const int sl = IDX[k * T + tid];
        POS[k * T + tid] = (unsigned short)(BO[k * (NB + 1) + sl] + WC[(k * NB + sl) * NW + warp] + POS[k * T + tid]);
      }
    __syncthreads();
    // (2) chains of this thread's tuple
    if (valid) {
      float rho[R];
#pragma unroll
      for (int a = 0; a < R; ++a) rho[a] = a == 0 ? 1.0f : 0.0f;
      for (int k = d - 1; k >= 1; --k) {
        const int p = POS[k * T + tid];
#pragma unroll
        for (int h = 0; h < H; ++h)
          RH[((size_t)k * H + h) * T + p] = make_float4(rho[4 * h], rho[4 * h + 1], rho[4 * h + 2], rho[4 * h + 3]);
        const float* S = Rs + (k * nmax + IDX[k * T + tid]) * SS;
        float nr[R];
#pragma unroll
        for (int a = 0; a < R; ++a) {
          float acc1 = 0.0f;
#pragma unroll
          for (int b = 0; b < R; b += 4) {
            const float4 s4 = *reinterpret_cast<const float4*>(S + a * R + b);
            acc1 = fmaf(s4.x, rho[b], acc1);
            acc1 = fmaf(s4.y, rho[b + 1], acc1);
            acc1 = fmaf(s4.z, rho[b + 2], acc1);
            acc1 = fmaf(s4.w, rho[b + 3], acc1);
          }
          nr[a] = acc1;
        }
#pragma unroll
        for (int a = 0; a < R; ++a) rho[a] = nr[a];
      }
      {
        const int p = POS[tid];
#pragma unroll
        for (int h = 0; h < H; ++h)
          RH[(size_t)h * T + p] = make_float4(rho[4 * h], rho[4 * h + 1], rho[4 * h + 2], rho[4 * h + 3]);
      }
      const float* S0 = Rs + IDX[tid] * SS;
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
      float l[R];
#pragma unroll
      for (int a = 0; a < R; ++a) l[a] = a == 0 ? wt : 0.0f;
      for (int k = 0; k < d; ++k) {
        const int p = POS[k * T + tid];
#pragma unroll
        for (int h = 0; h < H; ++h)
          LW[((size_t)k * H + h) * T + p] = make_float4(l[4 * h], l[4 * h + 1], l[4 * h + 2], l[4 * h + 3]);
        if (k + 1 == d) break;
        const float* S = Ls + (k * nmax + IDX[k * T + tid]) * SS;
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
    __syncthreads();
    // (3) accumulation: this thread's item over its share of the bucket
    if (ik >= 0) {
      const int p0 = BO[ik * (NB + 1) + is], p1 = BO[ik * (NB + 1) + is + 1];
      const float4* lw = LW + (size_t)ik * H * T;
      const float4* rh = RH + (size_t)ik * H * T;
      if (ik == 0 || ik == d - 1) {
        for (int p = p0 + ip; p < p1; p += np) {
          float lv[R], rv[R];
#pragma unroll
          for (int h = 0; h < H; ++h) {
            const float4 a4 = lw[(size_t)h * T + p];
            const float4 b4 = rh[(size_t)h * T + p];
            lv[4 * h] = a4.x; lv[4 * h + 1] = a4.y; lv[4 * h + 2] = a4.z; lv[4 * h + 3] = a4.w;
            rv[4 * h] = b4.x; rv[4 * h + 1] = b4.y; rv[4 * h + 2] = b4.z; rv[4 * h + 3] = b4.w;
          }
          if (ik == 0) {
#pragma unroll
            for (int b = 0; b < R; ++b) acc[0][b] = fmaf(lv[0], rv[b], acc[0][b]);
          } else {
#pragma unroll
            for (int a = 0; a < R; ++a) acc[a][0] = fmaf(lv[a], rv[0], acc[a][0]);
          }
        }
      } else {
        for (int p = p0 + ip; p < p1; p += np) {
          float lv[R], rv[R];
#pragma unroll
          for (int h = 0; h < H; ++h) {
            const float4 a4 = lw[(size_t)h * T + p];
            const float4 b4 = rh[(size_t)h * T + p];
            lv[4 * h] = a4.x; lv[4 * h + 1] = a4.y; lv[4 * h + 2] = a4.z; lv[4 * h + 3] = a4.w;
            rv[4 * h] = b4.x; rv[4 * h + 1] = b4.y; rv[4 * h + 2] = b4.z; rv[4 * h + 3] = b4.w;
          }
#pragma unroll
          for (int a = 0; a < R; ++a)
#pragma unroll
            for (int b = 0; b < R; ++b) acc[a][b] = fmaf(lv[a], rv[b], acc[a][b]);
        }
      }
    }
    __syncthreads();
  }
  // sum the parts of every (core, slice) in shared memory, then write the CTA's partial
  float* cacc = reinterpret_cast<float*>(RH);  // d * nmax * R * R floats (fits in RH)
  for (int e = tid; e < d * nmax * R * R; e += blockDim.x) cacc[e] = 0.0f;
  __syncthreads();
  if (ik >= 0) {
    float* dst = cacc + (ik * nmax + is) * R * R;
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
      for (int b = 0; b < R; ++b)
        if (acc[a][b] != 0.0f) atomicAdd(dst + a * R + b, acc[a][b]);
  }
  __syncthreads();
  float* out = g.grad_part + (long long)blockIdx.x * g.gsize;
  for (int k = 0; k < d; ++k) {
    const int ra = g.rl[k], rb = g.rr[k + 1], nk = g.n[k];
    for (int e = tid; e < ra * nk * rb; e += blockDim.x) {
      const int b = e % rb, i = (e / rb) % nk, a = e / (rb * nk);
      out[g.goff[k] + e] = cacc[(k * nmax + i) * R * R + a * R + b];
    }
  }
  if (g.loss_part) {
    double v = lsum;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (tid == 0) {
      double s2 = 0.0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s2 += red[i];
      g.loss_part[blockIdx.x] = s2;
    }
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

// SM count of the current device, looked up once per device index.
static int num_sms() { return device_sm_count(); }

struct GatherLayout {
  int R;
  int grid;
  size_t smem;
  size_t loss_off, grad_off, total;
  // bucketed adjoint
  int bucketed, T, NB;
  int parts[T3F_MAX_D];
  int item0[T3F_MAX_D + 1];
};

static size_t completion_smem(int d, int nmax, int R, int T, bool same) {
  const size_t SS = (size_t)R * R + 4;
  const int NB = nmax + 1, NW = (T + 31) / 32;
  size_t b = sizeof(float) * ((same ? 1 : 2) * (size_t)d * nmax * SS + 2 * (size_t)d * R * T);
  b += 2 * (size_t)d * T;                           // POS
  b += ((size_t)d * T + 15) & ~(size_t)15;          // IDX
  b += sizeof(unsigned short) * (((size_t)d * NB * NW + 1) & ~(size_t)1);  // WC (counts <= T)
  b += sizeof(int) * ((size_t)d * NB + (size_t)d * (NB + 1));
  return b;
}

// Choose the bucketed adjoint when its items fit one CTA and its buffers fit shared memory:
// the largest chunk T whose buffers let two CTAs share an SM (one CTA's barrier waits overlap
// the other's chains), else the largest that fits one CTA.
static bool plan_completion(const TTV& L, bool same, int R, GatherLayout* lay) {
  if (R > 8 || L.nmax > 254) return false;
  const int d = L.d;
  for (int pass = 0; pass < 2; ++pass)
  for (int T = 256; T >= 128; T -= 32) {
    if (L.nmax * R > T) continue;
    // two CTAs per SM: 228 KB per SM less 1 KB reserved and the static block per CTA
    const size_t cap = pass == 0 ? (228 * 1024 - 2 * 1200) / 2 : 220 * 1024;
    if (completion_smem(d, L.nmax, R, T, same) > cap) continue;
    // boundary cores take one item per slice, interior cores share the rest evenly
    int bnd = 0, inner = 0;
    for (int k = 0; k < d; ++k) {
      if (k == 0 || k == d - 1) bnd += L.n[k];
      else inner += L.n[k];
    }
    const int P2 = inner ? (T - bnd) / inner : 1;
    if (P2 < 1) continue;
    int it = 0;
    for (int k = 0; k < d; ++k) {
      lay->item0[k] = it;
      lay->parts[k] = (k == 0 || k == d - 1) ? 1 : P2;
      it += L.n[k] * lay->parts[k];
    }
    lay->item0[d] = it;
    if (it > T) continue;
    lay->bucketed = pass == 0 ? 2 : 1;  // CTAs per SM
    lay->T = T;
    lay->NB = L.nmax + 1;
    lay->smem = completion_smem(d, L.nmax, R, T, same);
    return true;
  }
  return false;
}

static GatherLayout gather_layout(const TTV& L, const TTV& Rv, long long N, bool bwd, bool same) {
  GatherLayout lay{};
  lay.R = pick_R(L.rmax > Rv.rmax ? L.rmax : Rv.rmax);
  const int R = lay.R ? lay.R : 16;
  const int nmax = L.nmax;
  if (!bwd) {
    // padded slices + the TMA landing zone of the packed object (rounded out to 16 bytes)
    const long long nfl = L.off[L.d - 1] + L.osz[L.d - 1];
    lay.smem = sizeof(float) * (size_t)L.d * nmax * (R * R + 4) + (size_t)((nfl * 4 + 12 + 15) / 16) * 16;
    lay.grid = gather_grid(N, num_sms() * 8);
  } else if (lay.R && plan_completion(L, same, R, &lay)) {
    long long g = (N + lay.T - 1) / lay.T;
    if (g > (long long)num_sms() * lay.bucketed) g = (long long)num_sms() * lay.bucketed;
    lay.grid = (int)(g < 1 ? 1 : g);
  } else {
    lay.smem = sizeof(float) * ((same ? 1 : 2) * (size_t)L.d * nmax * (R * R + 4) + (size_t)L.d * nmax * (R * R + 1) +
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
  g->Lnfl = L.off[L.d - 1] + L.osz[L.d - 1];
  g->Rnfl = Rv.off[Rv.d - 1] + Rv.osz[Rv.d - 1];
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
static t3f_status launch_completion(const GatherArgs& g, const GatherLayout& lay, cudaStream_t s) {
  CompletionArgs ca;
  memset(&ca, 0, sizeof(ca));
  ca.g = g;
  ca.T = lay.T;
  ca.NB = lay.NB;
  for (int k = 0; k < g.d; ++k) ca.parts[k] = lay.parts[k];
  for (int k = 0; k <= g.d; ++k) ca.item0[k] = lay.item0[k];
  auto kern = k_completion<R>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.smem) != cudaSuccess)
    return T3F_ERR_CUDA;
  kern<<<lay.grid, lay.T, lay.smem, s>>>(ca);
  return launch_status();
}

template <int R>
static t3f_status launch_bwd(const GatherArgs& g, const GatherLayout& lay, cudaStream_t s) {
  if (lay.bucketed) return launch_completion<(R <= 4 ? 4 : 8)>(g, lay, s);
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
  if (!lay.R || lay.smem > 227 * 1024) return T3F_ERR_UNSUPPORTED;
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
  if (!lay.R || lay.smem > 227 * 1024) return T3F_ERR_UNSUPPORTED;
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
    // the Riemannian form sums into partial slot 0 (every element is read before it is
    // written) and the gauge projection writes the output from there
    target = gp;
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
static std::mutex g_noalloc_mu[kNoAllocMaxDevices];
static void* g_noalloc_ptr[kNoAllocMaxDevices];

// Device address of the scratch array on the current device. The array's name in host
// code is only a host-side stand-in, so the address is looked up with that device current
// and cached per device. Only a successful lookup is cached: a failed one (for example a
// first call made while a stream is being captured) clears the runtime's pending error and
// is retried by the next call.
static t3f_status noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return T3F_ERR_CUDA;
  }
  if (dev < 0 || dev >= kNoAllocMaxDevices) return T3F_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mu[dev]);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return T3F_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
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

// The error word at the start of the shared scratch array: the device-side status of the
// last t3f_gather_noalloc call on this device (an index tuple out of range reads back as
// T3F_ERR_ARG). Synchronises `stream`.
extern "C" t3f_status t3f_gather_noalloc_status(t3f_stream_t stream) {
  void* scratch = nullptr;
  T3F_CHECK(noalloc_scratch(&scratch));
  return t3f_device_status(scratch, stream);
}
