// Internal declarations shared by the translation units of libt3f (not part of the ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "t3f.h"

namespace t3f {

// Device view of a packed batch of TT objects, passed to kernels by value.
struct TTV {
  int d;
  int batch;
  int dtype;
  int is_matrix;
  int r[T3F_MAX_D + 1];
  int n[T3F_MAX_D];
  int m[T3F_MAX_D];                 // 1 for TT-vectors
  long long off[T3F_MAX_D];         // element offset of the block of core k
  long long osz[T3F_MAX_D];         // elements of core k of one object
  void* p;
  int rmax;                         // max_k r_k
  int nmax;                         // max_k n_k
};

// Host-side validation and conversion of a descriptor. `want_dtype` < 0 accepts any.
t3f_status make_view(const t3f_tt* t, TTV* v, int want_dtype, bool matrix_expected);

// Element offset of object b's core k.
__host__ __device__ inline long long core_base(const TTV& v, int k, int b) {
  return v.off[k] + (long long)b * v.osz[k];
}

template <typename T>
__device__ __forceinline__ float ldf(const T* p, long long i);
template <>
__device__ __forceinline__ float ldf<float>(const float* p, long long i) { return __ldg(p + i); }
template <>
__device__ __forceinline__ float ldf<__nv_bfloat16>(const __nv_bfloat16* p, long long i) {
  return __bfloat162float(p[i]);
}

// Workspace header: the first 256 bytes of every workspace hold the device error word.
constexpr size_t kWsHeader = 256;
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// SM count of the current device, looked up once per device index (152 when the lookup
// fails; the pending runtime error is then cleared).
inline int device_sm_count() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cache[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    cudaGetLastError();
    return 152;
  }
  int sms = cache[dev].load(std::memory_order_relaxed);
  if (sms <= 0) {
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
      cudaGetLastError();
      return 152;
    }
    cache[dev].store(sms, std::memory_order_relaxed);
  }
  return sms;
}

// Gauge projection of one core on its m x r1 unfolding, staged in shared memory (paper
// Section 3.2: out = Z - U (U^T Z), U with orthonormal columns): U and Z land with their
// columns zero-padded to R4 = r1 rounded up to 4; G = U^T Z is formed in 4 x 4 register
// blocks with the row range split over the threads left over (partial blocks summed in
// shared memory); each thread item of the update takes one row and four columns of Z - U G.
// Z is read completely before out is written, so out may alias Z. Every thread of the block
// calls it; sm holds gauge_staged_floats(m, r1) floats, 16-byte aligned.
__host__ __device__ inline int gauge_parts(int r1) {
  const int q = (r1 + 3) / 4, nb = q * q, p = 256 / nb;
  return p < 1 ? 1 : (p > 8 ? 8 : p);
}
__host__ __device__ inline long long gauge_staged_floats(int m, int r1) {
  const long long R4 = (r1 + 3) & ~3;
  return R4 * R4 * (1 + gauge_parts(r1)) + 2LL * m * R4;
}
__device__ __forceinline__ void gauge_core_staged(const float* Uk, const float* Zk, float* Ok, int m, int r1,
                                                  float* sm) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int R4 = (r1 + 3) & ~3, Q = R4 / 4, nblk = Q * Q, parts = gauge_parts(r1);
  float* G = sm;                        // R4 x R4
  float* Gp = G + R4 * R4;              // parts x R4 x R4 partial blocks
  float* Us = Gp + parts * R4 * R4;     // m x R4
  float* Zs = Us + m * R4;              // m x R4
  for (int e = tid; e < m * R4; e += nth) {
    const int q = e / R4, c = e - q * R4;
    Us[e] = c < r1 ? __ldg(Uk + q * r1 + c) : 0.0f;
    Zs[e] = c < r1 ? Zk[q * r1 + c] : 0.0f;
  }
  __syncthreads();
  for (int w = tid; w < nblk * parts; w += nth) {
    const int blk = w % nblk, p = w / nblk, ga = blk / Q, gb = blk - ga * Q;
    const int q0 = (int)(((long long)p * m) / parts), q1 = (int)(((long long)(p + 1) * m) / parts);
    float acc[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = 0.0f;
    for (int q = q0; q < q1; ++q) {
      const float4 u = *reinterpret_cast<const float4*>(Us + q * R4 + 4 * ga);
      const float4 z = *reinterpret_cast<const float4*>(Zs + q * R4 + 4 * gb);
      const float uv[4] = {u.x, u.y, u.z, u.w}, zv[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(uv[x], zv[y], acc[x][y]);
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
      *reinterpret_cast<float4*>(Gp + (size_t)p * R4 * R4 + (4 * ga + x) * R4 + 4 * gb) =
          make_float4(acc[x][0], acc[x][1], acc[x][2], acc[x][3]);
  }
  __syncthreads();
  for (int e = tid; e < R4 * R4; e += nth) {
    float s = 0.0f;
    for (int p = 0; p < parts; ++p) s += Gp[(size_t)p * R4 * R4 + e];
    G[e] = s;
  }
  __syncthreads();
  for (int w = tid; w < m * Q; w += nth) {
    const int q = w / Q, gb = w - q * Q;
    const float4 z = *reinterpret_cast<const float4*>(Zs + q * R4 + 4 * gb);
    float o[4] = {z.x, z.y, z.z, z.w};
    for (int a4 = 0; a4 < R4; a4 += 4) {
      const float4 u = *reinterpret_cast<const float4*>(Us + q * R4 + a4);
      const float uv[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        const float4 g = *reinterpret_cast<const float4*>(G + (a4 + x) * R4 + 4 * gb);
        o[0] = fmaf(-uv[x], g.x, o[0]);
        o[1] = fmaf(-uv[x], g.y, o[1]);
        o[2] = fmaf(-uv[x], g.z, o[2]);
        o[3] = fmaf(-uv[x], g.w, o[3]);
      }
    }
#pragma unroll
    for (int y = 0; y < 4; ++y)
      if (4 * gb + y < r1) Ok[q * r1 + 4 * gb + y] = o[y];
  }
}

t3f_status check_ws(void* ws, size_t ws_bytes, size_t need);
t3f_status launch_status();  // cudaGetLastError() mapped to a status

// Pair-sweep machinery (sweep.cu) -------------------------------------------------------
struct SweepPlan {
  int TA, TB;          // objects per tile on each side
  size_t smem;         // dynamic shared memory bytes
};
SweepPlan plan_sweep(const TTV& A, const TTV& B, int max_pairs);

// Left (dir = 0) or right (dir = 1) transfer sweep over all pairs (a, b) of A x B, tiled
// TA x TB. out[a * bB + b] receives <A_a, B_b> (nullable). store (nullable) receives the
// partial of every interface j = 0..d for every pair at store + ioff[j] + pair * rA_j rB_j.
t3f_status run_pair_sweep(const TTV& A, const TTV& B, int dir, float* out, float* store,
                          const long long* ioff, cudaStream_t s);

// Diagonal pairs (a, a): out[a] = <A_a, B_a> (A and B of equal batch).
t3f_status run_zip_sweep(const TTV& A, const TTV& B, float* out, cudaStream_t s);
// <A_a, A_a> for every object: whole-core staging when the cores fit, else the zip sweep.
t3f_status run_self_sweep(const TTV& A, float* out, cudaStream_t s);

// Interface offsets for a partial store of bA*bB pairs; returns total floats.
long long partial_offsets(const TTV& A, const TTV& B, long long pairs, long long* ioff);

// Gauge projection dU_k <- (I - U_k U_k^T) Z_k for k < d, copy for k = d (project.cu).
t3f_status run_gauge_project(const TTV& U, const float* Z, float* out, cudaStream_t s);

// Register-tiled project_sum sweeps (psweep.cu): X side ranks <= 32, Z ranks <= 8.
bool psweep_supported(const TTV& X, const TTV& Z);
// xtoff (right sweep only): A / B1 / B2 are transposed copies written by run_xtranspose, core k
// at xtoff[k]
t3f_status run_psweep(const TTV& X, const TTV& Z, int dir, const float* A, const float* B1, const float* B2,
                      float* st1, float* st2, const long long* ioff, cudaStream_t s, int* err = nullptr,
                      const long long* xtoff = nullptr);
// Transposed copies Y_k[c][i][r] = X_k[r][i][c] of nsets (<= 3) X-shaped TTs into dst (16-byte
// aligned; set t at t * xtranspose_offsets(X, nullptr) floats, core k at toff[k]).
long long xtranspose_offsets(const TTV& X, long long* toff);
t3f_status run_xtranspose(const TTV& X, const float* const* srcs, int nsets, float* dst, cudaStream_t s);
int passemble_ranges(const TTV& Z);
// Tensor-core (TF32) form of the project_sum sweeps (psweep_tc.cu): X ranks <= 32, Z ranks
// <= 8, modes 8 or 16; the left (U) and right (V) sweeps in one launch after a pre-pass that
// writes the per-core shared operands into img (psweep_tc_img_bytes(U) bytes of workspace).
bool psweep_tc_supported(const TTV& X, const TTV& Z);
size_t psweep_tc_img_bytes(const TTV& X);
t3f_status run_psweep_tc(const TTV& U, const TTV& V, const TTV& Z, float* stL, const long long* ioffL, float* stR,
                         const long long* ioffR, void* img, int* err, cudaStream_t s);
t3f_status run_passemble(const TTV& X, const TTV& Z, const float* L, const float* R, const long long* ioff,
                         const float* c, float* part, int nranges, cudaStream_t s);
t3f_status run_pgrad(const TTV& X, const TTV& Z, const float* U, const float* V, const float* W, const float* L,
                     const float* R, const float* P, const float* Q, const long long* ioff, const float* c, float* dZ,
                     float* dc, cudaStream_t s, const long long* xtoff = nullptr);

// Tiled Gram sweep (gram_tile.cu): ranks <= 64, F32 or BF16 cores.
bool gram_tile_supported(const TTV& A, const TTV& B);
t3f_status run_gram_tile(const TTV& A, const TTV& B, float* out, cudaStream_t s);

// Tensor-core Gram sweep (gram_mma.cu): TF32 (F32 cores) or BF16 (F32 or BF16 cores)
// operands, FP32 accumulation; ranks <= 64.
bool gram_mma_supported(const TTV& A, const TTV& B, int math);
t3f_status run_gram_mma(const TTV& A, const TTV& B, float* out, int math, int* err, cudaStream_t s);

// Tiled Gram adjoint (gram_tile_bwd.cu).
bool gram_tile_bwd_supported(const TTV& A, const TTV& B);
size_t ws_gram_tile_bwd(const TTV& A, const TTV& B);
t3f_status run_gram_tile_bwd(const TTV& A, const TTV& B, const float* dG, float* dA, float* dB, void* ws,
                             size_t ws_bytes, cudaStream_t s);

// Workspace sizes (bytes, header included) of the operations.
size_t ws_gram_bwd(const TTV& A, const TTV& B);
size_t ws_norm(const TTV& A);
size_t ws_gather(const TTV& X, long long N, bool bwd);
size_t ws_rgather(const TTV& U, const TTV& V, long long N);
size_t ws_orth(const TTV& X);
size_t ws_psum(const TTV& U, const TTV& Z, bool bwd);
size_t ws_project(const TTV& U, const TTV& Z);
size_t ws_tangent_gram(const TTV& A, const TTV& B);
size_t ws_completion_hvp(const TTV& U, const TTV& V, long long N);

// tensor-core Gram adjoint (gram_mma_bwd.cu): the sweeps' partial slots and the gradient products
size_t gram_tc_bwd_tiles(const TTV& A, const TTV& B);
long long gram_tc_bwd_slots(const TTV& A);
size_t ws_gram_bwd_tc(const TTV& A, const TTV& B);
t3f_status run_gram_tc_backward(const TTV& A, const TTV& B, const float* dG, float* dA, float* dB, int math,
                                char* scr, int* err, cudaStream_t s);
size_t ws_round(const TTV& X);

// Deterministic two-level sum of nsplit partial arrays of `size` floats (tangent.cu); mid
// holds ws_split_reduce(size) bytes.
t3f_status run_split_reduce(const float* part, int nsplit, long long size, float* mid, float* G, cudaStream_t s);
size_t ws_split_reduce(long long size);

// TF32 tensor-core Gram of tangent coordinates fed by TMA (tgram_tc.cu).
size_t ws_tangent_gram_tc(const TTV& A, const TTV& B);
t3f_status run_tangent_gram_tc(const TTV& A, const TTV& B, float* G, void* ws, size_t ws_bytes, cudaStream_t s);

}  // namespace t3f

#define T3F_CHECK(x)                       \
  do {                                     \
    t3f_status _st = (x);                  \
    if (_st != T3F_OK) return _st;         \
  } while (0)
