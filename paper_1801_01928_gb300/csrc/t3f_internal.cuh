// Internal declarations shared by the translation units of libt3f (not part of the ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

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
