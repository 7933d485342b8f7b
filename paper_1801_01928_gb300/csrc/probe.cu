// FP32 FMA throughput probe: the denominator of the CUDA-core roofline, measured on the GPU
// at hand instead of derived from the nominal clock. Each thread runs 8 independent FMA
// chains (enough instruction-level parallelism to keep the FMA pipes busy at full
// occupancy); the result is written so that the compiler keeps every chain.
#include "t3f_internal.cuh"

namespace t3f {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(long long iters, T seed, T* out) {
  T a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = seed + (T)1e-3 * (T)(threadIdx.x + j);
  const T m = (T)0.999999, c = (T)1e-7;
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int j = 0; j < 8; ++j) a[j] = fma(a[j], m, c);
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace t3f

using namespace t3f;

// FLOPs executed by one t3f_fma_probe (or t3f_fma_probe_f64) launch:
// grid * 256 threads * iters * 16 * 8 FMAs * 2.
extern "C" double t3f_fma_probe_flops(int32_t grid, int64_t iters) {
  return (double)grid * 256.0 * (double)iters * 16.0 * 8.0 * 2.0;
}

// Launch the FMA probe: `grid` CTAs of 256 threads (use a multiple of the SM count), `iters`
// outer iterations; out: device float [grid * 256].
extern "C" t3f_status t3f_fma_probe(int32_t grid, int64_t iters, float* out, t3f_stream_t stream) {
  if (grid < 1 || iters < 1 || !out) return T3F_ERR_ARG;
  k_fma_probe<float><<<grid, 256, 0, (cudaStream_t)stream>>>(iters, 1.0f, out);
  return launch_status();
}

// The same probe in FP64 (DFMA); out: device double [grid * 256].
extern "C" t3f_status t3f_fma_probe_f64(int32_t grid, int64_t iters, double* out, t3f_stream_t stream) {
  if (grid < 1 || iters < 1 || !out) return T3F_ERR_ARG;
  k_fma_probe<double><<<grid, 256, 0, (cudaStream_t)stream>>>(iters, 1.0, out);
  return launch_status();
}
