// FP64 FMA throughput probe: the denominator of the operator's roofline.  The
// operator kernels are bound by FP64 arithmetic on this part, so their peak is
// measured here, under the same clocks as the kernels, instead of taken from
// a nominal figure.  No counterpart in the paper (a measurement aid).
#include "kernels.cuh"

namespace dg {

static __device__ double g_probe_sink;

// every thread runs kChains independent FMA chains for `iters` steps; the
// multiplier keeps the values bounded, the final test keeps the work alive
constexpr int kChains = 8;

__global__ void __launch_bounds__(256) fp64_fma_probe_kernel(int64_t iters, double seed) {
  double a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = seed + 1e-3 * j + 1e-9 * threadIdx.x;
  const double m = 0.999999, c = 1e-7;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (s == -1.0) g_probe_sink = s;   // never true; the compiler cannot know
}

}  // namespace dg

using namespace dg;

extern "C" dg_status dg_fp64_fma_probe(int64_t iters, double* tflops, double* ms, void* stream) {
  if (!tflops || !ms || iters < 1) {
    set_last_error("bad argument");
    return DG_EINVAL;
  }
  const cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  dg_status st = DG_OK;
  try {
    int dev = 0, sms = 0;
    DG_CUDA(cudaGetDevice(&dev));
    DG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = 8 * sms;   // 8 CTAs of 256 threads per SM: the whole FP64 pipe busy
    DG_CUDA(cudaEventCreate(&e0));
    DG_CUDA(cudaEventCreate(&e1));
    fp64_fma_probe_kernel<<<grid, 256, 0, s>>>(iters / 8 + 1, 1.0);   // warm-up
    DG_CUDA(cudaEventRecord(e0, s));
    fp64_fma_probe_kernel<<<grid, 256, 0, s>>>(iters, 1.0);
    DG_CUDA(cudaEventRecord(e1, s));
    DG_CUDA(cudaGetLastError());
    DG_CUDA(cudaEventSynchronize(e1));
    float t = 0.0f;
    DG_CUDA(cudaEventElapsedTime(&t, e0, e1));
    *ms = t;
    *tflops = 2.0 * kChains * (double)iters * (double)grid * 256.0 / (t * 1e-3) / 1e12;
    set_last_error("");
  } catch (const Error& e) {
    set_last_error(e.what());
    st = e.code;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return st;
}
