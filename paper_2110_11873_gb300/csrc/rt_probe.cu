// Measurement aid: the FP64 fused multiply-add rate of this GPU.
//
// The paper has no counterpart.  The GMRES Arnoldi step and the FP64
// operator apply are bound by the FP64 pipe on this GPU, not by HBM, so their
// roofline needs that pipe's rate; this kernel measures it.  Every thread runs
// kChains independent dependent chains a = a*m + c, so the pipe always has
// independent work; nothing else is issued inside the loop.  The caller
// times the launch on its stream (CUDA events) and divides the FLOP count
// this entry point returns by the time.
#include "rt_common.cuh"

namespace rt {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;
constexpr int kProbeCtasPerSm = 4;

__global__ void __launch_bounds__(kProbeThreads) k_dfma_probe(int iters, double* __restrict__ sink) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  const double m = 0.9999999, k = 1e-7;   // a stays near 1: no overflow, no denormals
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, k);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (blockIdx.x == 0 && threadIdx.x == 0) sink[0] = s;   // keeps the chains live
}

}  // namespace
}  // namespace rt

using namespace rt;

extern "C" {

int64_t rt_probe_fp64_fma(int32_t iters, double* sink_dev, void* stream) {
  clear_error();
  if (iters < 1 || !sink_dev) {
    set_error("iters must be >= 1 and sink_dev non-NULL");
    return -1;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess) {
    set_error("no CUDA device");
    return -1;
  }
  const int grid = sms * kProbeCtasPerSm;
  k_dfma_probe<<<grid, kProbeThreads, 0, as_stream(stream)>>>(iters, sink_dev);
  RT_COUNT(1);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("k_dfma_probe launch failed: %s", cudaGetErrorString(e));
    return -1;
  }
  // 2 FLOP per fused multiply-add
  return (int64_t)grid * kProbeThreads * kChains * (int64_t)iters * 2;
}

}  // extern "C"
