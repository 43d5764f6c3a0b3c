// Arithmetic throughput of the device's FP64 and FP32 pipes, measured the way the sweep uses them
// (fused multiply-adds), for roofline accounting: the sweep kernels are bound by FP64 (or FP32)
// FMA issue, and this is their ceiling on the GPU at hand, at its current clocks.
//
// Every thread runs kChains independent FMA chains x <- x * a + b, so each warp always has
// independent FMAs to issue; the grid holds 4 blocks of 256 threads per SM.  The best of five
// launches, timed with CUDA events on the caller's stream, is reported.
#include "common.cuh"

namespace rte {
namespace {
constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(T* sink, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (T)-1.2345) sink[0] = s;   // never true; keeps the chains from being removed
}

template <typename T>
int probe(int iters, double* tflops, cudaStream_t st) {
  int dev = 0, sms = 0;
  RTE_CUDA_TRY(cudaGetDevice(&dev));
  RTE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = 4 * sms;
  DevBuf<T> sink;
  RTE_TRY(sink.alloc(1));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  RTE_CUDA_TRY(cudaEventCreate(&e0));
  int err = RTE_OK;
  float best = 1e30f;
  if (cudaEventCreate(&e1) != cudaSuccess) err = fail(RTE_ECUDA, "cudaEventCreate");
  for (int r = 0; r < 7 && err == RTE_OK; ++r) {   // two untimed launches, then five timed
    cudaEventRecord(e0, st);
    fma_probe_kernel<T><<<blocks, kProbeThreads, 0, st>>>(sink.p, iters, (T)0.999999, (T)1e-7); RTE_NOTE_LAUNCH();
    cudaEventRecord(e1, st);
    cudaError_t ce = cudaEventSynchronize(e1);
    if (ce == cudaSuccess) ce = cudaGetLastError();
    if (ce != cudaSuccess) {
      err = fail(RTE_ECUDA, std::string("FMA probe: ") + cudaGetErrorString(ce));
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r >= 2 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (err != RTE_OK) return err;
  *tflops = 2.0 * kChains * (double)blocks * kProbeThreads * iters / (best * 1e-3) / 1e12;
  return RTE_OK;
}
}  // namespace
}  // namespace rte

using namespace rte;

extern "C" int rte_fma_peak(int device, int kind, double* tflops, void* stream) {
  if (!tflops || (kind != 0 && kind != 1)) return fail(RTE_EINVAL, "rte_fma_peak: bad argument");
  int n_dev = 0;
  RTE_CUDA_TRY(cudaGetDeviceCount(&n_dev));
  if (device < 0 || device >= n_dev) return fail(RTE_EINVAL, "rte_fma_peak: no such device");
  DeviceGuard g(device);
  cudaStream_t st = (cudaStream_t)stream;
  // iteration counts sized for launches of a few milliseconds on GB300 (FP64 at ~1/64 the FP32 rate)
  return kind == 0 ? probe<double>(2000, tflops, st) : probe<float>(40000, tflops, st);
}
