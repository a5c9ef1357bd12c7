// Measured arithmetic peaks of the current GPU: the FP32 and FP64 roofs that the hop kernels
// are compared against next to the HBM roof. Each thread runs eight independent fused
// multiply-add chains a <- a x + y (x just below 1, so the chains settle instead of overflowing),
// every SM holds as many threads as fit, and launches repeat until the requested time has
// passed; the rate is counted as two floating-point operations per multiply-add.
#include <algorithm>

#include "fs_engine.h"
#include "fsmlmc.h"

namespace {

constexpr int CHAINS = 8;
constexpr int THREADS = 256;

template <int KIND>
__global__ void __launch_bounds__(THREADS) peak_kernel(float* sink, int iters) {
  if constexpr (KIND == FS_PEAK_F64) {
    double a[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; c++) a[c] = 1e-3 * (threadIdx.x + c);
    const double x = 0.9999, y = 1e-7;
    for (int i = 0; i < iters; i++)
#pragma unroll
      for (int c = 0; c < CHAINS; c++) a[c] = __fma_rn(a[c], x, y);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CHAINS; c++) s += a[c];
    if (s == -1.0) sink[blockIdx.x] = (float)s;  // never true; keeps the chains live
  } else if constexpr (KIND == FS_PEAK_F32X2) {
    float2 a[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; c++) a[c] = make_float2(1e-3f * (threadIdx.x + c), 2e-3f * c);
    const float2 x = make_float2(0.9999f, 0.9999f), y = make_float2(1e-7f, 2e-7f);
    for (int i = 0; i < iters; i++)
#pragma unroll
      for (int c = 0; c < CHAINS; c++) a[c] = __ffma2_rn(a[c], x, y);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CHAINS; c++) s += a[c].x + a[c].y;
    if (s == -1.f) sink[blockIdx.x] = s;
  } else {
    float a[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; c++) a[c] = 1e-3f * (threadIdx.x + c);
    const float x = 0.9999f, y = 1e-7f;
    for (int i = 0; i < iters; i++)
#pragma unroll
      for (int c = 0; c < CHAINS; c++) a[c] = __fmaf_rn(a[c], x, y);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CHAINS; c++) s += a[c];
    if (s == -1.f) sink[blockIdx.x] = s;
  }
}

// multiply-adds per thread and iteration
int fma_per_iter(int kind) { return kind == FS_PEAK_F32X2 ? 2 * CHAINS : CHAINS; }

}  // namespace

extern "C" int fs_measure_peak(int kind, double seconds, double* tflops, double* elapsed_ms) {
  if (!tflops || !(seconds > 0.0) || seconds > 60.0) return FS_ERR_ARG;
  if (kind != FS_PEAK_F32 && kind != FS_PEAK_F32X2 && kind != FS_PEAK_F64) return FS_ERR_ARG;
  if (cudaPeekAtLastError() != cudaSuccess) return FS_ERR_CUDA;  // not ours to clear
  int dev = 0, nsm = 0, per_sm = 0;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float* sink = nullptr;
  auto kern = kind == FS_PEAK_F64 ? peak_kernel<FS_PEAK_F64>
                                  : (kind == FS_PEAK_F32X2 ? peak_kernel<FS_PEAK_F32X2> : peak_kernel<FS_PEAK_F32>);
  int rc = FS_OK;
  auto ok = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == FS_OK) rc = FS_ERR_CUDA;
    return rc == FS_OK;
  };
  if (ok(cudaGetDevice(&dev)) && ok(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) &&
      ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, 0)) &&
      ok(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) && ok(cudaEventCreate(&e0)) &&
      ok(cudaEventCreate(&e1))) {
    const int blocks = nsm * std::max(per_sm, 1);
    if (ok(cudaMalloc(&sink, sizeof(float) * blocks))) {
      // calibrate: one short launch, then size the launches to about 20 ms each
      int iters = 1 << 14;
      float ms = 0.f;
      kern<<<blocks, THREADS, 0, s>>>(sink, iters);
      ok(cudaGetLastError());
      if (ok(cudaEventRecord(e0, s))) {
        kern<<<blocks, THREADS, 0, s>>>(sink, iters);
        ok(cudaGetLastError());
      }
      if (ok(cudaEventRecord(e1, s)) && ok(cudaEventSynchronize(e1)) && ok(cudaEventElapsedTime(&ms, e0, e1))) {
        const double scale = std::min(64.0, std::max(1.0 / 64.0, 20.0 / std::max((double)ms, 1e-3)));
        iters = std::max(1, (int)(iters * scale));
        const int launches = std::max(1, (int)(seconds * 1000.0 / 20.0));
        double fmas = 0.0;
        if (ok(cudaEventRecord(e0, s))) {
          for (int k = 0; k < launches && rc == FS_OK; k++) {
            kern<<<blocks, THREADS, 0, s>>>(sink, iters);
            ok(cudaGetLastError());
            fmas += (double)blocks * THREADS * iters * fma_per_iter(kind);
          }
        }
        if (ok(cudaEventRecord(e1, s)) && ok(cudaEventSynchronize(e1)) && ok(cudaEventElapsedTime(&ms, e0, e1))) {
          *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
          if (elapsed_ms) *elapsed_ms = ms;
        }
        fs::note_launch(launches + 2);
      }
    }
  }
  if (sink) cudaFree(sink);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  return rc;
}
