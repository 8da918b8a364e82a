// Throughput probes of the GPU's FP64 units: the measured denominators of the roofline that the
// benchmark reports for the FP64 reduction (whose contractions are DFMA loops, see kernels.cu).  The
// paper has no counterpart; these kernels are measurement support only and never run in a reduction.
//
//   dfma_loop: every thread runs kChains independent FMA chains x <- x a + b (2 flops each), so the
//              FP64 pipe, not the FMA latency, bounds the rate.
//   dmma_loop: every warp runs kChains independent chains of mma.sync m8n8k4 f64 (8 x 8 x 4 products,
//              512 flops per warp instruction), the FP64 tensor-core path of the ISA.
// Both write one value per thread so that the compiler keeps every chain.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/bidiag.h"

namespace {

constexpr int kChains = 8;
constexpr int kBlock = 256;

__global__ void __launch_bounds__(kBlock) dfma_loop(double* out, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kBlock) dmma_loop(double* out, int iters, double a, double b) {
  double c[kChains][2];
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    c[k][0] = 1e-3 * k;
    c[k][1] = 2e-3 * k;
  }
  const double av = a * (1.0 + 1e-6 * (threadIdx.x & 31)), bv = b;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(c[k][0]), "+d"(c[k][1])
                   : "d"(av), "d"(bv));
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += c[k][0] + c[k][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Best-of-`reps` rate (GFLOP/s) of one probe kernel on stream st.
template <typename K>
cudaError_t time_probe(K kernel, int grid, int iters, double flops, double* out, cudaStream_t st, int reps,
                       double* gflops) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double best = 0.0;
  for (int r = 0; r <= reps && e == cudaSuccess; ++r) {   // r = 0 is the warm-up
    if ((e = cudaEventRecord(e0, st)) != cudaSuccess) break;
    kernel<<<grid, kBlock, 0, st>>>(out, iters, 0.9999999, 1e-7);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = cudaEventRecord(e1, st)) != cudaSuccess) break;
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
    float ms = 0.f;
    if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
    if (r > 0 && ms > 0.f) best = std::max(best, flops / (ms * 1e-3) / 1e9);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  *gflops = best;
  return e;
}

}  // namespace

extern "C" int bidiag_measure_fp64_peaks(int device, void* cuda_stream, double* gflops_fma, double* gflops_mma) {
  if (!gflops_fma) return -3;
  if (!gflops_mma) return -4;
  int nsm = 0;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return e == cudaErrorInvalidDevice ? -1 : BIDIAG_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int grid = nsm * 4;          // four 256-thread blocks per SM: 32 warps, enough to fill the pipes
  double* out = nullptr;
  if (cudaMalloc(&out, (size_t)grid * kBlock * sizeof(double)) != cudaSuccess) return BIDIAG_ERR_NOMEM;
  // about 60 GFLOP per DFMA launch and 80 GFLOP per MMA launch: tens of milliseconds each
  const int it_fma = 24000, it_mma = 1200;
  const double f_fma = 2.0 * kChains * (double)it_fma * grid * kBlock;
  const double f_mma = 512.0 * kChains * (double)it_mma * grid * (kBlock / 32);
  e = time_probe(dfma_loop, grid, it_fma, f_fma, out, st, 5, gflops_fma);
  if (e == cudaSuccess) e = time_probe(dmma_loop, grid, it_mma, f_mma, out, st, 5, gflops_mma);
  cudaFree(out);
  return e == cudaSuccess ? BIDIAG_OK : BIDIAG_ERR_CUDA;
}
