// FP64 pipe throughput microbenchmark: the measured denominator behind the ALU roofline that
// bench.py reports for the WENO-theta kernels.  Dependent FMA chains per thread, swept over
// warps per SM and instruction-level parallelism, plus partial warps, DADD, DIV, SQRT and
// FP32 FMA for comparison.  Build and run on the GPU:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 -o fp64_peak fp64_peak.cu && ./fp64_peak
#include <cstdio>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { printf("CUDA error %s at %d\n", cudaGetErrorString(e_), __LINE__); return 1; } } while (0)

template <int ILP>
__global__ void k_dfma(double* out, int iters, double b, double c, int active_lanes) {
  if ((threadIdx.x & 31) >= active_lanes) return;
  double a[ILP];
#pragma unroll
  for (int k = 0; k < ILP; ++k) a[k] = threadIdx.x * 1e-3 + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < ILP; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0;
#pragma unroll
  for (int k = 0; k < ILP; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int ILP>
__global__ void k_dadd(double* out, int iters, double b, double c) {
  double a[ILP];
#pragma unroll
  for (int k = 0; k < ILP; ++k) a[k] = threadIdx.x * 1e-3 + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < ILP; ++k) a[k] = __dadd_rn(a[k], b);
  }
  double s = 0;
#pragma unroll
  for (int k = 0; k < ILP; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s + c;
}

template <int ILP>
__global__ void k_ddiv(double* out, int iters, double b, double c) {
  double a[ILP];
#pragma unroll
  for (int k = 0; k < ILP; ++k) a[k] = 1.0 + threadIdx.x * 1e-6 + k * 1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < ILP; ++k) a[k] = b / a[k];
  }
  double s = 0;
#pragma unroll
  for (int k = 0; k < ILP; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s + c;
}

template <int ILP>
__global__ void k_dsqrt(double* out, int iters, double b, double c) {
  double a[ILP];
#pragma unroll
  for (int k = 0; k < ILP; ++k) a[k] = 1.0 + threadIdx.x * 1e-6 + k * 1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < ILP; ++k) a[k] = sqrt(a[k] * b);
  }
  double s = 0;
#pragma unroll
  for (int k = 0; k < ILP; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s + c;
}

template <int ILP>
__global__ void k_ffma(float* out, int iters, float b, float c) {
  float a[ILP];
#pragma unroll
  for (int k = 0; k < ILP; ++k) a[k] = threadIdx.x * 1e-3f + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < ILP; ++k) a[k] = fmaf(a[k], b, c);
  }
  float s = 0;
#pragma unroll
  for (int k = 0; k < ILP; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int main() {
  int dev = 0;
  cudaDeviceProp p;
  CK(cudaGetDeviceProperties(&p, dev));
  int clk = 0, memclk = 0;
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  cudaDeviceGetAttribute(&memclk, cudaDevAttrMemoryClockRate, dev);
  printf("device %s sm_%d%d SMs=%d clock_kHz=%d l2=%d smem_per_block_optin=%zu regs_per_sm=%d\n", p.name, p.major, p.minor,
         p.multiProcessorCount, clk, p.l2CacheSize, p.sharedMemPerBlockOptin, p.regsPerMultiprocessor);
  const int sms = p.multiProcessorCount;
  double* d;
  float* f;
  CK(cudaMalloc(&d, sizeof(double) * sms * 1024 * 4));
  CK(cudaMalloc(&f, sizeof(float) * sms * 1024 * 4));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto timeit = [&](auto launch) {
    launch();
    cudaDeviceSynchronize();
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
      cudaEventRecord(e0);
      launch();
      cudaEventRecord(e1);
      cudaEventSynchronize(e1);
      float ms;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) best = ms;
    }
    return best;
  };
  const int iters = 4000;
  // DFMA vs warps per SM and ILP
  for (int wps : {1, 2, 4, 8, 16, 32}) {
    for (int ilp : {1, 4, 8}) {
      int threads = wps * 32;
      float ms;
      if (ilp == 1) ms = timeit([&] { k_dfma<1><<<sms, threads>>>(d, iters, 1.0000001, 1e-9, 32); });
      else if (ilp == 4) ms = timeit([&] { k_dfma<4><<<sms, threads>>>(d, iters, 1.0000001, 1e-9, 32); });
      else ms = timeit([&] { k_dfma<8><<<sms, threads>>>(d, iters, 1.0000001, 1e-9, 32); });
      double ops = (double)sms * threads * iters * ilp;
      printf("DFMA warps/SM=%2d ilp=%d: %.3f ms  %.1f Gfma/s  %.3f fma/clk/SM (at %d MHz)\n", wps, ilp, ms, ops / ms * 1e-6,
             ops / (ms * 1e-3) / sms / (clk * 1e3), clk / 1000);
    }
  }
  // partial warps
  for (int lanes : {1, 8, 16, 32}) {
    float ms = timeit([&] { k_dfma<4><<<sms, 16 * 32>>>(d, iters, 1.0000001, 1e-9, lanes); });
    double ops = (double)sms * 16 * lanes * iters * 4;
    printf("DFMA active lanes=%2d (16 warps/SM ilp4): %.3f ms  %.1f G lane-fma/s\n", lanes, ms, ops / ms * 1e-6);
  }
  {
    float ms = timeit([&] { k_dadd<4><<<sms, 16 * 32>>>(d, iters, 1e-9, 0.5); });
    double ops = (double)sms * 16 * 32 * iters * 4;
    printf("DADD 16 warps/SM ilp4: %.3f ms  %.1f Gop/s\n", ms, ops / ms * 1e-6);
  }
  for (int ilp : {1, 4}) {
    float ms = ilp == 1 ? timeit([&] { k_ddiv<1><<<sms, 16 * 32>>>(d, iters / 8, 1.0000001, 0.5); })
                        : timeit([&] { k_ddiv<4><<<sms, 16 * 32>>>(d, iters / 8, 1.0000001, 0.5); });
    double ops = (double)sms * 16 * 32 * (iters / 8) * ilp;
    printf("DDIV 16 warps/SM ilp%d: %.3f ms  %.2f Gdiv/s\n", ilp, ms, ops / ms * 1e-6);
  }
  for (int ilp : {1, 4}) {
    float ms = ilp == 1 ? timeit([&] { k_dsqrt<1><<<sms, 16 * 32>>>(d, iters / 8, 1.0000001, 0.5); })
                        : timeit([&] { k_dsqrt<4><<<sms, 16 * 32>>>(d, iters / 8, 1.0000001, 0.5); });
    double ops = (double)sms * 16 * 32 * (iters / 8) * ilp;
    printf("DSQRT 16 warps/SM ilp%d: %.3f ms  %.2f Gsqrt/s\n", ilp, ms, ops / ms * 1e-6);
  }
  {
    float ms = timeit([&] { k_ffma<8><<<sms, 16 * 32>>>(f, iters * 16, 1.0000001f, 1e-9f); });
    double ops = (double)sms * 16 * 32 * iters * 16 * 8;
    printf("FFMA 16 warps/SM ilp8: %.3f ms  %.1f Gfma/s\n", ms, ops / ms * 1e-6);
  }
  CK(cudaGetLastError());
  CK(cudaDeviceSynchronize());
  printf("done\n");
  return 0;
}
