// FP64 / FP32 FMA throughput probe (not part of libh2gb): measures the
// float64 and float32 FMA rate of one GPU with full and partly masked warps;
// the float64 figure is the roofline denominator of the update kernels.
// Build: nvcc -gencode arch=compute_103a,code=sm_103a -O3 fp64_probe.cu
#include <cstdio>
#include <cuda_runtime.h>
template <typename T>
__global__ void fma_loop(T* out, int iters, int active_lanes, T b, T c) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  T a0 = tid, a1 = tid + 1, a2 = tid + 2, a3 = tid + 3, a4 = tid + 4, a5 = tid + 5, a6 = tid + 6, a7 = tid + 7;
  if (lane < active_lanes) {
    for (int i = 0; i < iters; ++i) {
      a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
      a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
    }
  }
  out[tid] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}
template <typename T>
double run(int blocks, int threads, int iters, int lanes) {
  T* out; cudaMalloc(&out, sizeof(T) * blocks * threads);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  fma_loop<T><<<blocks, threads>>>(out, iters, lanes, (T)0.999999, (T)1e-7);
  cudaDeviceSynchronize();
  cudaEventRecord(e0);
  for (int r = 0; r < 3; ++r) fma_loop<T><<<blocks, threads>>>(out, iters, lanes, (T)0.999999, (T)1e-7);
  cudaEventRecord(e1); cudaEventSynchronize(e1);
  float ms; cudaEventElapsedTime(&ms, e0, e1);
  cudaFree(out);
  double flops = 3.0 * blocks * threads * (double)iters * 8 * 2 * lanes / 32.0;
  return flops / (ms * 1e-3) / 1e12;
}
int main() {
  cudaDeviceProp p; cudaGetDeviceProperties(&p, 0);
  int sms = p.multiProcessorCount;
  printf("device %s sms %d\n", p.name, sms);
  for (int lanes : {32, 24, 16, 1}) {
    double t = run<double>(sms * 8, 256, 4096, lanes);
    printf("FP64 FMA lanes=%2d: %.3f TFLOP/s (useful)\n", lanes, t);
  }
  for (int lanes : {32, 24}) {
    double t = run<float>(sms * 8, 256, 65536, lanes);
    printf("FP32 FMA lanes=%2d: %.2f TFLOP/s (useful)\n", lanes, t);
  }
  cudaError_t e = cudaGetLastError();
  printf("status %s\n", cudaGetErrorString(e));
  return e == cudaSuccess ? 0 : 1;
}
