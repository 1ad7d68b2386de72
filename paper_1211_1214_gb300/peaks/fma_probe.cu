// FMA throughput probe for the ALU roofline: each thread runs 8 independent FMA chains; prints TFLOP/s.
#include <cstdio>
#include <cuda_runtime.h>
template <typename T> __global__ void k(T *out, int iters, T a, T b) {
  T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; i++) {
    x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
    x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
template <typename T> void run(const char *name, int nsm) {
  int blocks = nsm * 8, threads = 256, iters = 1 << 14;
  T *out; cudaMalloc(&out, sizeof(T) * blocks * threads);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  for (int w = 0; w < 3; w++) k<T><<<blocks, threads>>>(out, iters, (T)0.999, (T)0.001);
  cudaEventRecord(e0);
  for (int w = 0; w < 5; w++) k<T><<<blocks, threads>>>(out, iters, (T)0.999, (T)0.001);
  cudaEventRecord(e1); cudaEventSynchronize(e1);
  float ms; cudaEventElapsedTime(&ms, e0, e1);
  double flops = 5.0 * blocks * threads * (double)iters * 8 * 2;
  printf("%s FMA throughput: %.2f TFLOP/s\n", name, flops / (ms * 1e-3) / 1e12);
  cudaFree(out);
}
int main() {
  cudaDeviceProp p; cudaGetDeviceProperties(&p, 0);
  printf("%s SMs=%d\n", p.name, p.multiProcessorCount);
  run<double>("fp64", p.multiProcessorCount);
  run<float>("fp32", p.multiProcessorCount);
  return 0;
}
