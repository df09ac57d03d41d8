// Arithmetic-rate probe for the design of the F-map kernels: FP64 FMA, FP32 FMA
// and MUFU.EX2 throughput of the current GPU (register-only loops, no memory
// traffic).  Build and run: python -m paper_1805_05652_gb300.probes
#include <cstdio>
#include <cuda_runtime.h>
template <typename T>
__global__ void k_fma(T* out, int iters, T a, T b) {
  T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
    x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
  }
  if (x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7 == (T)-1.2345) out[0] = x0;
}
__global__ void k_ex2(float* out, int iters, float a) {
  float x0 = threadIdx.x * 1e-3f, x1 = x0 + 0.1f, x2 = x0 + 0.2f, x3 = x0 + 0.3f;
  for (int i = 0; i < iters; ++i) {
    asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(x0)); asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(x1));
    asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(x2)); asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(x3));
    x0 *= a; x1 *= a; x2 *= a; x3 *= a;
  }
  if (x0 + x1 + x2 + x3 == -1.2345f) out[0] = x0;
}
int main() {
  int dev = 0, sms = 0, clk = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  float* of; double* od; cudaMalloc(&of, 64); cudaMalloc(&od, 64);
  cudaEvent_t a, b; cudaEventCreate(&a); cudaEventCreate(&b);
  const int blocks = sms * 8, threads = 256;
  for (int rep = 0; rep < 2; ++rep) {
    int it = 4096;
    cudaEventRecord(a); k_fma<double><<<blocks, threads>>>(od, it, 0.999, 1e-3); cudaEventRecord(b); cudaEventSynchronize(b);
    float ms; cudaEventElapsedTime(&ms, a, b);
    double n = (double)blocks * threads * it * 8;
    printf("DFMA: %.3f TFLOP/s  (%.2f /clk/SM at %d MHz attr)\n", 2 * n / ms / 1e9, n / (ms * 1e-3) / sms / (clk * 1e3), clk / 1000);
    it = 1 << 16;
    cudaEventRecord(a); k_fma<float><<<blocks, threads>>>(of, it, 0.999f, 1e-3f); cudaEventRecord(b); cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms, a, b);
    n = (double)blocks * threads * it * 8;
    printf("FFMA: %.3f TFLOP/s  (%.2f /clk/SM)\n", 2 * n / ms / 1e9, n / (ms * 1e-3) / sms / (clk * 1e3));
    it = 1 << 14;
    cudaEventRecord(a); k_ex2<<<blocks, threads>>>(of, it, 0.5f); cudaEventRecord(b); cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms, a, b);
    n = (double)blocks * threads * it * 4;
    printf("EX2: %.3f Tops/s  (%.2f /clk/SM)\n", n / ms / 1e9, n / (ms * 1e-3) / sms / (clk * 1e3));
  }
  printf("SMs %d, clock attr %d kHz, err %s\n", sms, clk, cudaGetErrorString(cudaGetLastError()));
  return 0;
}
