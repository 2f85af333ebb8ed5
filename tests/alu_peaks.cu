// alu_peaks.cu -- ALU throughput microbenchmark (test infrastructure): FP32 FMA, FP64 FMA and
// MUFU rsqrt rates of the whole GPU, the denominators of the ALU rooflines. Bounded loops, no waits.
#include <cstdio>
#include <cuda_runtime.h>
template<int ILP> __global__ void k32(float* out, int iters, float a, float b) {
  float x[ILP];
#pragma unroll
  for (int i = 0; i < ILP; i++) x[i] = (threadIdx.x + i) * 1e-3f;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < ILP; i++) x[i] = fmaf(x[i], a, b);
  }
  float s = 0; for (int i = 0; i < ILP; i++) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
template<int ILP> __global__ void k64(double* out, int iters, double a, double b) {
  double x[ILP];
#pragma unroll
  for (int i = 0; i < ILP; i++) x[i] = (threadIdx.x + i) * 1e-3;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < ILP; i++) x[i] = fma(x[i], a, b);
  }
  double s = 0; for (int i = 0; i < ILP; i++) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
template<int ILP> __global__ void kmufu(float* out, int iters, float b) {
  float x[ILP];
#pragma unroll
  for (int i = 0; i < ILP; i++) x[i] = 1.0f + (threadIdx.x + i) * 1e-3f;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < ILP; i++) x[i] = rsqrtf(x[i]) + b;
  }
  float s = 0; for (int i = 0; i < ILP; i++) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
// packed FP32x2 FMA (one instruction, two lanes' worth of FMAs)
template<int ILP> __global__ void k32x2(float* out, int iters, float a, float b) {
  float2 x[ILP];
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
  for (int i = 0; i < ILP; i++) x[i] = make_float2((threadIdx.x + i) * 1e-3f, (threadIdx.x + 2 * i) * 1e-3f);
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < ILP; i++) x[i] = __ffma2_rn(x[i], a2, b2);
  }
  float s = 0; for (int i = 0; i < ILP; i++) s += x[i].x + x[i].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
int main() {
  int dev = 0; cudaDeviceProp p; cudaGetDeviceProperties(&p, dev);
  int sms = p.multiProcessorCount;
  printf("{\"name\":\"%s\",\"sms\":%d", p.name, sms);
  const int threads = 256, blocksPerSm = 8, blocks = sms * blocksPerSm;
  float* o32; double* o64; cudaMalloc(&o32, blocks * threads * 4); cudaMalloc(&o64, blocks * threads * 8);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  float ms;
  for (int rep = 0; rep < 2; rep++) {
    int it32 = 20000;
    cudaEventRecord(e0); k32<8><<<blocks, threads>>>(o32, it32, 0.9999f, 1e-4f); cudaEventRecord(e1);
    cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    double f32 = 2.0 * 8 * it32 * (double)blocks * threads / (ms * 1e-3) / 1e12;
    int it64 = 500;
    cudaEventRecord(e0); k64<8><<<blocks, threads>>>(o64, it64, 0.9999, 1e-4); cudaEventRecord(e1);
    cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    double f64 = 2.0 * 8 * it64 * (double)blocks * threads / (ms * 1e-3) / 1e12;
    double ms64 = ms;
    int itm = 4000;
    cudaEventRecord(e0); kmufu<8><<<blocks, threads>>>(o32, itm, 1e-4f); cudaEventRecord(e1);
    cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    double mu = 8.0 * itm * (double)blocks * threads / (ms * 1e-3) / 1e12;
    cudaEventRecord(e0); k32x2<8><<<blocks, threads>>>(o32, it32, 0.9999f, 1e-4f); cudaEventRecord(e1);
    cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    double f32x2 = 4.0 * 8 * it32 * (double)blocks * threads / (ms * 1e-3) / 1e12;
    if (rep == 1) printf(",\"fp32_fma_tflops\":%.3f,\"fp32x2_fma_tflops\":%.3f,\"fp64_fma_tflops\":%.4f,\"fp64_ms\":%.2f,\"mufu_rsqrt_tops\":%.4f", f32, f32x2, f64, ms64, mu);
  }
  cudaError_t err = cudaGetLastError();
  printf(",\"err\":\"%s\"}\n", cudaGetErrorString(err));
  return err == cudaSuccess ? 0 : 1;
}
