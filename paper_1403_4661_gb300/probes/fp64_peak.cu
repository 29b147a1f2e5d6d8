// Throughput probe of the float64 pipe (FFMA64, DMMA m8n8k4) and FFMA32 on the current GPU; the
// roofline denominator of the float64 contractions.  Not part of libsht.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fp64_peak paper_1403_4661_gb300/probes/fp64_peak.cu && ./fp64_peak
#include <cstdio>
#include <cuda_runtime.h>
__global__ void ffma64(double *out, int iters, double a, double b) {
  double x[8];
  for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
  }
  double s = 0; for (int i = 0; i < 8; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void dmma(double *out, int iters) {
  double a = threadIdx.x * 1e-3, b = 1.0 + threadIdx.x * 1e-4;
  double c[4][2] = {};
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(c[i][0]), "+d"(c[i][1]) : "d"(a), "d"(b));
  }
  double s = 0; for (int i = 0; i < 4; ++i) s += c[i][0] + c[i][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void ffma32(float *out, int iters, float a, float b) {
  float x[8];
  for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 1e-3f + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], a, b);
  }
  float s = 0; for (int i = 0; i < 8; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
int main() {
  int blocks = 152 * 8, threads = 256;
  double *out; cudaMalloc(&out, sizeof(double) * blocks * threads);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  float ms;
  for (int rep = 0; rep < 2; ++rep) {
    int iters = 4096;
    cudaEventRecord(e0); ffma64<<<blocks, threads>>>(out, iters, 0.999, 1e-3); cudaEventRecord(e1);
    cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    double fl = 2.0 * 8 * iters * (double)blocks * threads;
    printf("FFMA64: %.3f ms  %.3f TFLOP/s\n", ms, fl / ms / 1e9);
    cudaEventRecord(e0); dmma<<<blocks, threads>>>(out, 1024); cudaEventRecord(e1);
    cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    fl = 2.0 * 8 * 8 * 4 * 4 * 1024.0 * (blocks * threads / 32);
    printf("DMMA m8n8k4: %.3f ms  %.3f TFLOP/s\n", ms, fl / ms / 1e9);
    cudaEventRecord(e0); ffma32<<<blocks, threads>>>((float *)out, 65536, 0.999f, 1e-3f); cudaEventRecord(e1);
    cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    fl = 2.0 * 8 * 65536.0 * (double)blocks * threads;
    printf("FFMA32: %.3f ms  %.3f TFLOP/s\n", ms, fl / ms / 1e9);
  }
  printf("err %s\n", cudaGetErrorString(cudaGetLastError()));
  return 0;
}
