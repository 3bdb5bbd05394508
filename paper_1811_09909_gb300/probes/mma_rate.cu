// Throughput probe behind the precision and tensor-pipe choices of the
// library: FP64 FMA against FP64 MMA (mma.sync m8n8k4 f64), FP32 FMA, and the
// TF32 / BF16 mma.sync paths.  Every warp runs independent chains of one
// instruction with no memory traffic; the third of three timed repetitions is
// reported (CUDA events), flops counted as 2 per multiply-add.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o mma_rate mma_rate.cu && ./mma_rate
#include <cstdio>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

template <int CH>
__global__ void dfma_k(double* out, int iters, double a, double b) {
  double acc[CH];
#pragma unroll
  for (int i = 0; i < CH; ++i) acc[i] = threadIdx.x * 1e-9 + i;
  for (int k = 0; k < iters; ++k)
#pragma unroll
    for (int i = 0; i < CH; ++i) acc[i] = fma(acc[i], a, b);
  double s = 0;
#pragma unroll
  for (int i = 0; i < CH; ++i) s += acc[i];
  if (s == 12345.678) out[0] = s;
}
template <int CH>
__global__ void ffma_k(float* out, int iters, float a, float b) {
  float acc[CH];
#pragma unroll
  for (int i = 0; i < CH; ++i) acc[i] = threadIdx.x * 1e-9f + i;
  for (int k = 0; k < iters; ++k)
#pragma unroll
    for (int i = 0; i < CH; ++i) acc[i] = fmaf(acc[i], a, b);
  float s = 0;
#pragma unroll
  for (int i = 0; i < CH; ++i) s += acc[i];
  if (s == 12345.678f) out[0] = s;
}
// m8n8k4 f64: A 8x4 (1 double per lane), B 4x8 (1 per lane), C/D 8x8 (2 per lane)
template <int CH>
__global__ void dmma_k(double* out, int iters, double a, double b) {
  double c[CH][2];
#pragma unroll
  for (int i = 0; i < CH; ++i) { c[i][0] = threadIdx.x; c[i][1] = i; }
  const double av = a + threadIdx.x * 1e-9, bv = b;
  for (int k = 0; k < iters; ++k)
#pragma unroll
    for (int i = 0; i < CH; ++i)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(c[i][0]), "+d"(c[i][1]) : "d"(av), "d"(bv));
  double s = 0;
#pragma unroll
  for (int i = 0; i < CH; ++i) s += c[i][0] + c[i][1];
  if (s == 12345.678) out[0] = s;
}
// m16n8k8 tf32: A 4 regs, B 2 regs, C 4 floats
template <int CH>
__global__ void tf32_k(float* out, int iters, float a, float b) {
  float c[CH][4];
#pragma unroll
  for (int i = 0; i < CH; ++i) for (int j = 0; j < 4; ++j) c[i][j] = j;
  unsigned A0 = __float_as_uint(a), B0 = __float_as_uint(b);
  for (int k = 0; k < iters; ++k)
#pragma unroll
    for (int i = 0; i < CH; ++i)
      asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                   : "+f"(c[i][0]), "+f"(c[i][1]), "+f"(c[i][2]), "+f"(c[i][3])
                   : "r"(A0), "r"(A0), "r"(A0), "r"(A0), "r"(B0), "r"(B0));
  float s = 0;
#pragma unroll
  for (int i = 0; i < CH; ++i) s += c[i][0] + c[i][1] + c[i][2] + c[i][3];
  if (s == 12345.678f) out[0] = s;
}
// m16n8k16 bf16
template <int CH>
__global__ void bf16_k(float* out, int iters, float a, float b) {
  float c[CH][4];
#pragma unroll
  for (int i = 0; i < CH; ++i) for (int j = 0; j < 4; ++j) c[i][j] = j;
  __nv_bfloat162 av = __floats2bfloat162_rn(a, a), bv = __floats2bfloat162_rn(b, b);
  unsigned A0 = *reinterpret_cast<unsigned*>(&av), B0 = *reinterpret_cast<unsigned*>(&bv);
  for (int k = 0; k < iters; ++k)
#pragma unroll
    for (int i = 0; i < CH; ++i)
      asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                   : "+f"(c[i][0]), "+f"(c[i][1]), "+f"(c[i][2]), "+f"(c[i][3])
                   : "r"(A0), "r"(A0), "r"(A0), "r"(A0), "r"(B0), "r"(B0));
  float s = 0;
#pragma unroll
  for (int i = 0; i < CH; ++i) s += c[i][0] + c[i][1] + c[i][2] + c[i][3];
  if (s == 12345.678f) out[0] = s;
}

int main() {
  int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  double* d; cudaMalloc(&d, 64); float* f = (float*)d;
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  const int blocks = sms * 4, thr = 256;
  const double warps = (double)blocks * thr / 32;
  auto run = [&](const char* name, auto fn, double flop_per_iter_per_warp, int iters) {
    float ms = 0;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0); fn(iters); cudaEventRecord(e1); cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
    }
    const double tflops = flop_per_iter_per_warp * iters * warps / (ms * 1e-3) / 1e12;
    printf("%-28s %8.3f ms  %9.2f TFLOP/s  (%s)\n", name, ms, tflops, cudaGetErrorString(cudaGetLastError()));
  };
  const int it = 20000;
  run("DFMA (8 chains)", [&](int n) { dfma_k<8><<<blocks, thr>>>(d, n, 1.0000001, 1e-9); }, 32.0 * 8 * 2, it / 4);
  run("DFMA (16 chains)", [&](int n) { dfma_k<16><<<blocks, thr>>>(d, n, 1.0000001, 1e-9); }, 32.0 * 16 * 2, it / 4);
  run("DMMA m8n8k4 (4 chains)", [&](int n) { dmma_k<4><<<blocks, thr>>>(d, n, 1.0000001, 1e-9); }, 8.0 * 8 * 4 * 2 * 4, it / 4);
  run("DMMA m8n8k4 (8 chains)", [&](int n) { dmma_k<8><<<blocks, thr>>>(d, n, 1.0000001, 1e-9); }, 8.0 * 8 * 4 * 2 * 8, it / 4);
  run("FFMA (8 chains)", [&](int n) { ffma_k<8><<<blocks, thr>>>(f, n, 1.0000001f, 1e-9f); }, 32.0 * 8 * 2, it * 4);
  run("FFMA (16 chains)", [&](int n) { ffma_k<16><<<blocks, thr>>>(f, n, 1.0000001f, 1e-9f); }, 32.0 * 16 * 2, it * 4);
  run("TF32 mma.sync m16n8k8 (4)", [&](int n) { tf32_k<4><<<blocks, thr>>>(f, n, 1.0f, 1e-3f); }, 16.0 * 8 * 8 * 2 * 4, it);
  run("BF16 mma.sync m16n8k16 (4)", [&](int n) { bf16_k<4><<<blocks, thr>>>(f, n, 1.0f, 1e-3f); }, 16.0 * 8 * 16 * 2 * 4, it);
  int clk; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
  printf("SMs %d, max clock %d MHz\n", sms, clk / 1000);
  return 0;
}
