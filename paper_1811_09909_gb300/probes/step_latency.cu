// Cost of one step of a persistent cooperative kernel whose steps are
// separated by a grid barrier (a monotonic arrival count: release add,
// acquire polls), as in the persistent V-cycle: 129 blocks of 1024 threads,
// a step of (a) the barrier alone, (b) two stores per thread, (c) sixteen
// loads of values other blocks wrote in the previous step plus two stores,
// (d) as (c) on the first 2112 threads only (a small level).  Every wait is
// bounded (200 ms of the global timer); an expired wait sets a flag and the
// kernel returns.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o step_latency step_latency.cu && ./step_latency
#include <cstdio>
#include <cuda_runtime.h>

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release(unsigned long long* p) {
  asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(p) : "memory");
}
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ bool grid_sync(unsigned long long* bar, unsigned long long& target, int* err,
                          volatile int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    target += gridDim.x;
    red_release(bar);
    int ok = 1;
    const unsigned long long t0 = now_ns();
    unsigned spin = 0;
    while (ld_acquire(bar) < target) {
      if ((++spin & 15u) == 0 && now_ns() - t0 > 200000000ull) {
        atomicOr(err, 1);
        ok = 0;
        break;
      }
    }
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

__global__ void __launch_bounds__(1024, 1) step_kernel(int mode, int steps, int active, int len,
                                                       float* buf, unsigned long long* bar,
                                                       int* err, unsigned long long* out) {
  __shared__ int s_ok;
  unsigned long long target = 0;
  if (threadIdx.x == 0) {
    const unsigned long long c0 = *(volatile unsigned long long*)bar;
    target = c0 - c0 % gridDim.x;
  }
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  if (!grid_sync(bar, target, err, &s_ok)) return;
  const unsigned long long t0 = now_ns();
  for (int s = 0; s < steps; ++s) {
    const float* src = buf + (size_t)(s & 1) * 2 * len;
    float* dst = buf + (size_t)((s + 1) & 1) * 2 * len;
    if (mode >= 1 && gid < (mode == 3 ? active : len)) {
      float v0 = 0.f, v1 = 0.f;
      if (mode >= 2) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          int j = gid + (c - 4) * 257 + c;
          j = j < 0 ? 0 : (j >= len ? len - 1 : j);
          v0 += src[j] * (1.f + c);
          v1 += src[len + j] * (2.f - c);
        }
      }
      dst[gid] = v0 + 1.f;
      dst[len + gid] = v1 - 1.f;
    }
    if (!grid_sync(bar, target, err, &s_ok)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[mode] = now_ns() - t0;
}

int main() {
  const int blocks = 129, len = 131584, steps = 2000;
  float* buf;
  unsigned long long *bar, *out;
  int* err;
  cudaMalloc(&buf, sizeof(float) * 4 * len);
  cudaMemset(buf, 0, sizeof(float) * 4 * len);
  cudaMalloc(&bar, 8);
  cudaMemset(bar, 0, 8);
  cudaMalloc(&out, 64);
  cudaMemset(out, 0, 64);
  cudaMalloc(&err, 4);
  cudaMemset(err, 0, 4);
  const char* names[] = {"barrier only", "2 stores + barrier", "16 loads + 2 stores (all threads)",
                         "16 loads + 2 stores (2112 threads)"};
  for (int rep = 0; rep < 2; ++rep)
    for (int mode = 0; mode < 4; ++mode) {
      int m = mode, st = steps, act = 2112, ln = len;
      void* args[] = {&m, &st, &act, &ln, &buf, &bar, &err, &out};
      cudaError_t e = cudaLaunchCooperativeKernel((void*)step_kernel, blocks, 1024, args, 0, 0);
      if (e == cudaSuccess) e = cudaDeviceSynchronize();
      if (e != cudaSuccess) {
        printf("%s\n", cudaGetErrorString(e));
        return 1;
      }
      unsigned long long h[8];
      int he = 0;
      cudaMemcpy(h, out, sizeof(h), cudaMemcpyDeviceToHost);
      cudaMemcpy(&he, err, 4, cudaMemcpyDeviceToHost);
      if (he) {
        printf("a barrier wait expired\n");
        return 1;
      }
      if (rep == 1) printf("%-40s %.3f us per step\n", names[mode], h[mode] / 1000.0 / steps);
    }
  return 0;
}
