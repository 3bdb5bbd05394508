// Latency probe behind the persistent V-cycle: the cost of one grid-wide
// barrier in a cooperative launch (a monotonic arrival count with release
// adds and acquire polls, per-block flags polled by one warp, and
// cooperative_groups' grid sync for comparison) against the cost of one
// kernel boundary inside a CUDA graph.  Every wait is bounded by a spin
// count; out[0] records an expired wait.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o bar_bench bar_bench.cu && ./bar_bench
#include <cstdio>
#include <cuda_runtime.h>
#include <cooperative_groups.h>
namespace cg = cooperative_groups;

__device__ __forceinline__ unsigned long long ldacq(const unsigned long long* p) {
  unsigned long long v; asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory"); return v;
}
__device__ __forceinline__ void redrel(unsigned long long* p) {
  asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(p) : "memory");
}
__device__ __forceinline__ void strel(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// (a) monotonic counter, red.release + ld.acquire poll by thread 0
__global__ void k_counter(unsigned long long* cnt, int iters, int* out) {
  __shared__ unsigned long long tgt;
  if (threadIdx.x == 0) { unsigned long long c0 = *(volatile unsigned long long*)cnt; tgt = c0 - c0 % gridDim.x; }
  __syncthreads();
  for (int k = 0; k < iters; ++k) {
    __syncthreads();
    if (threadIdx.x == 0) {
      tgt += gridDim.x;
      redrel(cnt);
      unsigned spin = 0;
      while (ldacq(cnt) < tgt) { if (++spin > (1u << 22)) { out[0] = 1; break; } }
    }
    __syncthreads();
  }
}

// (b) per-block flags, warp 0 polls all flags
__global__ void k_flags(unsigned long long* flags, int iters, int* out, int stride) {
  __shared__ unsigned long long f0;
  if (threadIdx.x == 0) f0 = *(volatile unsigned long long*)&flags[blockIdx.x * stride];
  __syncthreads();
  for (int k = 0; k < iters; ++k) {
    __syncthreads();
    if (threadIdx.x < 32) {
      const unsigned long long want = f0 + k + 1;
      if (threadIdx.x == 0) strel(&flags[blockIdx.x * stride], want);
      unsigned spin = 0;
      for (;;) {
        bool ok = true;
        for (int b = threadIdx.x; b < gridDim.x; b += 32) ok &= ldacq(&flags[b * stride]) >= want;
        if (__all_sync(0xffffffffu, ok)) break;
        if (++spin > (1u << 22)) { out[0] = 2; break; }
      }
    }
    __syncthreads();
  }
}

// (c) cooperative groups grid sync
__global__ void k_cg(int iters) {
  cg::grid_group g = cg::this_grid();
  for (int k = 0; k < iters; ++k) g.sync();
}

__global__ void k_empty() {}

int main() {
  int sms = 0; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  unsigned long long* cnt; int* out;
  cudaMalloc(&cnt, 8 * 4096); cudaMemset(cnt, 0, 8 * 4096);
  cudaMalloc(&out, 4); cudaMemset(out, 0, 4);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  const int iters = 2000;
  for (int threads : {1024, 512}) {
    for (int blocks : {sms, sms / 2, 16}) {
      float ms;
      void* args1[] = {&cnt, (void*)&iters, &out};
      for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0);
        cudaLaunchCooperativeKernel((void*)k_counter, blocks, threads, args1, 0, 0);
        cudaEventRecord(e1); cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
      }
      printf("counter  blocks %3d thr %4d: %.3f us/barrier (%s)\n", blocks, threads, ms * 1e3 / iters, cudaGetErrorString(cudaGetLastError()));
      for (int stride : {1, 16}) {
        cudaMemset(cnt, 0, 8 * 4096);
        void* args2[] = {&cnt, (void*)&iters, &out, &stride};
        for (int rep = 0; rep < 2; ++rep) {
          cudaEventRecord(e0);
          cudaLaunchCooperativeKernel((void*)k_flags, blocks, threads, args2, 0, 0);
          cudaEventRecord(e1); cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
        }
        printf("flags(s%2d) blocks %3d thr %4d: %.3f us/barrier (%s)\n", stride, blocks, threads, ms * 1e3 / iters, cudaGetErrorString(cudaGetLastError()));
      }
      void* args3[] = {(void*)&iters};
      for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0);
        cudaLaunchCooperativeKernel((void*)k_cg, blocks, threads, args3, 0, 0);
        cudaEventRecord(e1); cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
      }
      printf("cg.sync  blocks %3d thr %4d: %.3f us/barrier (%s)\n", blocks, threads, ms * 1e3 / iters, cudaGetErrorString(cudaGetLastError()));
      cudaMemset(cnt, 0, 8 * 4096);
    }
  }
  // graph of N empty kernels
  cudaStream_t s; cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  cudaGraph_t g; cudaGraphExec_t ge;
  cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
  for (int i = 0; i < 200; ++i) k_empty<<<152, 1024, 0, s>>>();
  cudaStreamEndCapture(s, &g);
  cudaGraphInstantiate(&ge, g, 0);
  float ms;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, s); cudaGraphLaunch(ge, s); cudaEventRecord(e1, s);
    cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
  }
  printf("graph empty kernel 152x1024: %.3f us/launch\n", ms * 1e3 / 200);
  // the same through cudaLaunchKernelEx, with and without the cooperative attribute
  for (int coop = 0; coop < 2; ++coop) {
    cudaGraph_t g2; cudaGraphExec_t ge2;
    cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
    for (int i = 0; i < 200; ++i) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(sms); cfg.blockDim = dim3(1024); cfg.stream = s;
      cudaLaunchAttribute a[1]; a[0].id = cudaLaunchAttributeCooperative; a[0].val.cooperative = coop;
      cfg.attrs = a; cfg.numAttrs = 1;
      cudaLaunchKernelEx(&cfg, k_empty);
    }
    cudaStreamEndCapture(s, &g2);
    cudaGraphInstantiate(&ge2, g2, 0);
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, s); cudaGraphLaunch(ge2, s); cudaEventRecord(e1, s);
      cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    }
    printf("graph kernel (cooperative=%d) %dx1024: %.3f us/launch (%s)\n", coop, sms, ms * 1e3 / 200,
           cudaGetErrorString(cudaGetLastError()));
  }
  int h = 0; cudaMemcpy(&h, out, 4, cudaMemcpyDeviceToHost);
  printf("timeouts flag %d\n", h);
  return 0;
}
