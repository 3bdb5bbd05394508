// Device helpers shared by the multigrid kernels: mesh numbering and packed
// symmetric indexing (see internal.h for the layouts).
#pragma once

#include "internal.h"

namespace hdgmg {

static __device__ __forceinline__ void elem_edges(int n, int e, int ed[4]) {
  const int j = e / n, i = e - j * n;
  const int nvert = n * (n + 1);
  ed[0] = j * (n + 1) + i;
  ed[1] = j * (n + 1) + i + 1;
  ed[2] = nvert + j * n + i;
  ed[3] = nvert + (j + 1) * n + i;
}

static __device__ __forceinline__ bool bnd_edge(int n, int edge) {
  const int nvert = n * (n + 1);
  if (edge < nvert) {
    const int i = edge % (n + 1);
    return i == 0 || i == n;
  }
  const int j = (edge - nvert) / n;
  return j == 0 || j == n;
}

static __host__ __device__ __forceinline__ int pk(int r, int c) {   // packed index, r >= c
  return r * (r + 1) / 2 + c;
}

static __device__ __forceinline__ int pk_any(int r, int c) { return r >= c ? pk(r, c) : pk(c, r); }

// ------------------------------------ deterministic block reductions
// block reduction by warp shuffles then one warp over the warp sums (a fixed
// order for a fixed block size); sh holds at least blockDim / 32 doubles
static __device__ __forceinline__ double block_sum(double v, double* sh) {
  __syncthreads();                         // sh may still be read by an earlier call
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = l < (int)(blockDim.x >> 5) ? sh[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (l == 0) sh[32] = v;
  }
  __syncthreads();
  return sh[32];
}

// returns true in the last block to finish, after all partials are visible;
// thread 0 published this block's partial before calling
static __device__ __forceinline__ bool last_block(unsigned* counter) {
  __shared__ bool is_last;
  if (threadIdx.x == 0) {
    __threadfence();                       // release the partial
    is_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    if (is_last) __threadfence();          // acquire every other block's partial
  }
  __syncthreads();
  return is_last;
}

// sum of n partials in a fixed order: thread t adds partial[t], partial[t + B],
// ... (loads issued together), then block_sum
static __device__ __forceinline__ double sum_partials(const double* partial, int n, double* sh) {
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  const int B = blockDim.x;
  int i = threadIdx.x, k = 0;
  for (; i < n && k < 4; i += B, ++k) v[k] = __ldcg(partial + i);
  double s = ((v[0] + v[1]) + v[2]) + v[3];
  for (; i < n; i += B) s += __ldcg(partial + i);
  return block_sum(s, sh);
}



// ---------------------------------------------- 2x2 agglomeration geometry
// Interior edges of macro-element C = (I, J) (fine mesh n = 2 nc):
//   ie 0: v(2I+1, 2J)  1: v(2I+1, 2J+1)  2: h(2I, 2J+1)  3: h(2I+1, 2J+1)
// Perimeter child edges (me, c): me 0 left v(2I, 2J+c), 1 right v(2I+2, 2J+c),
//   2 bottom h(2I+c, 2J), 3 top h(2I+c, 2J+2); c = 0 is the half at the
//   lower coordinate.  Local index: interior ie*2+k, boundary (me*2+c)*2+k.
static __device__ __forceinline__ int fine_v(int n, int i, int j) { return j * (n + 1) + i; }
static __device__ __forceinline__ int fine_h(int n, int i, int j) { return n * (n + 1) + j * n + i; }

static __device__ __forceinline__ int interior_edge(int n, int I, int J, int ie) {
  switch (ie) {
    case 0: return fine_v(n, 2 * I + 1, 2 * J);
    case 1: return fine_v(n, 2 * I + 1, 2 * J + 1);
    case 2: return fine_h(n, 2 * I, 2 * J + 1);
    default: return fine_h(n, 2 * I + 1, 2 * J + 1);
  }
}

static __device__ __forceinline__ int perimeter_edge(int n, int I, int J, int me, int c) {
  switch (me) {
    case 0: return fine_v(n, 2 * I, 2 * J + c);
    case 1: return fine_v(n, 2 * I + 2, 2 * J + c);
    case 2: return fine_h(n, 2 * I + c, 2 * J);
    default: return fine_h(n, 2 * I + c, 2 * J + 2);
  }
}

// child ch = cj*2 + ci, local edge le -> (interior?, slot) with slot = ie or me*2+c
static __device__ __forceinline__ void child_map(int ch, int le, bool& interior, int& slot) {
  const int ci = ch & 1, cj = ch >> 1;
  switch (le) {
    case 0: interior = (ci == 1); slot = interior ? cj : (0 * 2 + cj); break;
    case 1: interior = (ci == 0); slot = interior ? cj : (1 * 2 + cj); break;
    case 2: interior = (cj == 1); slot = interior ? 2 + ci : (2 * 2 + ci); break;
    default: interior = (cj == 0); slot = interior ? 2 + ci : (3 * 2 + ci); break;
  }
}

static __device__ __forceinline__ int coarse_v(int nc, int I, int J) { return J * (nc + 1) + I; }
static __device__ __forceinline__ int coarse_h(int nc, int I, int J) { return nc * (nc + 1) + J * nc + I; }

static inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

// row-major packed lower triangle: t = i(i+1)/2 + j, 0 <= j <= i
static __device__ __forceinline__ void tri_rc(int t, int& i, int& j) {
  int r = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  while (r * (r + 1) / 2 > t) --r;
  while ((r + 1) * (r + 2) / 2 <= t) ++r;
  i = r;
  j = t - r * (r + 1) / 2;
}

// 1/sqrt(d) for d > 0.  FP64: FP32 seed and two Newton-Raphson steps for the
// inverse square root, y <- y (3 - d y^2) / 2; FP32: the hardware estimate
// and one Newton step.
static __device__ __forceinline__ double inv_sqrt(double d) {
  double y = (double)rsqrtf((float)d);
  y = y * (1.5 - 0.5 * d * y * y);
  y = y * (1.5 - 0.5 * d * y * y);
  return y;
}
static __device__ __forceinline__ float inv_sqrt(float d) {
  float y = rsqrtf(d);
  return y * (1.5f - 0.5f * d * y * y);
}

}  // namespace hdgmg
