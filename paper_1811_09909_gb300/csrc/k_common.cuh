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
