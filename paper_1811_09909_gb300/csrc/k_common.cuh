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

}  // namespace hdgmg
