// Edge/element kernels templated on the number of trace modes per edge ND
// and on the storage of the element operators (NS = false: symmetric, packed
// lower triangle; NS = true: non-symmetric, full row-major):
//   K6  trace matvec y += alpha A x, one thread per element, A_e in
//       structure-of-arrays layout, results added into the two edge owners
//       with atomics (exactly two contributions per entry, so the sum does
//       not depend on their order)
//   K2  edge block-Jacobi blocks D = A_e0[edge] + A_e1[edge] and D^-1
//       (Cholesky when symmetric; Gauss-Jordan without pivoting otherwise,
//       D having a positive-definite symmetric part)
//   K7  block-Jacobi update e += omega D^-1 (r - A e)  (Sec. 4.1)
// Each (type, ND) pair is compiled in its own translation unit
// (k_edge_inst.cu) so that the fully unrolled kernels build in parallel.
#pragma once

#include "k_common.cuh"

namespace hdgmg {

// element operator entries are read in their storage type TA and used in T
template <typename T>
static __device__ __forceinline__ T load_entry(const T* p) { return *p; }
static __device__ __forceinline__ float load_entry(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}

// ---------------------------------------------------------------- K6 matvec
// xadd (nullable, modes 0 and 1 only): x + J xadd is applied instead of x,
// i.e. the P1 correction of the next level is prolonged on the fly
// MULTI: blockIdx.y is the right-hand side of a blocked solve (x, y with
// stride ND n_edges, xadd with the P1 stride 2 n_edges); the one-right-hand-
// side instantiation carries no offset code
template <typename T, int ND, bool NS, typename TA = T, bool MULTI = false>
__global__ void __launch_bounds__(128) matvec_kernel(int n, const TA* __restrict__ A,
                                                     const T* __restrict__ x, T* __restrict__ y,
                                                     T alpha, const T* __restrict__ xadd) {
  constexpr int NL = 4 * ND;
  const int nE = n * n;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nE) return;
  const int nedge = 2 * n * (n + 1);
  if (MULTI) {
    x += (size_t)blockIdx.y * ND * nedge;
    y += (size_t)blockIdx.y * ND * nedge;
    if (xadd) xadd += (size_t)blockIdx.y * 2 * nedge;
  }
  int ed[4];
  elem_edges(n, e, ed);
  T xl[NL];
#pragma unroll
  for (int c = 0; c < NL; ++c) {
    const size_t ix = (size_t)(c % ND) * nedge + ed[c / ND];
    xl[c] = x[ix];
    if (xadd && c % ND < 2) xl[c] += xadd[ix];
  }
  if constexpr (NS) {
    // full storage: one row at a time (rows not unrolled, which keeps the
    // NL^2-entry kernel small to compile), added straight into y
#pragma unroll
    for (int le = 0; le < 4; ++le) {
      if (bnd_edge(n, ed[le])) continue;
#pragma unroll 1
      for (int k = 0; k < ND; ++k) {
        const TA* Ar = A + (size_t)(le * ND + k) * NL * nE + e;
        T s = T(0);
#pragma unroll
        for (int c = 0; c < NL; ++c) s += load_entry(Ar + (size_t)c * nE) * xl[c];
        atomicAdd(&y[(size_t)k * nedge + ed[le]], alpha * s);
      }
    }
  } else {
    T yl[NL];
#pragma unroll
    for (int c = 0; c < NL; ++c) yl[c] = T(0);
#pragma unroll
    for (int r = 0; r < NL; ++r) {
#pragma unroll
      for (int c = 0; c < r; ++c) {
        const T a = load_entry(A + (size_t)pk(r, c) * nE + e);
        yl[r] += a * xl[c];
        yl[c] += a * xl[r];
      }
      yl[r] += load_entry(A + (size_t)pk(r, r) * nE + e) * xl[r];
    }
#pragma unroll
    for (int le = 0; le < 4; ++le) {
      if (bnd_edge(n, ed[le])) continue;
#pragma unroll
      for (int k = 0; k < ND; ++k)
        atomicAdd(&y[(size_t)k * nedge + ed[le]], alpha * yl[le * ND + k]);
    }
  }
}

// rows LE ND ... LE ND + ND - 1 of A_e (FP64, packed symmetric) times xl,
// added into y with atomics, returning their part of xl^T A_e xl
template <int ND, int LE>
__device__ __forceinline__ double matvec_rows_q(const double* __restrict__ Ae, int nE,
                                                const double* xl, double* yE, int nedge) {
  constexpr int NL = 4 * ND;
  double q = 0.0;
#pragma unroll
  for (int k = 0; k < ND; ++k) {
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < NL; ++c) s += Ae[(size_t)pk_any(LE * ND + k, c) * nE] * xl[c];
    atomicAdd(yE + (size_t)k * nedge, s);
    q = fma(xl[LE * ND + k], s, q);
  }
  return q;
}

// K6 fused into the PCG iteration (FP64 operator in symmetric storage, one
// right-hand side): the new search direction p+ = z + beta p (beta =
// scal[4], z the preconditioned residual in TZ), Ap += A p+ (Ap zeroed by the
// previous update), and the quadratic form p+ . A p+ = sum_e p+_e^T A_e p+_e
// summed element by element (each thread over its rows and element groups,
// then block_sum, then the last block over the block partials in block
// order) into scal[1], with alpha = scal[0] / scal[1] in scal[2].  One thread
// per (element, row block): a block of four warps covers a group of 32
// consecutive elements (lane l: element 32 g + l) and warp w forms the ND
// rows of local edge w (every warp load of an entry row is one contiguous
// 32-element run; the FP64 pipe, not HBM, bounds this kernel, so four times
// the warps of one thread per element hide its latency).  A fixed grid
// strides over the groups.  Warp w first forms p+ on local edge w of the
// group's elements (one fma per value, the same as
// cg_update_dir_test_kernel's) into shared memory; every warp then reads the
// element's 4 ND values from there.  Rows of Dirichlet edges are skipped,
// where p+ is zero.
template <int ND, typename TZ>
__global__ void __launch_bounds__(128, 4) cg_matvec_kernel(int n, const double* __restrict__ A,
                                                           const TZ* __restrict__ z,
                                                           const double* __restrict__ p,
                                                           double* __restrict__ Ap,
                                                           double* __restrict__ scal,
                                                           double* __restrict__ partial,
                                                           unsigned* __restrict__ counter) {
  constexpr int NL = 4 * ND;
  __shared__ double sh[33];
  __shared__ double xs[NL][32];
  const int nE = n * n;
  const int lane = threadIdx.x & 31, le = threadIdx.x >> 5;
  const int nedge = 2 * n * (n + 1);
  const int ngroups = (nE + 31) >> 5;
  const double beta = scal[4];
  double q = 0.0;
  for (int gi = blockIdx.x; gi < ngroups; gi += gridDim.x) {
    const int e = gi * 32 + lane;
    int ed[4] = {0, 0, 0, 0};
    if (e < nE) {
      elem_edges(n, e, ed);
      const int E = le == 0 ? ed[0] : le == 1 ? ed[1] : le == 2 ? ed[2] : ed[3];
#pragma unroll
      for (int k = 0; k < ND; ++k) {
        const size_t ix = (size_t)k * nedge + E;
        xs[le * ND + k][lane] = fma(beta, p[ix], (double)z[ix]);
      }
    }
    __syncthreads();
    if (e < nE) {
      const int E = le == 0 ? ed[0] : le == 1 ? ed[1] : le == 2 ? ed[2] : ed[3];
      if (!bnd_edge(n, E)) {
        double xl[NL];
#pragma unroll
        for (int c = 0; c < NL; ++c) xl[c] = xs[c][lane];
        const double* Ae = A + e;
        double* yE = Ap + E;
        switch (le) {   // warp-uniform
          case 0: q += matvec_rows_q<ND, 0>(Ae, nE, xl, yE, nedge); break;
          case 1: q += matvec_rows_q<ND, 1>(Ae, nE, xl, yE, nedge); break;
          case 2: q += matvec_rows_q<ND, 2>(Ae, nE, xl, yE, nedge); break;
          default: q += matvec_rows_q<ND, 3>(Ae, nE, xl, yE, nedge); break;
        }
      }
    }
    __syncthreads();   // xs is rewritten by the next group
  }
  q = block_sum(q, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = q;
  if (!last_block(counter)) return;
  const double pap = sum_partials(partial, gridDim.x, sh);
  if (threadIdx.x == 0) {
    scal[1] = pap;
    scal[2] = scal[0] / pap;
    *counter = 0u;
  }
}

// ----------------------------------------------------- K2 block-Jacobi blocks
template <typename T, int ND, bool NS>
__global__ void bj_blocks_kernel(int n, const T* __restrict__ A, T* __restrict__ Dinv,
                                 int* __restrict__ err) {
  const int nedge = 2 * n * (n + 1);
  const int edge = blockIdx.x * blockDim.x + threadIdx.x;
  if (edge >= nedge) return;
  constexpr int NENT = NS ? ND * ND : ND * (ND + 1) / 2;
  constexpr int NL = 4 * ND;
  if (bnd_edge(n, edge)) {
#pragma unroll
    for (int t = 0; t < NENT; ++t) Dinv[(size_t)t * nedge + edge] = T(0);
    return;
  }
  const int nE = n * n;
  const int nvert = n * (n + 1);
  int e0, le0, e1, le1;
  if (edge < nvert) {
    const int j = edge / (n + 1), i = edge % (n + 1);
    e0 = j * n + i - 1; le0 = 1;    // left element, its right edge
    e1 = j * n + i;     le1 = 0;    // right element, its left edge
  } else {
    const int j = (edge - nvert) / n, i = (edge - nvert) % n;
    e0 = (j - 1) * n + i; le0 = 3;  // element below, its top edge
    e1 = j * n + i;       le1 = 2;  // element above, its bottom edge
  }
  T D[ND][ND];
  if constexpr (NS) {
#pragma unroll
    for (int a = 0; a < ND; ++a)
#pragma unroll
      for (int b = 0; b < ND; ++b)
        D[a][b] = A[(size_t)((le0 * ND + a) * NL + le0 * ND + b) * nE + e0] +
                  A[(size_t)((le1 * ND + a) * NL + le1 * ND + b) * nE + e1];
    // Gauss-Jordan without pivoting: Inv = D^-1
    T Inv[ND][ND];
#pragma unroll
    for (int a = 0; a < ND; ++a)
#pragma unroll
      for (int b = 0; b < ND; ++b) Inv[a][b] = (a == b) ? T(1) : T(0);
    bool bad = false;
#pragma unroll
    for (int k = 0; k < ND; ++k) {
      T d = D[k][k];
      if (!(d > T(0))) { bad = true; d = T(1); }
      const T di = T(1) / d;
#pragma unroll
      for (int j = 0; j < ND; ++j) {
        D[k][j] *= di;
        Inv[k][j] *= di;
      }
#pragma unroll
      for (int i = 0; i < ND; ++i) {
        if (i == k) continue;
        const T fct = D[i][k];
#pragma unroll
        for (int j = 0; j < ND; ++j) {
          D[i][j] -= fct * D[k][j];
          Inv[i][j] -= fct * Inv[k][j];
        }
      }
    }
#pragma unroll
    for (int a = 0; a < ND; ++a)
#pragma unroll
      for (int b = 0; b < ND; ++b) Dinv[(size_t)(a * ND + b) * nedge + edge] = Inv[a][b];
    if (bad) atomicOr(err, 2);
    return;
  } else {
#pragma unroll
  for (int a = 0; a < ND; ++a)
#pragma unroll
    for (int b = 0; b <= a; ++b) {
      const T v = A[(size_t)pk(le0 * ND + a, le0 * ND + b) * nE + e0] +
                  A[(size_t)pk(le1 * ND + a, le1 * ND + b) * nE + e1];
      D[a][b] = v;
      D[b][a] = v;
    }
  // Cholesky D = L L^T, then D^-1 = L^-T L^-1
  bool bad = false;
#pragma unroll
  for (int k = 0; k < ND; ++k) {
    T d = D[k][k];
#pragma unroll
    for (int j = 0; j < k; ++j) d -= D[k][j] * D[k][j];
    if (!(d > T(0))) { bad = true; d = T(1); }
    d = sqrt(d);
    D[k][k] = d;
#pragma unroll
    for (int i = k + 1; i < ND; ++i) {
      T s = D[i][k];
#pragma unroll
      for (int j = 0; j < k; ++j) s -= D[i][j] * D[k][j];
      D[i][k] = s / d;
    }
  }
  T Li[ND][ND];
#pragma unroll
  for (int i = 0; i < ND; ++i)
#pragma unroll
    for (int j = 0; j < ND; ++j) Li[i][j] = T(0);
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    Li[j][j] = T(1) / D[j][j];
#pragma unroll
    for (int i = j + 1; i < ND; ++i) {
      T s = T(0);
#pragma unroll
      for (int k = j; k < i; ++k) s -= D[i][k] * Li[k][j];
      Li[i][j] = s / D[i][i];
    }
  }
#pragma unroll
  for (int a = 0; a < ND; ++a)
#pragma unroll
    for (int b = 0; b <= a; ++b) {
      T s = T(0);
#pragma unroll
      for (int k = a; k < ND; ++k) s += Li[k][a] * Li[k][b];
      Dinv[(size_t)pk(a, b) * nedge + edge] = s;
    }
  if (bad) atomicOr(err, 2);
  }
}

// --------------------------------------------------- K7 block-Jacobi update
// every vector load of an edge (r, y, e, xadd) is issued before its stores,
// so that the edge's ND round trips overlap (D^-1 is read in the product:
// holding all its ND^2 entries would cost registers at large ND)
template <typename T, int ND, bool NS, bool MULTI = false>
__global__ void bj_update_kernel(int n, const T* __restrict__ Dinv, const T* __restrict__ r,
                                 T* __restrict__ y, T* __restrict__ e, T omega, int first,
                                 const T* __restrict__ xadd) {
  const int nedge = 2 * n * (n + 1);
  const int edge = blockIdx.x * blockDim.x + threadIdx.x;
  if (edge >= nedge || bnd_edge(n, edge)) return;
  if (MULTI) {                              // right-hand side blockIdx.y of a blocked solve
    const size_t o = (size_t)blockIdx.y * ND * nedge;
    r += o;
    y += o;
    e += o;
    if (xadd) xadd += (size_t)blockIdx.y * 2 * nedge;
  }
  T d[ND], eo[ND];
  if (first) {
#pragma unroll
    for (int k = 0; k < ND; ++k) {
      d[k] = r[(size_t)k * nedge + edge];
      eo[k] = T(0);
    }
  } else {
#pragma unroll
    for (int k = 0; k < ND; ++k) {
      const size_t ix = (size_t)k * nedge + edge;
      d[k] = r[ix] - y[ix];
      eo[k] = e[ix];
    }
    if (xadd) {
      eo[0] += xadd[edge];
      eo[1] += xadd[(size_t)nedge + edge];
    }
#pragma unroll
    for (int k = 0; k < ND; ++k) y[(size_t)k * nedge + edge] = T(0);
  }
#pragma unroll
  for (int a = 0; a < ND; ++a) {
    T s = T(0);
#pragma unroll
    for (int b = 0; b < ND; ++b)
      s += Dinv[(size_t)(NS ? a * ND + b : pk_any(a, b)) * nedge + edge] * d[b];
    const size_t ix = (size_t)a * nedge + edge;
    e[ix] = first ? omega * s : eo[a] + omega * s;
  }
}


// The last post-smoothing step of the finest FP32 level when it closes the
// preconditioner of the FP64 PCG (symmetric storage, one right-hand side):
// the update of bj_update_kernel (first = 0) and r.z with z the new e and r
// the FP64 residual r64, over the interior edges (r is zero on Dirichlet
// edges), summed per thread over its edges, then block_sum, then the last
// block over the block partials in block order: scal[3] = r.z, scal[4] =
// beta = scal[3] / scal[0], scal[0] = scal[3].  A fixed grid strides over the
// edges (a fixed reduction order for a given mesh).
template <int ND>
__global__ void __launch_bounds__(256) bj_update_dot_kernel(
    int n, const float* __restrict__ Dinv, const float* __restrict__ r, float* __restrict__ y,
    float* __restrict__ e, float omega, const float* __restrict__ xadd,
    const double* __restrict__ r64, double* __restrict__ scal, double* __restrict__ partial,
    unsigned* __restrict__ counter) {
  __shared__ double sh[33];
  const int nedge = 2 * n * (n + 1);
  double q = 0.0;
  for (int edge = blockIdx.x * blockDim.x + threadIdx.x; edge < nedge;
       edge += gridDim.x * blockDim.x) {
    if (bnd_edge(n, edge)) continue;
    float d[ND], eo[ND];
#pragma unroll
    for (int k = 0; k < ND; ++k) {
      const size_t ix = (size_t)k * nedge + edge;
      d[k] = r[ix] - y[ix];
      eo[k] = e[ix];
    }
    if (xadd) {
      eo[0] += xadd[edge];
      eo[1] += xadd[(size_t)nedge + edge];
    }
#pragma unroll
    for (int k = 0; k < ND; ++k) y[(size_t)k * nedge + edge] = 0.f;
#pragma unroll
    for (int a = 0; a < ND; ++a) {
      float sa = 0.f;
#pragma unroll
      for (int b = 0; b < ND; ++b) sa += Dinv[(size_t)pk_any(a, b) * nedge + edge] * d[b];
      const size_t ix = (size_t)a * nedge + edge;
      const float ea = eo[a] + omega * sa;
      e[ix] = ea;
      q += r64[ix] * (double)ea;
    }
  }
  q = block_sum(q, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = q;
  if (!last_block(counter)) return;
  const double rz = sum_partials(partial, gridDim.x, sh);
  if (threadIdx.x == 0) {
    scal[3] = rz;
    scal[4] = rz / scal[0];
    scal[0] = rz;
    *counter = 0u;
  }
}

template <int ND>
void launch_bj_update_dot_nd(cudaStream_t s, int n, const float* Dinv, const float* r, float* y,
                             float* e, float omega, const float* xadd, const double* r64,
                             double* scal, double* partial, unsigned* counter) {
  note_launch();
  const int g = nblk(2 * n * (n + 1), 256), blocks = g < kDotBlocks ? g : kDotBlocks;
  bj_update_dot_kernel<ND><<<blocks, 256, 0, s>>>(n, Dinv, r, y, e, omega, xadd, r64, scal, partial,
                                                  counter);
}

// k > 1 right-hand sides of a blocked solve: one launch over gridDim.y = k
// (the right-hand sides' blocks read the operator from L2 together)
template <typename T, int ND, bool NS>
void launch_matvec_nd(cudaStream_t s, int n, const T* A, const T* x, T* y, T alpha,
                      const T* xadd, int k) {
  note_launch();
  if (k > 1)
    matvec_kernel<T, ND, NS, T, true><<<dim3(nblk(n * n, 128), k), 128, 0, s>>>(n, A, x, y, alpha,
                                                                                 xadd);
  else
    matvec_kernel<T, ND, NS><<<nblk(n * n, 128), 128, 0, s>>>(n, A, x, y, alpha, xadd);
}

template <int ND, bool NS>
void launch_matvec_bf16_nd(cudaStream_t s, int n, const __nv_bfloat16* A, const float* x, float* y,
                           float alpha, const float* xadd, int k) {
  note_launch();
  if (k > 1)
    matvec_kernel<float, ND, NS, __nv_bfloat16, true><<<dim3(nblk(n * n, 128), k), 128, 0, s>>>(
        n, A, x, y, alpha, xadd);
  else
    matvec_kernel<float, ND, NS, __nv_bfloat16><<<nblk(n * n, 128), 128, 0, s>>>(n, A, x, y, alpha,
                                                                                xadd);
}

// grid: at most kDotBlocks blocks striding over the groups of 32 elements
// (fixed for a given mesh, so the reduction order is too)
template <int ND>
void launch_cg_matvec_nd(cudaStream_t s, int n, const double* A, const float* z32,
                         const double* z64, const double* p, double* Ap, double* scal,
                         double* partial, unsigned* counter) {
  note_launch();
  const int g = nblk(n * n, 32), blocks = g < kDotBlocks ? g : kDotBlocks;
  if (z32)
    cg_matvec_kernel<ND, float><<<blocks, 128, 0, s>>>(n, A, z32, p, Ap, scal, partial, counter);
  else
    cg_matvec_kernel<ND, double><<<blocks, 128, 0, s>>>(n, A, z64, p, Ap, scal, partial, counter);
}

template <typename T, int ND, bool NS>
void launch_bj_blocks_nd(cudaStream_t s, int n, const T* A, T* Dinv, int* err) {
  note_launch();
  bj_blocks_kernel<T, ND, NS><<<nblk(2 * n * (n + 1), 128), 128, 0, s>>>(n, A, Dinv, err);
}

template <typename T, int ND, bool NS>
void launch_bj_update_nd(cudaStream_t s, int n, const T* Dinv, const T* r, T* y, T* e, T omega,
                         int first, const T* xadd, int k) {
  note_launch();
  if (k > 1)
    bj_update_kernel<T, ND, NS, true><<<dim3(nblk(2 * n * (n + 1), 128), k), 128, 0, s>>>(
        n, Dinv, r, y, e, omega, first, xadd);
  else
    bj_update_kernel<T, ND, NS><<<nblk(2 * n * (n + 1), 128), 128, 0, s>>>(n, Dinv, r, y, e, omega,
                                                                           first, xadd);
}

}  // namespace hdgmg
