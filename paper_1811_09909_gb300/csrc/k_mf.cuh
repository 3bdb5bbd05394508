// Matrix-free FP32 application of the finest trace operator (symmetric
// volume blocks, the shared-eigenbasis route of the condensation).  With
// s_i = kappa_e g_i + tau e_i and the basis tables P, Q ([nv][nt]) the
// condensed element operator is
//   A_e = kappa_e K + tau I - sum_i (kappa_e P_i + tau Q_i)^T (kappa_e P_i + tau Q_i) / s_i
// (Sec. 2, static condensation of the local problems eqs. HDG_local1/2,
// diagonalised by the basis), so A_e x costs nt^2 + 4 nv nt FMA per element
// instead of reading nt (nt + 1) / 2 stored entries.  The tables depend on
// the mesh (h, tau) and p only; they travel in the kernel's parameter block
// (__grid_constant__), so every FMA reads its table entry from the constant
// bank and concurrent contexts cannot interfere.  FP32 throughout: the
// subtraction cancels for smooth x (relative error up to ~1e-4 of the
// terms), which is why it is an option of the V-cycle only.
#pragma once

#include "k_common.cuh"

namespace hdgmg {

template <int ND>
struct MfTables {
  static constexpr int NT = 4 * ND, NV = ND * ND;
  float K[NT * NT];   // [r][c]
  float P[NV * NT];   // [i][c]
  float Q[NV * NT];   // tau Q
  float g[NV];
  float e[NV];        // tau e
  float tau;
};

// One thread per element, the whole element in one instruction stream (every
// warp runs the same code and reads the same table entries, so the
// instruction and constant caches serve all of them; splitting an element
// over four warps with per-warp code paths thrashed the instruction cache).
// y += alpha A_e x added into the two edge owners with atomics (two
// contributions per entry); xadd as in matvec_kernel; MULTI: blockIdx.y is
// the right-hand side of a blocked solve.
template <int ND, bool MULTI>
__global__ void __launch_bounds__(128) matvec_mf_kernel(int n, const __grid_constant__ MfTables<ND> T,
                                                        const double* __restrict__ kap,
                                                        const float* __restrict__ x,
                                                        float* __restrict__ y, float alpha,
                                                        const float* __restrict__ xadd) {
  constexpr int NT = 4 * ND, NV = ND * ND;
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
  float xl[NT];
#pragma unroll
  for (int c = 0; c < NT; ++c) {
    const size_t ix = (size_t)(c % ND) * nedge + ed[c / ND];
    xl[c] = x[ix];
    if (xadd && c % ND < 2) xl[c] += xadd[ix];
  }
  const float kp = (float)kap[e];
  float acc[NT];
#pragma unroll
  for (int r = 0; r < NT; ++r) {   // kappa K x + tau x
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < NT; ++c) s = fmaf(T.K[r * NT + c], xl[c], s);
    acc[r] = fmaf(kp, s, T.tau * xl[r]);
  }
#pragma unroll
  for (int i = 0; i < NV; ++i) {   // - (kappa P_i + Q_i)^T w_i, w_i = (kappa P_i + Q_i) x / s_i
    float a = 0.f, b = 0.f;
#pragma unroll
    for (int c = 0; c < NT; ++c) {
      a = fmaf(T.P[i * NT + c], xl[c], a);
      b = fmaf(T.Q[i * NT + c], xl[c], b);
    }
    const float w = fmaf(kp, a, b) / fmaf(kp, T.g[i], T.e[i]);
    const float kw = kp * w;
#pragma unroll
    for (int r = 0; r < NT; ++r) acc[r] = fmaf(-T.P[i * NT + r], kw, fmaf(-T.Q[i * NT + r], w, acc[r]));
  }
#pragma unroll
  for (int le = 0; le < 4; ++le) {
    if (bnd_edge(n, ed[le])) continue;
#pragma unroll
    for (int k = 0; k < ND; ++k) atomicAdd(&y[(size_t)k * nedge + ed[le]], alpha * acc[le * ND + k]);
  }
}

// tables: host array laid out as MfTables<ND> (K, P, tau Q, g, tau e, tau)
template <int ND>
void launch_matvec_mf_nd(cudaStream_t s, int n, const float* tables, const double* kap,
                         const float* x, float* y, float alpha, const float* xadd, int k) {
  MfTables<ND> T;
  static_assert(sizeof(MfTables<ND>) == sizeof(float) * mf_table_size(ND), "table layout");
  memcpy(&T, tables, sizeof(T));
  note_launch();
  if (k > 1)
    matvec_mf_kernel<ND, true><<<dim3(nblk(n * n, 128), k), 128, 0, s>>>(n, T, kap, x, y, alpha, xadd);
  else
    matvec_mf_kernel<ND, false><<<nblk(n * n, 128), 128, 0, s>>>(n, T, kap, x, y, alpha, xadd);
}

}  // namespace hdgmg
