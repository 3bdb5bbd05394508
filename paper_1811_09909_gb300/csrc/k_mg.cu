// Multigrid kernels for the HDG trace system (arXiv:1811.09909, Sec. 3):
//   K6  trace matvec y += alpha A x, element by element (packed symmetric A_e)
//   K2  edge block-Jacobi blocks and their inverses (Sec. 4.1, block-Jacobi)
//   K7  block-Jacobi update e += omega D^-1 (r - A e)
//   K3  p-coarsening A_{N-1} = J_N^T A_N J_N (eq. ANm1)
//   K4  2x2 agglomeration: local Schur complement, prolongation/restriction
//       blocks and local-correction blocks (eqs. n_1_Ik, n_1_Qk, Akm1,
//       localCorrection)
//   K8  local correction, K9 restriction, K11 prolongation
//   K10 coarsest level: dense Cholesky (assembly, factorisation, solve)
//
// Every kernel takes the operator storage: packed symmetric, or (ns, the
// convection-diffusion operator) full row-major; the non-symmetric transfer
// uses the restriction block Rt built from A_BI where the symmetric one
// reuses Pi (Q_{k-1} = I_k^T).
//
// Vectors are [nd][n_edges] with Dirichlet (boundary) entries held at zero;
// every level owns an accumulator y that is zero between kernels: the matvec
// adds into it and the consumer of y resets it.
#include <cmath>
#include <mutex>

#include "internal.h"
#include "k_common.cuh"

namespace hdgmg {

namespace {

// ------------------------------------------------------- K3 p-coarsening
template <typename T>
__global__ void pcoarsen_kernel(int nE, int ndf, bool ns, const T* __restrict__ Af,
                                T* __restrict__ Ac) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nE) return;
  const int nlf = 4 * ndf;
  for (int r = 0; r < 8; ++r)
    for (int c = 0; c < (ns ? 8 : r + 1); ++c) {
      const int rf = (r / 2) * ndf + (r % 2), cf = (c / 2) * ndf + (c % 2);
      if (ns)
        Ac[(size_t)(r * 8 + c) * nE + e] = Af[(size_t)(rf * nlf + cf) * nE + e];
      else
        Ac[(size_t)pk(r, c) * nE + e] = Af[(size_t)pk(rf, cf) * nE + e];
    }
}

__constant__ double c_Jc[2][2][2];   // child injection [child][fine mode][coarse mode]
// the same in FP32: the FP32 cycle reads these (a per-use FP64 -> FP32
// conversion runs on GB300's narrow FP64 pipe)
__constant__ float c_Jcf[2][2][2];

}  // namespace
}  // namespace hdgmg
#include "k_p1.cuh"
namespace hdgmg {
namespace {

// -------------------------------------------------- K4 agglomeration setup
// One warp per macro-element C: the 24 x 24 local block assembled from the
// four children lives in shared memory and every product is spread over the
// 32 lanes:
//   A_II = L L^T, A_II^-1 = L^-T L^-1, Y = -A_II^-1 A_IB,
//   S = A_BB + A_IB^T Y, A_c = J^T S J, Pi = Y J.
template <typename T, int WPB>
__global__ void __launch_bounds__(32 * WPB) agglomerate_warp_kernel(
    int nc, const T* __restrict__ Af, T* __restrict__ Ac, T* __restrict__ AIIinv,
    T* __restrict__ Yout, T* __restrict__ Pi, int* __restrict__ err) {
  constexpr int PER = 64 + 128 + 256 + 64 + 64 + 128 + 128;
  __shared__ T sh[WPB * PER];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nC = nc * nc;
  const int C = blockIdx.x * WPB + warp;
  if (C >= nC) return;
  const int J = C / nc, I = C - J * nc;
  const int n = 2 * nc, nEf = n * n;
  T* AII = sh + warp * PER;      // 8 x 8
  T* AIB = AII + 64;             // 8 x 16
  T* ABB = AIB + 128;            // 16 x 16, becomes S
  T* Lm = ABB + 256;             // 8 x 8 Cholesky factor
  T* Ai = Lm + 64;               // 8 x 8 A_II^-1
  T* Yw = Ai + 64;               // 8 x 16
  T* SJ = Yw + 128;              // 16 x 8, also holds L^-1 before Y is formed
  for (int t = lane; t < 448; t += 32) AII[t] = T(0);
  __syncwarp();
  for (int ch = 0; ch < 4; ++ch) {
    const int ef = (2 * J + (ch >> 1)) * n + 2 * I + (ch & 1);
    for (int t = lane; t < 64; t += 32) {
      const int r = t >> 3, c = t & 7;
      bool ir, ic;
      int sr, sc;
      child_map(ch, r >> 1, ir, sr);
      child_map(ch, c >> 1, ic, sc);
      const int lr = sr * 2 + (r & 1), lc = sc * 2 + (c & 1);
      const T a = Af[(size_t)pk_any(r, c) * nEf + ef];
      if (ir && ic) AII[lr * 8 + lc] += a;
      else if (ir && !ic) AIB[lr * 16 + lc] += a;
      else if (!ir && !ic) ABB[lr * 16 + lc] += a;
    }
    __syncwarp();
  }
  // Cholesky of A_II
  for (int t = lane; t < 64; t += 32) Lm[t] = AII[t];
  __syncwarp();
  bool bad = false;
  for (int k = 0; k < 8; ++k) {
    T di = T(0);
    if (lane == 0) {
      T d = Lm[k * 8 + k];
      if (!(d > T(0))) {
        bad = true;
        d = T(1);
      }
      di = inv_sqrt(d);
      Lm[k * 8 + k] = d * di;
    }
    di = __shfl_sync(0xffffffffu, di, 0);
    if (lane > k && lane < 8) Lm[lane * 8 + k] *= di;
    __syncwarp();
    const int m = 7 - k;
    if (lane < m * (m + 1) / 2) {
      int ii, jj;
      tri_rc(lane, ii, jj);
      const int i = k + 1 + ii, j = k + 1 + jj;
      Lm[i * 8 + j] -= Lm[i * 8 + k] * Lm[j * 8 + k];
    }
    __syncwarp();
  }
  if (bad) atomicOr(err, 4);
  // L^-1 (columns by lanes 0..7) into SJ[0..63]
  if (lane < 8) {
    const int j = lane;
    for (int i = 0; i < 8; ++i) {
      T s = (i == j) ? T(1) : T(0);
      if (i >= j) {
        for (int k = j; k < i; ++k) s -= Lm[i * 8 + k] * SJ[k * 8 + j];
        s = s / Lm[i * 8 + i];
      }
      SJ[i * 8 + j] = s;
    }
  }
  __syncwarp();
  // A_II^-1 = L^-T L^-1
  for (int t = lane; t < 64; t += 32) {
    const int a = t >> 3, b = t & 7;
    T s = T(0);
    for (int k = (a > b ? a : b); k < 8; ++k) s += SJ[k * 8 + a] * SJ[k * 8 + b];
    Ai[t] = s;
  }
  __syncwarp();
  // Y = -A_II^-1 A_IB
  for (int t = lane; t < 128; t += 32) {
    const int a = t >> 4, b = t & 15;
    T s = T(0);
#pragma unroll
    for (int k = 0; k < 8; ++k) s -= Ai[a * 8 + k] * AIB[k * 16 + b];
    Yw[t] = s;
  }
  __syncwarp();
  // S = A_BB + A_IB^T Y (in place)
  for (int t = lane; t < 256; t += 32) {
    const int a = t >> 4, b = t & 15;
    T s = ABB[t];
#pragma unroll
    for (int k = 0; k < 8; ++k) s += AIB[k * 16 + a] * Yw[k * 16 + b];
    ABB[t] = s;
  }
  __syncwarp();
  // SJ = S J (16 x 8)
  for (int t = lane; t < 128; t += 32) {
    const int a = t >> 3, cb = t & 7, me = cb >> 1, kc = cb & 1;
    T s = T(0);
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int kf = 0; kf < 2; ++kf) s += ABB[a * 16 + (me * 2 + c) * 2 + kf] * (T)c_Jc[c][kf][kc];
    SJ[t] = s;
  }
  __syncwarp();
  // outputs
  for (int t = lane; t < 36; t += 32) {
    int ca, cb;
    tri_rc(t, ca, cb);
    const int me = ca >> 1, kc = ca & 1;
    T s = T(0);
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int kf = 0; kf < 2; ++kf) s += (T)c_Jc[c][kf][kc] * SJ[((me * 2 + c) * 2 + kf) * 8 + cb];
    Ac[(size_t)t * nC + C] = s;
    AIIinv[(size_t)t * nC + C] = Ai[ca * 8 + cb];
  }
  for (int t = lane; t < 64; t += 32) {
    const int a = t >> 3, cb = t & 7, me = cb >> 1, kc = cb & 1;
    T s = T(0);
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int kf = 0; kf < 2; ++kf) s += Yw[a * 16 + (me * 2 + c) * 2 + kf] * (T)c_Jc[c][kf][kc];
    Pi[(size_t)t * nC + C] = s;
  }
  for (int t = lane; t < 128; t += 32) Yout[(size_t)t * nC + C] = Yw[t];
}

// Non-symmetric variant (one warp per macro-element): A_BI is assembled on
// its own, A_II = LU without pivoting (positive-definite symmetric part),
//   A_II^-1, Y = -A_II^-1 A_IB, S = A_BB + A_BI Y, A_c = J^T S J (full),
//   Pi = Y J, Z = -A_BI A_II^-1 and Rt = Z^T J (Q_{k-1} = [J^T Z, J^T]).
template <typename T, int WPB>
__global__ void __launch_bounds__(32 * WPB) agglomerate_ns_warp_kernel(
    int nc, const T* __restrict__ Af, T* __restrict__ Ac, T* __restrict__ AIIinv,
    T* __restrict__ Yout, T* __restrict__ Pi, T* __restrict__ Rt, int* __restrict__ err) {
  constexpr int PER = 64 + 128 + 128 + 256 + 64 + 64 + 128 + 128 + 128;
  __shared__ T sh[WPB * PER];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nC = nc * nc;
  const int C = blockIdx.x * WPB + warp;
  if (C >= nC) return;
  const int J = C / nc, I = C - J * nc;
  const int n = 2 * nc, nEf = n * n;
  T* AII = sh + warp * PER;      // 8 x 8
  T* AIB = AII + 64;             // 8 x 16
  T* ABI = AIB + 128;            // 16 x 8
  T* ABB = ABI + 128;            // 16 x 16, becomes S
  T* LUm = ABB + 256;            // 8 x 8 LU factors of A_II
  T* Ai = LUm + 64;              // 8 x 8 A_II^-1
  T* Yw = Ai + 64;               // 8 x 16
  T* SJ = Yw + 128;              // 16 x 8
  T* Zw = SJ + 128;              // 16 x 8
  for (int t = lane; t < PER; t += 32) AII[t] = T(0);
  __syncwarp();
  for (int ch = 0; ch < 4; ++ch) {
    const int ef = (2 * J + (ch >> 1)) * n + 2 * I + (ch & 1);
    for (int t = lane; t < 64; t += 32) {
      const int r = t >> 3, c = t & 7;
      bool ir, ic;
      int sr, sc;
      child_map(ch, r >> 1, ir, sr);
      child_map(ch, c >> 1, ic, sc);
      const int lr = sr * 2 + (r & 1), lc = sc * 2 + (c & 1);
      const T a = Af[(size_t)(r * 8 + c) * nEf + ef];
      if (ir && ic) AII[lr * 8 + lc] += a;
      else if (ir && !ic) AIB[lr * 16 + lc] += a;
      else if (!ir && ic) ABI[lr * 8 + lc] += a;
      else ABB[lr * 16 + lc] += a;
    }
    __syncwarp();
  }
  // LU of A_II (unit lower part below the diagonal)
  for (int t = lane; t < 64; t += 32) LUm[t] = AII[t];
  __syncwarp();
  bool bad = false;
  for (int k = 0; k < 8; ++k) {
    T di = T(0);
    if (lane == 0) {
      T d = LUm[k * 8 + k];
      if (!(d > T(0))) {
        bad = true;
        d = T(1);
      }
      di = T(1) / d;
    }
    di = __shfl_sync(0xffffffffu, di, 0);
    if (lane > k && lane < 8) LUm[lane * 8 + k] *= di;
    __syncwarp();
    const int m = 7 - k;
    for (int t = lane; t < m * m; t += 32) {
      const int i = k + 1 + t / m, j = k + 1 + t % m;
      LUm[i * 8 + j] -= LUm[i * 8 + k] * LUm[k * 8 + j];
    }
    __syncwarp();
  }
  if (bad) atomicOr(err, 4);
  // A_II^-1 column by column (lanes 0..7)
  if (lane < 8) {
    const int j = lane;
    T col[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      T s = (i == j) ? T(1) : T(0);
#pragma unroll
      for (int k = 0; k < i; ++k) s -= LUm[i * 8 + k] * col[k];
      col[i] = s;
    }
#pragma unroll
    for (int i = 7; i >= 0; --i) {
      T s = col[i];
#pragma unroll
      for (int k = i + 1; k < 8; ++k) s -= LUm[i * 8 + k] * col[k];
      col[i] = s / LUm[i * 8 + i];
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) Ai[i * 8 + j] = col[i];
  }
  __syncwarp();
  // Y = -A_II^-1 A_IB, Z = -A_BI A_II^-1
  for (int t = lane; t < 128; t += 32) {
    const int a = t >> 4, b = t & 15;
    T s = T(0);
#pragma unroll
    for (int k = 0; k < 8; ++k) s -= Ai[a * 8 + k] * AIB[k * 16 + b];
    Yw[t] = s;
    const int bz = t >> 3, az = t & 7;
    T z = T(0);
#pragma unroll
    for (int k = 0; k < 8; ++k) z -= ABI[bz * 8 + k] * Ai[k * 8 + az];
    Zw[t] = z;
  }
  __syncwarp();
  // S = A_BB + A_BI Y (in place)
  for (int t = lane; t < 256; t += 32) {
    const int a = t >> 4, b = t & 15;
    T s = ABB[t];
#pragma unroll
    for (int k = 0; k < 8; ++k) s += ABI[a * 8 + k] * Yw[k * 16 + b];
    ABB[t] = s;
  }
  __syncwarp();
  // SJ = S J (16 x 8)
  for (int t = lane; t < 128; t += 32) {
    const int a = t >> 3, cb = t & 7, me = cb >> 1, kc = cb & 1;
    T s = T(0);
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int kf = 0; kf < 2; ++kf) s += ABB[a * 16 + (me * 2 + c) * 2 + kf] * (T)c_Jc[c][kf][kc];
    SJ[t] = s;
  }
  __syncwarp();
  // outputs: A_c = J^T S J, A_II^-1, Pi = Y J, Rt = Z^T J, Y
  for (int t = lane; t < 64; t += 32) {
    const int ca = t >> 3, cb = t & 7;
    const int me = ca >> 1, kc = ca & 1;
    T s = T(0);
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int kf = 0; kf < 2; ++kf) s += (T)c_Jc[c][kf][kc] * SJ[((me * 2 + c) * 2 + kf) * 8 + cb];
    Ac[(size_t)t * nC + C] = s;
    AIIinv[(size_t)t * nC + C] = Ai[t];
    const int a = t >> 3, mb = cb >> 1, kb = cb & 1;
    T pi = T(0), rt = T(0);
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int kf = 0; kf < 2; ++kf) {
        const int b = (mb * 2 + c) * 2 + kf;
        pi += Yw[a * 16 + b] * (T)c_Jc[c][kf][kb];
        rt += Zw[b * 8 + a] * (T)c_Jc[c][kf][kb];
      }
    Pi[(size_t)t * nC + C] = pi;
    Rt[(size_t)t * nC + C] = rt;
  }
  for (int t = lane; t < 128; t += 32) Yout[(size_t)t * nC + C] = Yw[t];
}

// ------------------------------------------------- K8 local correction
// e_I <- e_I + A_II^-1 (r - A e)_I = A_II^-1 r_I + Y e_B, one work item per
// (macro-element C, interior dof a): t = a * nC + C, so that a warp reads one
// row entry of 32 consecutive macro-elements' blocks.  The items of one C
// write distinct interior entries and read only perimeter entries of e.
template <typename T>
__device__ __forceinline__ void local_correction_item(int nc, bool ns, const T* __restrict__ AIIinv,
                                                      const T* __restrict__ Y, const T* r, T* e,
                                                      int t) {
  const int nC = nc * nc;
  const int a = t / nC, C = t - a * nC;
  const int J = C / nc, I = C - J * nc;
  const int n = 2 * nc;
  const int nedge = 2 * n * (n + 1);
  T s = T(0);
#pragma unroll
  for (int ie = 0; ie < 4; ++ie) {
    const int ed = interior_edge(n, I, J, ie);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int kk = ie * 2 + k;
      s += AIIinv[(size_t)(ns ? a * 8 + kk : pk_any(a, kk)) * nC + C] * r[(size_t)k * nedge + ed];
    }
  }
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const int ed = perimeter_edge(n, I, J, b >> 1, b & 1);
#pragma unroll
    for (int k = 0; k < 2; ++k) s += Y[(size_t)(a * 16 + b * 2 + k) * nC + C] * e[(size_t)k * nedge + ed];
  }
  e[(size_t)(a & 1) * nedge + interior_edge(n, I, J, a >> 1)] = s;
}

template <typename T, bool NS>
__global__ void local_correction_kernel(const P1Geom g, const T* __restrict__ AIIinv,
                                        const T* __restrict__ Y, const T* __restrict__ r,
                                        T* __restrict__ e) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t o = (size_t)blockIdx.y * 2 * g.nedge;        // right-hand side of a blocked solve
  if (t < 8 * g.nC) p1_lc<T, NS>(g, AIIinv, Y, r + o, e + o, t);
}


// --------------------------------------------------------- K9 restriction
// r_c = J^T s_B + Rt^T s_I (Q_{k-1} of eq. n_1_Qk: Rt^T = -J^T A_BI A_II^-1,
// which is Pi^T for symmetric A), s = r - y, y = A e.  One work item per
// (coarse edge E, coarse mode kc): t = kc * nedc + E.  The block argument
// (named Pi) is Rt.
template <typename T>
__device__ __forceinline__ void restrict_h_item(int nc, const T* __restrict__ Pi, const T* r,
                                                const T* y, T* rc, int t) {
  const int nedc = 2 * nc * (nc + 1);
  const int kc = t >= nedc ? 1 : 0, E = t - kc * nedc;
  if (bnd_edge(nc, E)) {
    rc[t] = T(0);
    return;
  }
  const int n = 2 * nc, nedge = 2 * n * (n + 1), nC = nc * nc;
  const int nvc = nc * (nc + 1);
  int ch[2], Cs[2], mes[2];
  if (E < nvc) {
    const int J = E / (nc + 1), I = E % (nc + 1);
    ch[0] = fine_v(n, 2 * I, 2 * J);
    ch[1] = fine_v(n, 2 * I, 2 * J + 1);
    Cs[0] = J * nc + I - 1; mes[0] = 1;    // left macro-element, its right edge
    Cs[1] = J * nc + I;     mes[1] = 0;
  } else {
    const int J = (E - nvc) / nc, I = (E - nvc) % nc;
    ch[0] = fine_h(n, 2 * I, 2 * J);
    ch[1] = fine_h(n, 2 * I + 1, 2 * J);
    Cs[0] = (J - 1) * nc + I; mes[0] = 3;  // macro-element below, its top edge
    Cs[1] = J * nc + I;       mes[1] = 2;
  }
  T acc = T(0);
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const T s0 = r[ch[c]] - y[ch[c]];
    const T s1 = r[(size_t)nedge + ch[c]] - y[(size_t)nedge + ch[c]];
    acc += (T)c_Jc[c][0][kc] * s0 + (T)c_Jc[c][1][kc] * s1;
  }
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const int C = Cs[side];
    const int J = C / nc, I = C - J * nc;
#pragma unroll
    for (int ie = 0; ie < 4; ++ie) {
      const int ed = interior_edge(n, I, J, ie);
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const T s = r[(size_t)k * nedge + ed] - y[(size_t)k * nedge + ed];
        acc += Pi[(size_t)((ie * 2 + k) * 8 + mes[side] * 2 + kc) * nC + C] * s;
      }
    }
  }
  rc[t] = acc;
}

template <typename T>
__global__ void restrict_h_kernel(const P1Geom g, const T* __restrict__ Pi, const T* __restrict__ r,
                                  const T* __restrict__ y, T* __restrict__ rc) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t o = (size_t)blockIdx.y * 2 * g.nedge, oc = (size_t)blockIdx.y * 2 * g.nedc;
  if (t < 2 * g.nedc) p1_restrict<T>(g, Pi, r + o, y + o, rc + oc, t);
}

// -------------------------------------------------------- K11 prolongation
// e_I += Pi e_c(C): one item per (macro-element C, interior dof a),
// t = a * nC + C; e_B += J e_c: one item per (coarse edge E, half c),
// t = 8 nC + c * nedc + E.  Every fine edge is touched exactly once, where y
// is reset.
template <typename T>
__device__ __forceinline__ void prolong_h_item(int nc, const T* __restrict__ Pi, const T* ec,
                                               T* e, T* y, int t) {
  const int nC = nc * nc, nedc = 2 * nc * (nc + 1), nvc = nc * (nc + 1);
  const int n = 2 * nc, nedge = 2 * n * (n + 1);
  if (t < 8 * nC) {
    const int a = t / nC, C = t - a * nC;
    const int J = C / nc, I = C - J * nc;
    const int ce[4] = {coarse_v(nc, I, J), coarse_v(nc, I + 1, J), coarse_h(nc, I, J),
                       coarse_h(nc, I, J + 1)};
    T s = T(0);
#pragma unroll
    for (int me = 0; me < 4; ++me) {
      s += Pi[(size_t)(a * 8 + me * 2) * nC + C] * ec[ce[me]];
      s += Pi[(size_t)(a * 8 + me * 2 + 1) * nC + C] * ec[(size_t)nedc + ce[me]];
    }
    const size_t ix = (size_t)(a & 1) * nedge + interior_edge(n, I, J, a >> 1);
    e[ix] += s;
    y[ix] = T(0);
    return;
  }
  const int u = t - 8 * nC;
  if (u >= 2 * nedc) return;
  const int c = u >= nedc ? 1 : 0, E = u - c * nedc;
  int ch;
  if (E < nvc) {
    const int J = E / (nc + 1), I = E % (nc + 1);
    ch = fine_v(n, 2 * I, 2 * J + c);
  } else {
    const int J = (E - nvc) / nc, I = (E - nvc) % nc;
    ch = fine_h(n, 2 * I + c, 2 * J);
  }
  const T x0 = ec[E], x1 = ec[(size_t)nedc + E];
#pragma unroll
  for (int kf = 0; kf < 2; ++kf) {
    const size_t ix = (size_t)kf * nedge + ch;
    e[ix] += (T)c_Jc[c][kf][0] * x0 + (T)c_Jc[c][kf][1] * x1;
    y[ix] = T(0);
  }
}

template <typename T>
__global__ void prolong_h_kernel(const P1Geom g, const T* __restrict__ Pi, const T* __restrict__ ec,
                                 T* __restrict__ e, T* __restrict__ y) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t o = (size_t)blockIdx.y * 2 * g.nedge, oc = (size_t)blockIdx.y * 2 * g.nedc;
  if (t < 8 * g.nC + 2 * g.nedc) p1_prolong<T>(g, Pi, ec + oc, e + o, y + o, t);
}

// ------------------------------------------------- p-transfer (J_N, J_N^T)
// J_N^T fused into the first block-Jacobi sweep of the P1 level below (same
// mesh, one thread per edge): r1 = r0 - y0 on modes 0 and 1, y0 reset on
// every mode, e1 = omega D1^-1 r1.
template <typename T, bool NS>
__global__ void bj_first_restrict_p_kernel(const P1Geom g, int nd0, const T* __restrict__ Dinv1,
                                           const T* __restrict__ r0, T* __restrict__ y0,
                                           T* __restrict__ r1, T* __restrict__ e1, T omega) {
  const int E = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t o0 = (size_t)blockIdx.y * nd0 * g.nedge, o1 = (size_t)blockIdx.y * 2 * g.nedge;
  if (E < g.nedge)
    p1_first_restrict_p<T, NS>(g, nd0, Dinv1, r0 + o0, y0 + o0, r1 + o1, e1 + o1, omega, E);
}

template <typename T>
__global__ void restrict_p_kernel(int n, int nd, const T* __restrict__ r, T* __restrict__ y,
                                  T* __restrict__ rc) {
  const int nedge = 2 * n * (n + 1);
  const int edge = blockIdx.x * blockDim.x + threadIdx.x;
  if (edge >= nedge) return;
  rc[edge] = r[edge] - y[edge];
  rc[(size_t)nedge + edge] = r[(size_t)nedge + edge] - y[(size_t)nedge + edge];
  for (int k = 0; k < nd; ++k) y[(size_t)k * nedge + edge] = T(0);
}

template <typename T>
__global__ void prolong_p_kernel(int n, const T* __restrict__ ec, T* __restrict__ e) {
  const int nedge = 2 * n * (n + 1);
  const int edge = blockIdx.x * blockDim.x + threadIdx.x;
  if (edge >= nedge) return;
  e[edge] += ec[edge];
  e[(size_t)nedge + edge] += ec[(size_t)nedge + edge];
}

// ------------------------------------------------------ K10 coarsest level
template <typename T>
__global__ void coarse_assemble_kernel(int n, bool ns, const T* __restrict__ A,
                                       const int* __restrict__ fidx, int nf,
                                       double* __restrict__ dense) {
  const int nE = n * n;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nE) return;
  int ed[4];
  elem_edges(n, e, ed);
  for (int r = 0; r < 8; ++r) {
    const int fr = fidx[ed[r / 2]];
    if (fr < 0) continue;
    for (int c = 0; c < 8; ++c) {
      const int fc = fidx[ed[c / 2]];
      if (fc < 0) continue;
      atomicAdd(&dense[(size_t)(fr * 2 + (r & 1)) * nf + fc * 2 + (c & 1)],
                (double)A[(size_t)(ns ? r * 8 + c : pk_any(r, c)) * nE + e]);
    }
  }
}

// Gauss-Jordan inverse without pivoting of a dense matrix with positive-
// definite symmetric part, in place in global memory (one block); the
// inverse ends up in M and is copied to Ainv.
__global__ void coarse_gj_kernel(int nf, double* __restrict__ M, double* __restrict__ Ainv,
                                 int* __restrict__ err) {
  extern __shared__ double colk[];
  __shared__ double piv;
  for (int k = 0; k < nf; ++k) {
    if (threadIdx.x == 0) {
      double d = M[(size_t)k * nf + k];
      if (!(d > 0.0)) {
        atomicOr(err, 8);
        d = 1.0;
      }
      piv = 1.0 / d;
      M[(size_t)k * nf + k] = 1.0;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nf; j += blockDim.x) M[(size_t)k * nf + j] *= piv;
    for (int i = threadIdx.x; i < nf; i += blockDim.x) colk[i] = (i == k) ? 0.0 : M[(size_t)i * nf + k];
    __syncthreads();
    for (int64_t t = threadIdx.x; t < (int64_t)nf * nf; t += blockDim.x) {
      const int i = (int)(t / nf), j = (int)(t - (int64_t)i * nf);
      if (i == k) continue;
      if (j == k)
        M[t] = -colk[i] * M[(size_t)k * nf + k];
      else
        M[t] -= colk[i] * M[(size_t)k * nf + j];
    }
    __syncthreads();
  }
  for (int64_t t = threadIdx.x; t < (int64_t)nf * nf; t += blockDim.x) Ainv[t] = M[t];
}

__global__ void coarse_factor_kernel(int nf, double* __restrict__ M, int* __restrict__ err) {
  __shared__ double dinv;
  for (int k = 0; k < nf; ++k) {
    if (threadIdx.x == 0) {
      double d = M[(size_t)k * nf + k];
      if (!(d > 0.0)) {
        atomicOr(err, 8);
        d = 1.0;
      }
      d = sqrt(d);
      M[(size_t)k * nf + k] = d;
      dinv = 1.0 / d;
    }
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < nf; i += blockDim.x) M[(size_t)i * nf + k] *= dinv;
    __syncthreads();
    const int m = nf - k - 1;
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      const int i = k + 1 + t / m, j = k + 1 + t % m;
      if (j <= i) M[(size_t)i * nf + j] -= M[(size_t)i * nf + k] * M[(size_t)j * nf + k];
    }
    __syncthreads();
  }
}

// Coarsest level, small case (the whole matrix fits in shared memory): one
// block assembles A_1 from the element matrices and inverts it in place by
// Gauss-Jordan elimination without pivoting (A_1 is SPD, or has a positive-
// definite symmetric part), in FP64.
template <typename T>
__global__ void coarse_setup_smem_kernel(int n, bool ns, const T* __restrict__ A,
                                         const int* __restrict__ fidx, int nf,
                                         double* __restrict__ Ainv, int* __restrict__ err) {
  extern __shared__ double M[];
  double* colk = M + (size_t)nf * nf;
  const int nE = n * n;
  for (int t = threadIdx.x; t < nf * nf; t += blockDim.x) M[t] = 0.0;
  __syncthreads();
  for (int t = threadIdx.x; t < nE * 64; t += blockDim.x) {
    const int e = t >> 6, r = (t >> 3) & 7, c = t & 7;
    int ed[4];
    elem_edges(n, e, ed);
    const int fr = fidx[ed[r >> 1]], fc = fidx[ed[c >> 1]];
    if (fr < 0 || fc < 0) continue;
    atomicAdd(&M[(size_t)(fr * 2 + (r & 1)) * nf + fc * 2 + (c & 1)],
              (double)A[(size_t)(ns ? r * 8 + c : pk_any(r, c)) * nE + e]);
  }
  __syncthreads();
  __shared__ double piv;
  for (int k = 0; k < nf; ++k) {
    if (threadIdx.x == 0) {
      double d = M[(size_t)k * nf + k];
      if (!(d > 0.0)) {
        atomicOr(err, 8);
        d = 1.0;
      }
      piv = 1.0 / d;
      M[(size_t)k * nf + k] = 1.0;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nf; j += blockDim.x) M[(size_t)k * nf + j] *= piv;
    for (int i = threadIdx.x; i < nf; i += blockDim.x) colk[i] = (i == k) ? 0.0 : M[(size_t)i * nf + k];
    __syncthreads();
    for (int t = threadIdx.x; t < nf * nf; t += blockDim.x) {
      const int i = t / nf, j = t - i * nf;
      if (i == k) continue;
      if (j == k)
        M[t] = -colk[i] * M[(size_t)k * nf + k];
      else
        M[t] -= colk[i] * M[(size_t)k * nf + j];
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < nf * nf; t += blockDim.x) Ainv[t] = M[t];
}

// Coarsest level: the dense FP64 inverse A_1^-1 = L^-T L^-1 is formed once at
// set-up from the Cholesky factor; each V-cycle applies it as one dense
// matrix-vector product (no sequential triangular sweeps).
__global__ void chol_linv_kernel(int nf, const double* __restrict__ L, double* __restrict__ Li) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;      // column of L^-1
  if (j >= nf) return;
  for (int i = 0; i < j; ++i) Li[(size_t)i * nf + j] = 0.0;
  for (int i = j; i < nf; ++i) {
    double s = (i == j) ? 1.0 : 0.0;
    for (int k = j; k < i; ++k) s -= L[(size_t)i * nf + k] * Li[(size_t)k * nf + j];
    Li[(size_t)i * nf + j] = s / L[(size_t)i * nf + i];
  }
}

__global__ void chol_gram_kernel(int nf, const double* __restrict__ Li, double* __restrict__ Ainv) {
  const int i = blockIdx.x;                                  // row of A^-1
  for (int j = threadIdx.x; j < nf; j += blockDim.x) {
    double s = 0.0;
    for (int k = (i > j ? i : j); k < nf; ++k) s += Li[(size_t)k * nf + i] * Li[(size_t)k * nf + j];
    Ainv[(size_t)i * nf + j] = s;
  }
}

// e = A_1^-1 r on the coarsest level's interior dofs; w: nf doubles visible
// to the whole block
template <typename T>
__device__ __forceinline__ void coarse_apply_block(int n, const int* __restrict__ fidx,
                                                   const int* __restrict__ fedge, int nf,
                                                   const double* Ainv, const T* r, T* e,
                                                   double* w) {
  const int nedge = 2 * n * (n + 1);
  for (int ed = threadIdx.x; ed < nedge; ed += blockDim.x) {
    const int f = fidx[ed];
    if (f >= 0) {
      w[f * 2] = (double)r[ed];
      w[f * 2 + 1] = (double)r[(size_t)nedge + ed];
    } else {
      e[ed] = T(0);
      e[(size_t)nedge + ed] = T(0);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nf; i += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < nf; ++j) s += Ainv[(size_t)i * nf + j] * w[j];
    e[(size_t)(i & 1) * nedge + fedge[i >> 1]] = (T)s;
  }
}

template <typename T>
__global__ void coarse_solve_kernel(int n, const int* __restrict__ fidx, const int* __restrict__ fedge,
                                    int nf, const double* __restrict__ Ainv, const T* __restrict__ r,
                                    T* __restrict__ e) {
  extern __shared__ double cw[];
  const size_t o = (size_t)blockIdx.y * 4 * n * (n + 1);   // right-hand side of a blocked solve
  coarse_apply_block<T>(n, fidx, fedge, nf, Ainv, r + o, e + o, cw);
}

// ------------------------------------------- fused V-cycle on the P1 tail
// P1 (two modes per edge) element matvec y += A x for one element, and the
// block-Jacobi update of one edge, for the single-block tail kernel.
template <typename T>
__device__ __forceinline__ void matvec_p1_item(int n, bool ns, const T* __restrict__ A, const T* x,
                                               T* y, int e) {
  const int nE = n * n, nedge = 2 * n * (n + 1);
  int ed[4];
  elem_edges(n, e, ed);
  T xl[8], yl[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    xl[c] = x[(size_t)(c & 1) * nedge + ed[c >> 1]];
    yl[c] = T(0);
  }
  if (ns) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) yl[r] += A[(size_t)(r * 8 + c) * nE + e] * xl[c];
  } else {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
#pragma unroll
      for (int c = 0; c < r; ++c) {
        const T a = A[(size_t)pk(r, c) * nE + e];
        yl[r] += a * xl[c];
        yl[c] += a * xl[r];
      }
      yl[r] += A[(size_t)pk(r, r) * nE + e] * xl[r];
    }
  }
#pragma unroll
  for (int le = 0; le < 4; ++le) {
    if (bnd_edge(n, ed[le])) continue;
    atomicAdd(&y[ed[le]], yl[le * 2]);
    atomicAdd(&y[(size_t)nedge + ed[le]], yl[le * 2 + 1]);
  }
}

template <typename T>
__device__ __forceinline__ void bj_p1_item(int n, bool ns, const T* __restrict__ Dinv, const T* r,
                                           T* y, T* e, T omega, bool first, int edge) {
  const int nedge = 2 * n * (n + 1);
  if (bnd_edge(n, edge)) return;
  const T d0 = first ? r[edge] : r[edge] - y[edge];
  const T d1 = first ? r[nedge + edge] : r[nedge + edge] - y[nedge + edge];
  if (!first) {
    y[edge] = T(0);
    y[nedge + edge] = T(0);
  }
  // packed [d00, d10, d11] or full [d00, d01, d10, d11]
  const T a00 = Dinv[edge], a10 = Dinv[(size_t)nedge + edge], a11 = Dinv[(size_t)2 * nedge + edge];
  T s0, s1;
  if (ns) {
    const T b10 = a11, b11 = Dinv[(size_t)3 * nedge + edge];
    s0 = a00 * d0 + a10 * d1;
    s1 = b10 * d0 + b11 * d1;
  } else {
    s0 = a00 * d0 + a10 * d1;
    s1 = a10 * d0 + a11 * d1;
  }
  if (first) {
    e[edge] = omega * s0;
    e[nedge + edge] = omega * s1;
  } else {
    e[edge] += omega * s0;
    e[nedge + edge] += omega * s1;
  }
}

// Edge-centric P1 operator, one thread per edge gathering both elements'
// rows (no atomics): SWEEP out = x + omega D^-1 (r - A x), else out = A x.
template <typename T, bool NS, bool SWEEP>
__global__ void edge_p1_kernel(const P1Geom g, const T* __restrict__ A, const T* __restrict__ Dinv,
                               const T* __restrict__ r, const T* __restrict__ x,
                               T* __restrict__ out, T omega) {
  const int E = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t o = (size_t)blockIdx.y * 2 * g.nedge;        // right-hand side of a blocked solve
  if (E < g.nedge) p1_edge<T, NS, SWEEP>(g, A, Dinv, r + o, x + o, out + o, omega, E);
}

template <typename T>
__device__ __forceinline__ void stage_copy(T* dst, const T* __restrict__ src, int count) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) dst[i] = src[i];
}

// One thread block runs Algorithm 1 on every level of the tail (P1 levels
// with few macro-elements down to the coarsest).  The level vectors r, e, y
// and all level operators of the tail are staged into shared memory at the
// start, and the steps are separated by block barriers instead of kernel
// launches.
template <typename T, int NTHR>
__global__ void __launch_bounds__(NTHR) vcycle_tail_kernel(const TailParams<T> P) {
  extern __shared__ __align__(16) unsigned char tail_smem[];
  const int tid = threadIdx.x, nth = blockDim.x;
  T* sm = reinterpret_cast<T*>(tail_smem);
  double* w = reinterpret_cast<double*>(tail_smem + P.w_off);
  const bool staged_inv = P.ainv_off >= 0;
  double* ainv_s = reinterpret_cast<double*>(tail_smem + (staged_inv ? P.ainv_off : 0));
  const double* ainv = staged_inv ? ainv_s : P.Ainv;
  for (int l = 0; l < P.nlev; ++l) {
    const TailLevel<T>& L = P.lv[l];
    T* base = sm + L.voff;
    for (int i = tid; i < 6 * L.nEdge; i += nth) base[i] = T(0);
    if (L.staged) {
      const int nE = L.n * L.n, nC = nE / 4;
      const int na = P.ns ? 64 : 36, nd2 = P.ns ? 4 : 3;
      stage_copy<T>(sm + L.a_off, L.A, na * nE);
      stage_copy<T>(sm + L.dinv_off, L.Dinv, nd2 * L.nEdge);
      stage_copy<T>(sm + L.aii_off, L.AIIinv, na * nC);
      stage_copy<T>(sm + L.y_off, L.Y, 128 * nC);
      stage_copy<T>(sm + L.pi_off, L.Pi, 64 * nC);
      if (P.ns) stage_copy<T>(sm + L.rt_off, L.Rt, 64 * nC);
    }
  }
  if (staged_inv) stage_copy<double>(ainv_s, P.Ainv, P.nf * P.nf);
  __syncthreads();
  {
    T* r0 = sm + P.lv[0].voff;
    for (int i = tid; i < 2 * P.lv[0].nEdge; i += nth) r0[i] = P.r_in[i];
  }
  __syncthreads();
  // down sweep: steps 2-4 of Algorithm 1
  for (int l = 0; l + 1 < P.nlev; ++l) {
    const TailLevel<T>& L = P.lv[l];
    const int n = L.n, nE = n * n, ned = L.nEdge, nc = n / 2;
    T* r = sm + L.voff;
    T* e = r + 2 * ned;
    T* y = e + 2 * ned;
    const T* A = L.staged ? sm + L.a_off : L.A;
    const T* Dinv = L.staged ? sm + L.dinv_off : L.Dinv;
    const T* AIIinv = L.staged ? sm + L.aii_off : L.AIIinv;
    const T* Yb = L.staged ? sm + L.y_off : L.Y;
    const T* Rt = P.ns ? (L.staged ? sm + L.rt_off : L.Rt) : (L.staged ? sm + L.pi_off : L.Pi);
    const bool ns = P.ns != 0;
    for (int i = tid; i < ned; i += nth) bj_p1_item<T>(n, ns, Dinv, r, y, e, P.omega, true, i);
    __syncthreads();
    for (int it = 1; it < L.m; ++it) {
      for (int i = tid; i < nE; i += nth) matvec_p1_item<T>(n, ns, A, e, y, i);
      __syncthreads();
      for (int i = tid; i < ned; i += nth) bj_p1_item<T>(n, ns, Dinv, r, y, e, P.omega, false, i);
      __syncthreads();
    }
    if (P.lc != HDGMG_LC_NONE) {
      for (int i = tid; i < 8 * nc * nc; i += nth) local_correction_item<T>(nc, ns, AIIinv, Yb, r, e, i);
      __syncthreads();
    }
    for (int i = tid; i < nE; i += nth) matvec_p1_item<T>(n, ns, A, e, y, i);
    __syncthreads();
    T* rc = sm + P.lv[l + 1].voff;
    for (int i = tid; i < 2 * P.lv[l + 1].nEdge; i += nth) restrict_h_item<T>(nc, Rt, r, y, rc, i);
    __syncthreads();
  }
  {  // B_1 = A_1^-1
    const TailLevel<T>& L = P.lv[P.nlev - 1];
    T* r = sm + L.voff;
    coarse_apply_block<T>(L.n, P.fidx, P.fedge, P.nf, ainv, r, r + 2 * L.nEdge, w);
    __syncthreads();
  }
  // up sweep: steps 4-6
  for (int l = P.nlev - 2; l >= 0; --l) {
    const TailLevel<T>& L = P.lv[l];
    const int n = L.n, nE = n * n, ned = L.nEdge, nc = n / 2;
    T* r = sm + L.voff;
    T* e = r + 2 * ned;
    T* y = e + 2 * ned;
    const T* A = L.staged ? sm + L.a_off : L.A;
    const T* Dinv = L.staged ? sm + L.dinv_off : L.Dinv;
    const T* AIIinv = L.staged ? sm + L.aii_off : L.AIIinv;
    const T* Yb = L.staged ? sm + L.y_off : L.Y;
    const T* Pi = L.staged ? sm + L.pi_off : L.Pi;
    const T* ec = sm + P.lv[l + 1].voff + 2 * P.lv[l + 1].nEdge;
    const bool ns = P.ns != 0;
    for (int i = tid; i < 8 * nc * nc + 2 * P.lv[l + 1].nEdge; i += nth)
      prolong_h_item<T>(nc, Pi, ec, e, y, i);
    __syncthreads();
    if (P.lc == HDGMG_LC_BOTH) {
      for (int i = tid; i < 8 * nc * nc; i += nth) local_correction_item<T>(nc, ns, AIIinv, Yb, r, e, i);
      __syncthreads();
    }
    for (int it = 0; it < L.m; ++it) {
      for (int i = tid; i < nE; i += nth) matvec_p1_item<T>(n, ns, A, e, y, i);
      __syncthreads();
      for (int i = tid; i < ned; i += nth) bj_p1_item<T>(n, ns, Dinv, r, y, e, P.omega, false, i);
      __syncthreads();
    }
  }
  {
    const T* e0 = sm + P.lv[0].voff + 2 * P.lv[0].nEdge;
    for (int i = tid; i < 2 * P.lv[0].nEdge; i += nth) P.e_out[i] = e0[i];
  }
}

// ------------------------------------ persistent V-cycle over the P1 levels
// Algorithm 1 from the first P1 level down to B_1 = A_1^-1 and back, in one
// cooperative launch: each step is a grid-stride loop over the work items of
// the launched kernels (the same item functions, so the same arithmetic), and
// a grid barrier replaces each kernel boundary.  Levels from P.tail on run on
// block 0 alone with block barriers while the other blocks wait at a single
// grid barrier.

__device__ __forceinline__ unsigned long long pc_now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long pc_ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void pc_red_release(unsigned long long* p) {
  asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(p) : "memory");
}

// one-dimensional bulk copies (TMA) global -> shared, completing on an mbarrier
__device__ __forceinline__ unsigned pc_smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void pc_mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(pc_smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void pc_mbar_expect(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(pc_smem_addr(bar)),
               "r"(bytes) : "memory");
}
__device__ __forceinline__ void pc_bulk_copy(void* dst, const void* src, unsigned bytes,
                                             unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          pc_smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(pc_smem_addr(bar))
      : "memory");
}
// L2 prefetch of [src, src + bytes): 16-byte aligned start, size a multiple
// of 16 bytes (no shared memory, no completion to wait for)
__device__ __forceinline__ void pc_l2_prefetch(const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Thread 0 of every block asks L2 for its share (1 / gridDim.x, in 16-byte
// units) of each operator array of the grid levels, so that the first step on
// each level finds its operators in L2 (the FP64 matvec between two cycles
// streams 124 MB through L2 at 256^2, p = 4).  Every array is a whole device
// allocation whose size is a multiple of 16 bytes (level sizes: 36 n^2,
// 3 or 4 * 2 n (n + 1), 36, 64 or 128 * n^2 / 4 entries of 4 or 8 bytes).
template <typename T, bool NS>
__device__ void pc_prefetch_grid_levels(const PCycleParams<T>& P, int top) {
  const int na = NS ? 64 : 36;
  auto share = [&](const void* base, size_t bytes) {
    const size_t units = bytes / 16, per = (units + gridDim.x - 1) / gridDim.x;
    const size_t u0 = per * blockIdx.x;
    if (u0 >= units) return;
    const size_t nu = units - u0 < per ? units - u0 : per;
    pc_l2_prefetch(static_cast<const char*>(base) + 16 * u0, (unsigned)(16 * nu));
  };
  for (int l = 0; l < top; ++l) {
    const PLevel<T>& L = P.lv[l];
    const size_t nE = L.g.nE, ned = L.g.nedge, nC = nE / 4, sz = sizeof(T);
    share(L.A, na * nE * sz);
    share(L.Dinv, (NS ? 4 : 3) * ned * sz);
    if (l + 1 < P.nlev) {
      share(L.AIIinv, na * nC * sz);
      share(L.Y, 128 * nC * sz);
      share(L.Pi, 64 * nC * sz);
      if (NS) share(L.Rt, 64 * nC * sz);
    }
  }
}

__device__ __forceinline__ bool pc_mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(pc_smem_addr(bar)), "r"(parity) : "memory");
  return ok != 0;
}
// wait for phase 0 of bar, at most wait_ns; false when the limit ran out
__device__ __forceinline__ bool pc_mbar_wait(unsigned long long* bar, unsigned long long wait_ns) {
  if (pc_mbar_test(bar, 0)) return true;
  const unsigned long long t0 = pc_now_ns();
  while (!pc_mbar_test(bar, 0))
    if (pc_now_ns() - t0 > wait_ns) return false;
  return true;
}

struct PcSync {
  unsigned long long target = 0;   // thread 0: arrivals that end the current barrier
  int first = 1;                   // no barrier passed yet
  int nstep = 0;                   // thread 0 of block 0: trace records written
};

// Step trace (P.trace non-null): thread 0 of block 0 records, after each
// barrier, the global timer and the tag of the step that barrier ended
// (level * 16 + kind, the PcStep values), up to P.trace_cap records.
enum PcStep {
  kPcStart = 0, kPcFirst = 1, kPcSweepDown = 2, kPcLc = 3, kPcResidRestrict = 4, kPcResid = 5,
  kPcRestrict = 6, kPcCoarse = 7, kPcProlong = 8, kPcSweepUp = 9, kPcTail = 10, kPcEnd = 11
};

template <typename T>
__device__ __forceinline__ void pc_stamp(const PCycleParams<T>& P, PcSync& st, int tag) {
  if (P.trace && blockIdx.x == 0 && threadIdx.x == 0 && st.nstep < P.trace_cap) {
    P.trace[2 * st.nstep] = pc_now_ns();
    P.trace[2 * st.nstep + 1] = (unsigned long long)tag;
    ++st.nstep;
  }
}

// Grid barrier on a monotonic arrival count: thread 0 of every block adds one
// with release semantics (after the block barrier, so the block's writes are
// published) and waits, with acquire loads, until the count reaches the next
// multiple of the grid size -- no reset, no second round trip.  The count is a
// multiple of the grid size between launches, so each launch starts from the
// multiple below the value it reads.  A wait longer than P.wait_ns sets bit 0
// of *P.err; an error set by any block ends every later wait at once (a block
// that gave up never arrives again, so no later barrier can complete).
// Returns false in every thread of the block once the wait failed.
template <typename T>
__device__ bool pc_grid_sync(const PCycleParams<T>& P, PcSync& st, volatile int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    st.target += gridDim.x;
    if (!(P.withhold && st.first)) pc_red_release(P.bar);
    st.first = 0;
    if (pc_ld_acquire(P.bar) < st.target) {
      const unsigned long long t0 = pc_now_ns();
      unsigned spin = 0;
      while (pc_ld_acquire(P.bar) < st.target) {
        if ((++spin & 15u) == 0) {
          if (*(volatile int*)P.err != 0) {
            ok = 0;
            break;
          }
          if (pc_now_ns() - t0 > P.wait_ns) {
            atomicOr(P.err, 1);
            ok = 0;
            break;
          }
        }
      }
    }
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

template <typename T>
__device__ __forceinline__ bool pc_sync(const PCycleParams<T>& P, bool grid, PcSync& st,
                                        volatile int* s_ok, int tag) {
  if (grid && !pc_grid_sync<T>(P, st, s_ok)) return false;
  if (!grid) __syncthreads();
  pc_stamp<T>(P, st, tag);
  return true;
}

// The two buffers a P1 level's sweeps ping-pong between, ordered so that the
// correction ends in L.e: the first sweep writes bufs[1]; with the fused
// prolongation + second local correction (LC_BOTH) the up sweep has one more
// buffer swap.
template <typename T>
__device__ __forceinline__ void pc_bufs(const PCycleParams<T>& P, int l, T* bufs[2]) {
  const PLevel<T>& L = P.lv[l];
  if (P.lc == HDGMG_LC_BOTH) {
    bufs[0] = L.y;
    bufs[1] = L.e;
  } else {
    bufs[0] = L.e;
    bufs[1] = L.y;
  }
}

// Grid-stride loop over the k x COUNT items of one step (k = P.nrhs right-hand
// sides of a blocked solve): j = rhs * COUNT + t; the body sees rhs and t.
#define PC_FOR(COUNT, FD)                                                         \
  for (int j_ = i0, cnt_ = (COUNT); j_ < P.nrhs * cnt_; j_ += di)                 \
    if (const int rhs = P.nrhs == 1 ? 0 : fdiv(j_, (FD)), t = j_ - rhs * cnt_; true)

// Steps 2-4 on P1 level l down to the restriction into level l + 1.  The
// first sweep from e = 0 of a level other than lv[0] and the first level of
// a staged block-0 tail is fused into the restriction above it; after a
// local correction the residual and the restriction are one step
// (p1_resid_restrict2).  Vectors of right-hand side rhs are offset by
// rhs * 2 n_edges (coarse level: rhs * 2 n_edges(coarse)).
template <typename T, bool NS>
__device__ bool pc_down(const PCycleParams<T>& P, int l, int i0, int di, bool grid, PcSync& st,
                        volatile int* s_ok) {
  const PLevel<T>& L = P.lv[l];
  const P1Geom& g = L.g;
  const int ned = g.nedge, V = 2 * g.nedge, Vc = 2 * g.nedc;
  T* bufs[2];
  pc_bufs<T>(P, l, bufs);
  int cur = 1;
  if (l == 0 || (P.staged && l == P.tail)) {
    if (l == 0 && P.rp_r0) {
      const int V0 = P.rp_nd0 * ned;
      PC_FOR(ned, g.dne)
      p1_first_restrict_p<T, NS>(g, P.rp_nd0, L.Dinv, P.rp_r0 + rhs * V0, P.rp_y0 + rhs * V0,
                                 L.r + rhs * V, bufs[1] + rhs * V, P.omega, t);
    } else {
      PC_FOR(ned, g.dne) p1_first<T, NS>(g, L.Dinv, L.r + rhs * V, bufs[1] + rhs * V, P.omega, t);
    }
    if (!pc_sync<T>(P, grid, st, s_ok, l * 16 + kPcFirst)) return false;
  }
  for (int it = 1; it < L.m; ++it) {
    PC_FOR(ned, g.dne)
    p1_edge<T, NS, true>(g, L.A, L.Dinv, L.r + rhs * V, (cur ? bufs[1] : bufs[0]) + rhs * V,
                         (cur ? bufs[0] : bufs[1]) + rhs * V, P.omega, t);
    cur ^= 1;
    if (!pc_sync<T>(P, grid, st, s_ok, l * 16 + kPcSweepDown)) return false;
  }
  // the next level's first sweep joins its restriction unless it is the
  // coarsest level (no smoothing) or the first, staged level of the tail
  const bool fuse_next = l + 1 < P.nlev - 1 && !(P.staged && l + 1 == P.tail);
  T* rc = P.lv[l + 1].r;
  T* cb[2];
  pc_bufs<T>(P, l + 1, cb);
  T* ec = fuse_next ? cb[1] : nullptr;
  const T* Dc = P.lv[l + 1].Dinv;
  if (P.lc != HDGMG_LC_NONE) {
    PC_FOR(8 * g.nC, g.dlc)
    p1_lc<T, NS>(g, L.AIIinv, L.Y, L.r + rhs * V, (cur ? bufs[1] : bufs[0]) + rhs * V, t);
    if (!pc_sync<T>(P, grid, st, s_ok, l * 16 + kPcLc)) return false;
    PC_FOR(2 * g.nedc, g.dc2)
    p1_resid_restrict2<T, NS>(g, L.A, L.r + rhs * V, (cur ? bufs[1] : bufs[0]) + rhs * V, rc + rhs * Vc, Dc,
                              ec ? ec + rhs * Vc : nullptr, P.omega, t);
    return pc_sync<T>(P, grid, st, s_ok, l * 16 + kPcResidRestrict);
  }
  PC_FOR(ned, g.dne)
  p1_edge<T, NS, false>(g, L.A, L.Dinv, L.r + rhs * V, (cur ? bufs[1] : bufs[0]) + rhs * V,
                        (cur ? bufs[0] : bufs[1]) + rhs * V, P.omega, t);
  if (!pc_sync<T>(P, grid, st, s_ok, l * 16 + kPcResid)) return false;
  PC_FOR(g.nedc, g.dc1)
  p1_restrict_first<T, NS>(g, L.Rt, L.r + rhs * V, (cur ? bufs[0] : bufs[1]) + rhs * V, rc + rhs * Vc, Dc,
                           ec ? ec + rhs * Vc : nullptr, P.omega, t);
  return pc_sync<T>(P, grid, st, s_ok, l * 16 + kPcRestrict);
}

// B_1 = A_1^-1 on the coarsest level: every participating block gathers the
// interior right-hand sides into w (shared memory, [k][nf]), then one item per
// (right-hand side, row).
template <typename T>
__device__ bool pc_coarse(const PCycleParams<T>& P, int i0, int di, bool grid, PcSync& st,
                          volatile int* s_ok, double* w) {
  const PLevel<T>& L = P.lv[P.nlev - 1];
  const int ned = L.g.nedge, nf = P.nf, V = 2 * ned;
  for (int q = threadIdx.x; q < P.nrhs * nf; q += blockDim.x) {
    const int rq = q / nf, jq = q - rq * nf;
    w[q] = (double)L.r[rq * V + (jq & 1) * ned + P.fedge[jq >> 1]];
  }
  __syncthreads();
  PC_FOR(ned + nf, P.dco) {
    if (t < ned) {
      if (P.fidx[t] < 0) {
        L.e[rhs * V + t] = T(0);
        L.e[rhs * V + ned + t] = T(0);
      }
    } else {
      const int row = t - ned;
      const double* Ar = P.Ainv + (size_t)row * nf;
      const double* wr = w + rhs * nf;
      double s = 0.0;
      for (int j = 0; j < nf; ++j) s += Ar[j] * wr[j];
      L.e[rhs * V + (row & 1) * ned + P.fedge[row >> 1]] = (T)s;
    }
  }
  return pc_sync<T>(P, grid, st, s_ok, (P.nlev - 1) * 16 + kPcCoarse);
}

// Steps 4-6 on P1 level l: prolongation from level l + 1 (fused with the
// second local correction under LC_BOTH), post-smoothing; the correction ends
// in L.e.  `final`: the last step of the kernel (no barrier after it).
template <typename T, bool NS>
__device__ bool pc_up(const PCycleParams<T>& P, int l, int i0, int di, bool grid, PcSync& st,
                      volatile int* s_ok, bool final) {
  const PLevel<T>& L = P.lv[l];
  const P1Geom& g = L.g;
  const int ned = g.nedge, V = 2 * g.nedge, Vc = 2 * g.nedc;
  T* bufs[2];
  pc_bufs<T>(P, l, bufs);
  int cur = L.m & 1;                   // where the down sweep left the correction
  const T* ec = P.lv[l + 1].e;
  if (P.lc == HDGMG_LC_BOTH) {
    PC_FOR(8 * g.nC + 2 * g.nedc, g.dpro)
    p1_prolong_lc<T, NS>(g, L.AIIinv, L.Y, L.r + rhs * V, ec + rhs * Vc, (cur ? bufs[1] : bufs[0]) + rhs * V,
                         (cur ? bufs[0] : bufs[1]) + rhs * V, t);
    cur ^= 1;
  } else {
    PC_FOR(8 * g.nC + 2 * g.nedc, g.dpro)
    p1_prolong<T>(g, L.Pi, ec + rhs * Vc, (cur ? bufs[1] : bufs[0]) + rhs * V, (cur ? bufs[0] : bufs[1]) + rhs * V, t);
  }
  if (!pc_sync<T>(P, grid, st, s_ok, l * 16 + kPcProlong)) return false;
  for (int it = 0; it < L.m; ++it) {
    PC_FOR(ned, g.dne)
    p1_edge<T, NS, true>(g, L.A, L.Dinv, L.r + rhs * V, (cur ? bufs[1] : bufs[0]) + rhs * V,
                         (cur ? bufs[0] : bufs[1]) + rhs * V, P.omega, t);
    cur ^= 1;
    if (final && it + 1 == L.m) return true;
    if (!pc_sync<T>(P, grid, st, s_ok, l * 16 + kPcSweepUp)) return false;
  }
  return true;
}

// block copy of `count` elements; 16-byte vectors when both ends allow it,
// several loads in flight per thread
template <typename T>
__device__ __forceinline__ void pc_copy(T* dst, const T* src, int count) {
  constexpr int V = 16 / sizeof(T);
  if ((((uintptr_t)dst | (uintptr_t)src) & 15) == 0) {
    const int nv = count / V;
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
    int i = threadIdx.x;
    for (; i + 3 * (int)blockDim.x < nv; i += 4 * blockDim.x) {
      const float4 a = s4[i], b = s4[i + blockDim.x], c = s4[i + 2 * blockDim.x],
                   d = s4[i + 3 * blockDim.x];
      d4[i] = a;
      d4[i + blockDim.x] = b;
      d4[i + 2 * blockDim.x] = c;
      d4[i + 3 * blockDim.x] = d;
    }
    for (; i < nv; i += blockDim.x) d4[i] = s4[i];
    for (int j = nv * V + threadIdx.x; j < count; j += blockDim.x) dst[j] = src[j];
  } else {
    for (int j = threadIdx.x; j < count; j += blockDim.x) dst[j] = src[j];
  }
}

// Block 0 runs levels P.tail ... coarsest.  Staged: their operators, the
// coarsest inverse and all their vectors are first copied into shared memory
// (a copy of the parameters points there), lv[tail].r is taken from global
// memory (where the grid's restriction put it) and lv[tail].e is written back.
// Block 0 of a staged tail: thread 0 requests the tail's operators and the
// coarsest inverse into shared memory by bulk copies on one mbarrier, before
// the grid levels start, so that the copies overlap their work.  Every
// array is a whole device allocation (16-byte aligned, its size a multiple
// of 16 bytes by construction of the level sizes).
template <typename T, bool NS>
__device__ void pc_prefetch(const PCycleParams<T>& P, unsigned char* smem, unsigned long long* mbar) {
  const int last = P.nlev - 1;
  const int na = NS ? 64 : 36;
  pc_mbar_init(mbar);
  pc_mbar_expect(mbar, (unsigned)P.stage_bytes);
  for (int l = P.tail; l < last; ++l) {
    const PLevel<T>& gl = P.lv[l];
    const unsigned nE = gl.g.nE, ned = gl.g.nedge, nC = nE / 4, sz = sizeof(T);
    pc_bulk_copy(smem + gl.so_A, gl.A, na * nE * sz, mbar);
    pc_bulk_copy(smem + gl.so_D, gl.Dinv, (NS ? 4 : 3) * ned * sz, mbar);
    pc_bulk_copy(smem + gl.so_AII, gl.AIIinv, na * nC * sz, mbar);
    pc_bulk_copy(smem + gl.so_Y, gl.Y, 128 * nC * sz, mbar);
    pc_bulk_copy(smem + gl.so_Pi, gl.Pi, 64 * nC * sz, mbar);
    if (gl.so_Rt != gl.so_Pi) pc_bulk_copy(smem + gl.so_Rt, gl.Rt, 64 * nC * sz, mbar);
  }
  pc_bulk_copy(smem + P.so_Ainv, P.Ainv, (unsigned)(sizeof(double) * P.nf * P.nf), mbar);
}

template <typename T, bool NS>
__device__ void pc_tail(const PCycleParams<T>& P, PCycleParams<T>& sP, unsigned char* smem,
                        unsigned long long* mbar, PcSync& st, volatile int* s_ok) {
  const int last = P.nlev - 1, t0 = P.tail;
  const int ti = threadIdx.x, td = blockDim.x;
  const PCycleParams<T>* Q = &P;
  double* w = reinterpret_cast<double*>(smem + P.so_w);
  if (P.staged) {
    {   // sP = P by the whole block, then thread 0 points the tail levels at shared memory
      static_assert(sizeof(PCycleParams<T>) % 8 == 0, "parameter block copied as 8-byte words");
      const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&P);
      unsigned long long* dst = reinterpret_cast<unsigned long long*>(&sP);
      for (int i = threadIdx.x; i < (int)(sizeof(PCycleParams<T>) / 8); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int l = t0; l <= last; ++l) {
        PLevel<T>& q = sP.lv[l];
        const int ned = q.g.nedge;
        T* v = reinterpret_cast<T*>(smem + q.so_v);
        q.r = v;
        q.e = v + 2 * ned;
        q.y = v + 4 * ned;
        if (l < last) {
          q.A = reinterpret_cast<const T*>(smem + q.so_A);
          q.Dinv = reinterpret_cast<const T*>(smem + q.so_D);
          q.AIIinv = reinterpret_cast<const T*>(smem + q.so_AII);
          q.Y = reinterpret_cast<const T*>(smem + q.so_Y);
          q.Pi = reinterpret_cast<const T*>(smem + q.so_Pi);
          q.Rt = reinterpret_cast<const T*>(smem + q.so_Rt);
        }
      }
      sP.Ainv = reinterpret_cast<const double*>(smem + P.so_Ainv);
    }
    for (int l = t0; l <= last; ++l) {
      const PLevel<T>& gl = P.lv[l];
      T* v = reinterpret_cast<T*>(smem + gl.so_v);
      for (int i = threadIdx.x; i < 6 * gl.g.nedge; i += blockDim.x) v[i] = T(0);
    }
    __syncthreads();
    if (!(t0 == 0 && P.rp_r0)) {
      const int ned = P.lv[t0].g.nedge;
      pc_copy<T>(reinterpret_cast<T*>(smem + P.lv[t0].so_v), P.lv[t0].r, 2 * ned);
    }
    // the operators were requested at the start of the kernel (pc_prefetch)
    if (!pc_mbar_wait(mbar, P.wait_ns)) {
      atomicOr(P.err, 2);
      pc_mbar_wait(mbar, P.wait_ns);   // let copies still in flight land before leaving
      *s_ok = 0;
    }
    __syncthreads();
    if (!*s_ok) return;
    Q = &sP;
  }
  for (int l = t0; l < last; ++l) pc_down<T, NS>(*Q, l, ti, td, false, st, s_ok);
  pc_coarse<T>(*Q, ti, td, false, st, s_ok, w);
  for (int l = last - 1; l >= t0; --l)
    pc_up<T, NS>(*Q, l, ti, td, false, st, s_ok, l == 0 && !P.staged);
  if (P.staged) {
    __syncthreads();
    const int ned = P.lv[t0].g.nedge;
    pc_copy<T>(P.lv[t0].e, reinterpret_cast<const T*>(smem + P.lv[t0].so_v) + 2 * ned, 2 * ned);
  }
}

template <typename T, bool NS, int NTHR>
__device__ void pc_body(const PCycleParams<T>& P, PCycleParams<T>& sP, unsigned char* smem,
                        unsigned long long* mbar, PcSync& st, volatile int* s_ok, int* s_tail) {
  const int last = P.nlev - 1;
  const int top = P.tail < last ? P.tail : last;   // levels [0, top) run on the whole grid
  // item j of a grid step goes to warp j / 32 mod (blocks x warps), warps
  // numbered across the blocks first: a level with fewer items than threads
  // spreads over every SM (its loads use all L1s) instead of filling the
  // first blocks; lane pairs (j, j ^ 1) stay in one warp
  const int gi = (((threadIdx.x >> 5) * gridDim.x + blockIdx.x) << 5) + (threadIdx.x & 31);
  const int gd = gridDim.x * NTHR;
  for (int l = 0; l < top; ++l)
    if (!pc_down<T, NS>(P, l, gi, gd, true, st, s_ok)) return;
  if (P.tail <= last) {
    if (blockIdx.x == 0) {
      *s_tail = 1;
      pc_tail<T, NS>(P, sP, smem, mbar, st, s_ok);
    }
    if (top > 0 && !pc_sync<T>(P, true, st, s_ok, P.tail * 16 + kPcTail)) return;
  } else {
    if (!pc_coarse<T>(P, gi, gd, true, st, s_ok, reinterpret_cast<double*>(smem + P.so_w))) return;
  }
  for (int l = top - 1; l >= 0; --l)
    if (!pc_up<T, NS>(P, l, gi, gd, true, st, s_ok, l == 0)) return;
}

template <typename T, bool NS, int NTHR>
__global__ void __launch_bounds__(NTHR, 1) pcycle_kernel(const __grid_constant__ PCycleParams<T> P) {
  extern __shared__ __align__(16) unsigned char pc_smem[];
  __shared__ int s_ok, s_tail;
  __shared__ __align__(8) unsigned long long s_mbar;
  __shared__ PCycleParams<T> sP;
  PcSync st;
  const bool prefetch = P.staged && blockIdx.x == 0;
  if (threadIdx.x == 0) {
    const unsigned long long c0 = *(volatile unsigned long long*)P.bar;
    st.target = c0 - c0 % gridDim.x;
    s_ok = *(volatile int*)P.err == 0;   // a wait of an earlier launch expired: do nothing
    s_tail = 0;
    if (s_ok && prefetch) pc_prefetch<T, NS>(P, pc_smem, &s_mbar);
  }
  __syncthreads();
  if (!s_ok) return;
  if (threadIdx.x == 0 && P.nrhs == 1) {
    const int last = P.nlev - 1;
    pc_prefetch_grid_levels<T, NS>(P, P.tail < last ? P.tail : last);
  }
  pc_stamp<T>(P, st, kPcStart);
  pc_body<T, NS, NTHR>(P, sP, pc_smem, &s_mbar, st, &s_ok, &s_tail);
  pc_stamp<T>(P, st, kPcEnd);
  // block 0 leaves no bulk copy into its shared memory in flight: when the
  // tail was not reached (a barrier wait ran out), wait for the prefetch
  // (bounded) before returning
  if (prefetch && !s_tail && !pc_mbar_wait(&s_mbar, P.wait_ns)) atomicOr(P.err, 2);
}

// ------------------------------------------------ point smoothers (Sec. 4.1)
// The two elements sharing interior edge E, and E's local edge in each.
__device__ __forceinline__ void edge_owners(int n, int E, int el[2], int le[2]) {
  const int nvert = n * (n + 1);
  if (E < nvert) {
    const int j = E / (n + 1), i = E - j * (n + 1);
    el[0] = j * n + i - 1; le[0] = 1;
    el[1] = j * n + i;     le[1] = 0;
  } else {
    const int j = (E - nvert) / n, i = (E - nvert) - j * n;
    el[0] = (j - 1) * n + i; le[0] = 3;
    el[1] = j * n + i;       le[1] = 2;
  }
}

__device__ __forceinline__ int ent(bool ns, int nl, int r, int c) {
  return ns ? r * nl + c : pk_any(r, c);
}

// Dpt[a][E] = 1 / A_{(E,a),(E,a)} (0 on Dirichlet edges)
template <typename T>
__global__ void point_diag_kernel(int n, int nd, bool ns, const T* __restrict__ A,
                                  T* __restrict__ Dpt) {
  const int nedge = 2 * n * (n + 1);
  const int E = blockIdx.x * blockDim.x + threadIdx.x;
  if (E >= nedge) return;
  if (bnd_edge(n, E)) {
    for (int a = 0; a < nd; ++a) Dpt[(size_t)a * nedge + E] = T(0);
    return;
  }
  const int nE = n * n, nl = 4 * nd;
  int el[2], le[2];
  edge_owners(n, E, el, le);
  for (int a = 0; a < nd; ++a) {
    T d = T(0);
    for (int s = 0; s < 2; ++s) {
      const int r = le[s] * nd + a;
      d += A[(size_t)ent(ns, nl, r, r) * nE + el[s]];
    }
    Dpt[(size_t)a * nedge + E] = T(1) / d;
  }
}

template <typename T>
__global__ void pj_update_kernel(int n, int nd, const T* __restrict__ Dpt, const T* __restrict__ r,
                                 T* __restrict__ y, T* __restrict__ e, T omega, int first) {
  const int nedge = 2 * n * (n + 1);
  const int E = blockIdx.x * blockDim.x + threadIdx.x;
  if (E >= nedge || bnd_edge(n, E)) return;
  for (int a = 0; a < nd; ++a) {
    const size_t ix = (size_t)a * nedge + E;
    if (first) {
      e[ix] = omega * Dpt[ix] * r[ix];
    } else {
      e[ix] += omega * Dpt[ix] * (r[ix] - y[ix]);
      y[ix] = T(0);
    }
  }
}

template <typename T>
__global__ void cheb_update_kernel(int n, int nd, const T* __restrict__ Dpt, const T* __restrict__ r,
                                   T* __restrict__ y, T* __restrict__ e, T* __restrict__ d,
                                   const double* __restrict__ coef, int k, int first_e,
                                   int first_d) {
  const int nedge = 2 * n * (n + 1);
  const int E = blockIdx.x * blockDim.x + threadIdx.x;
  if (E >= nedge || bnd_edge(n, E)) return;
  const T c1 = (T)coef[2 * k], c2 = (T)coef[2 * k + 1];
  for (int a = 0; a < nd; ++a) {
    const size_t ix = (size_t)a * nedge + E;
    const T res = first_e ? r[ix] : r[ix] - y[ix];
    if (!first_e) y[ix] = T(0);
    const T dn = first_d ? c2 * Dpt[ix] * res : c1 * d[ix] + c2 * Dpt[ix] * res;
    d[ix] = dn;
    e[ix] = first_e ? dn : e[ix] + dn;
  }
}

// One colour of the point Gauss-Seidel sweep: the edges of a colour share no
// element, so they update in parallel exactly as in sequential order; inside
// an edge the modes go in order (backward: reverse order).  e in place.
template <typename T>
__global__ void gs_colour_kernel(int n, int nd, bool ns, const T* __restrict__ A,
                                 const T* __restrict__ Dpt, const T* __restrict__ r,
                                 T* __restrict__ e, int colour, int backward) {
  const int nedge = 2 * n * (n + 1);
  const int E = blockIdx.x * blockDim.x + threadIdx.x;
  if (E >= nedge || bnd_edge(n, E)) return;
  const int nvert = n * (n + 1);
  const int col = E < nvert ? (E % (n + 1)) % 2 : 2 + ((E - nvert) / n) % 2;
  if (col != colour) return;
  const int nE = n * n, nl = 4 * nd;
  int el[2], le[2];
  edge_owners(n, E, el, le);
  int ed[2][4];
  elem_edges(n, el[0], ed[0]);
  elem_edges(n, el[1], ed[1]);
  for (int t = 0; t < nd; ++t) {
    const int a = backward ? nd - 1 - t : t;
    T s = T(0);
    for (int side = 0; side < 2; ++side) {
      const int rrow = le[side] * nd + a;
      for (int c = 0; c < nl; ++c)
        s += A[(size_t)ent(ns, nl, rrow, c) * nE + el[side]] *
             e[(size_t)(c % nd) * nedge + ed[side][c / nd]];
    }
    const size_t ix = (size_t)a * nedge + E;
    e[ix] += (r[ix] - s) * Dpt[ix];
  }
}

// start vector of the power iteration: 1 + (h mod 1024) / 1024 with
// h = (i * 2654435761) mod 2^32, i = mode * n_edges + edge; 0 on Dirichlet edges
template <typename T>
__global__ void power_start_kernel(int n, int nd, T* __restrict__ x) {
  const int nedge = 2 * n * (n + 1);
  const int E = blockIdx.x * blockDim.x + threadIdx.x;
  if (E >= nedge) return;
  const bool b = bnd_edge(n, E);
  for (int a = 0; a < nd; ++a) {
    const unsigned long long i = (unsigned long long)a * nedge + E;
    const unsigned long long h = (i * 2654435761ull) & 0xffffffffull;
    x[(size_t)a * nedge + E] = b ? T(0) : (T)(1.0 + (double)(h % 1024ull) / 1024.0);
  }
}

template <typename T>
__global__ void scale_by_kernel(int64_t len, const T* __restrict__ Dpt, T* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] *= Dpt[i];
}

template <typename T>
__global__ void normalize_kernel(int64_t len, const T* __restrict__ y, const double* __restrict__ nrm2,
                                 T* __restrict__ x) {
  const double inv = 1.0 / sqrt(*nrm2);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = (T)((double)y[i] * inv);
}

// ------------------------------------------------------------ vector ops
template <typename T>
__global__ void dot_partial_kernel(int64_t len, const T* __restrict__ a,
                                   const T* __restrict__ b, double* __restrict__ partial) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    s += (double)a[i] * (double)b[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void dot_final_kernel(int nparts, const double* __restrict__ partial, double* out) {
  __shared__ double sh[1024];
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += partial[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

template <typename T>
__global__ void mask_kernel(int n, int nd, T* __restrict__ x) {
  const int nedge = 2 * n * (n + 1);
  const int edge = blockIdx.x * blockDim.x + threadIdx.x;
  if (edge >= nedge || !bnd_edge(n, edge)) return;
  for (int k = 0; k < nd; ++k) x[(size_t)k * nedge + edge] = T(0);
}

template <typename A, typename B>
__global__ void convert_kernel(int64_t len, const A* __restrict__ in, B* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (B)in[i];
}

// ---------------------------------------- fused PCG vector kernels
// Dot products finish in the last block to arrive (fixed reduction order, so
// the result is deterministic) and apply the scalar recurrences there:
//   mode 0: scal[1] = p.Ap,     scal[2] = alpha = scal[0] / scal[1]
//   mode 1: scal[3] = r.z,      scal[4] = beta = scal[3] / scal[0], scal[0] = scal[3]
//   mode 2: scal[5] = r.r
template <typename T, typename TB = T>
__global__ void __launch_bounds__(256) dot_fused_kernel(int64_t len, const T* __restrict__ a,
                                                        const TB* __restrict__ b,
                                                        double* __restrict__ partial,
                                                        unsigned* __restrict__ counter,
                                                        double* __restrict__ scal, int mode) {
  __shared__ double sh[33];
  if (blockIdx.y) {          // right-hand side of a blocked solve: its vectors, partials, scalars
    a += (size_t)blockIdx.y * len;
    b += (size_t)blockIdx.y * len;
    partial += (size_t)blockIdx.y * gridDim.x;
    counter += blockIdx.y;
    scal += 8 * blockIdx.y;
  }
  double s = 0.0;
  const int64_t G = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * G < len; i += 4 * G) {      // four independent loads in flight, summed in order
    const double a0 = (double)a[i], a1 = (double)a[i + G], a2 = (double)a[i + 2 * G],
                 a3 = (double)a[i + 3 * G];
    const double b0 = (double)b[i], b1 = (double)b[i + G], b2 = (double)b[i + 2 * G],
                 b3 = (double)b[i + 3 * G];
    s += a0 * b0;
    s += a1 * b1;
    s += a2 * b2;
    s += a3 * b3;
  }
  for (; i < len; i += G) s += (double)a[i] * (double)b[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
  if (!last_block(counter)) return;
  __syncthreads();
  const double tot = sum_partials(partial, gridDim.x, sh);
  if (threadIdx.x == 0) {
    if (mode == 0) {
      scal[1] = tot;
      scal[2] = scal[0] / tot;
    } else if (mode == 1) {
      scal[3] = tot;
      scal[4] = tot / scal[0];
      scal[0] = tot;
    } else {
      scal[5] = tot;
    }
    *counter = 0u;
  }
}

// p = z + beta p and Ap = 0; blockIdx.y: right-hand side of a blocked solve,
// whose p is held at zero once it has converged (scal[7] != 0)
template <typename T, typename TZ = T>
__global__ void cg_direction_zero_kernel(int64_t len, const double* __restrict__ scal,
                                         const TZ* __restrict__ z, T* __restrict__ p,
                                         T* __restrict__ Ap) {
  if (blockIdx.y) {
    const size_t o = (size_t)blockIdx.y * len;
    z += o;
    p += o;
    Ap += o;
    scal += 8 * blockIdx.y;
  }
  const bool done = gridDim.y > 1 && scal[7] != 0.0;
  const T beta = (T)scal[4];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x) {
    p[i] = done ? T(0) : (T)z[i] + beta * p[i];
    Ap[i] = T(0);
  }
}

// Blocked form of cg_update_test_kernel, blockIdx.y = right-hand side j with
// scalars scal[8 j ...] (7: converged), partials partial[j][gridDim.x] and
// counters counter[j]: x += alpha p and r -= alpha A p unless j has converged,
// r.r; the last block of j tests r.r <= tol2 scal[6] (or NaN) and marks j
// converged; the last of those (counter[k]) counts the iteration and stops
// the loop once every right-hand side has converged or after max_it.
template <typename T>
__global__ void __launch_bounds__(256) cg_update_test_block_kernel(
    int64_t len, double* __restrict__ scal, T* __restrict__ x, T* __restrict__ r,
    const T* __restrict__ p, const T* __restrict__ Ap, double* __restrict__ partial,
    unsigned* __restrict__ counter, cudaGraphConditionalHandle h, int* __restrict__ it,
    int max_it, double tol2) {
  __shared__ double sh[33];
  __shared__ bool last_all;
  const int j = blockIdx.y, k = gridDim.y;
  const size_t o = (size_t)j * len;
  double* sc = scal + 8 * j;
  const bool done = sc[7] != 0.0;
  const T alpha = done ? T(0) : (T)sc[2];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x) {
    T ri = r[o + i];
    if (!done) {
      x[o + i] += alpha * p[o + i];
      ri -= alpha * Ap[o + i];
      r[o + i] = ri;
    }
    s += (double)ri * (double)ri;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partial[(size_t)j * gridDim.x + blockIdx.x] = s;
  if (!last_block(counter + j)) return;
  const double rr = sum_partials(partial + (size_t)j * gridDim.x, gridDim.x, sh);
  if (threadIdx.x == 0) {
    sc[5] = rr;
    counter[j] = 0u;
    if (!(rr > tol2 * sc[6])) sc[7] = 1.0;
    __threadfence();
    last_all = atomicAdd(counter + k, 1u) == (unsigned)(k - 1);
    if (last_all) {
      __threadfence();
      bool all = true;
      for (int q = 0; q < k; ++q) all = all && ((volatile double*)scal)[8 * q + 7] != 0.0;
      counter[k] = 0u;
      const int kk = ++(*it);
      if (all || kk >= max_it) {
        if (h)
          cudaGraphSetConditional(h, 0);
        else
          it[1] = 1;
      }
    }
  }
}

// x += alpha p, r -= alpha Ap, scal[5] = r.r, then the loop test of the
// graph: stop when r.r <= tol2 * scal[6], on NaN, or after max_it iterations
// (h == 0: no graph; it[1] = 1 tells the host loop to stop)
template <typename T>
__global__ void __launch_bounds__(256) cg_update_test_kernel(
    int64_t len, double* __restrict__ scal, T* __restrict__ x, T* __restrict__ r,
    const T* __restrict__ p, const T* __restrict__ Ap, double* __restrict__ partial,
    unsigned* __restrict__ counter, cudaGraphConditionalHandle h, int* __restrict__ it,
    int max_it, double tol2, float* __restrict__ r32) {
  __shared__ double sh[33];
  const T alpha = (T)scal[2];
  double s = 0.0;
  const int64_t G = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + G < len; i += 2 * G) {          // two values per pass, loads first
    const T p0 = p[i], p1 = p[i + G], q0 = Ap[i], q1 = Ap[i + G];
    const T x0 = x[i], x1 = x[i + G], s0 = r[i], s1 = r[i + G];
    x[i] = x0 + alpha * p0;
    x[i + G] = x1 + alpha * p1;
    const T r0 = s0 - alpha * q0, r1 = s1 - alpha * q1;
    r[i] = r0;
    r[i + G] = r1;
    if (r32) {
      r32[i] = (float)r0;
      r32[i + G] = (float)r1;
    }
    s += (double)r0 * (double)r0;
    s += (double)r1 * (double)r1;
  }
  for (; i < len; i += G) {
    x[i] += alpha * p[i];
    const T ri = r[i] - alpha * Ap[i];
    r[i] = ri;
    if (r32) r32[i] = (float)ri;
    s += (double)ri * (double)ri;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
  if (!last_block(counter)) return;
  __syncthreads();
  const double rr = sum_partials(partial, gridDim.x, sh);
  if (threadIdx.x == 0) {
    scal[5] = rr;
    *counter = 0u;
    const int k = ++(*it);
    if (!(rr > tol2 * scal[6]) || k >= max_it) {
      if (h)
        cudaGraphSetConditional(h, 0);
      else
        it[1] = 1;                // host-driven loop: the stop flag it reads back
    }
  }
}

// The update that closes the fused PCG iteration (after cg_matvec_kernel):
// p+ = fma(beta, p, z) -- the direction cg_matvec_kernel applied A to --,
// x += alpha p+, r -= alpha Ap, p = p+, Ap = 0 for the next matvec, the FP32
// copy of r (r32, nullable) and r.r with the loop test of
// cg_update_test_kernel.
template <typename TZ>
__global__ void __launch_bounds__(256) cg_update_dir_test_kernel(
    int64_t len, double* __restrict__ scal, double* __restrict__ x, double* __restrict__ r,
    double* __restrict__ p, double* __restrict__ Ap, const TZ* __restrict__ z,
    double* __restrict__ partial, unsigned* __restrict__ counter, cudaGraphConditionalHandle h,
    int* __restrict__ it, int max_it, double tol2, float* __restrict__ r32) {
  __shared__ double sh[33];
  const double alpha = scal[2], beta = scal[4];
  double s = 0.0;
  const int64_t G = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + G < len; i += 2 * G) {          // two values per pass, loads first
    const double z0 = (double)z[i], z1 = (double)z[i + G], p0 = p[i], p1 = p[i + G];
    const double q0 = Ap[i], q1 = Ap[i + G], x0 = x[i], x1 = x[i + G];
    const double s0 = r[i], s1 = r[i + G];
    const double d0 = fma(beta, p0, z0), d1 = fma(beta, p1, z1);
    p[i] = d0;
    p[i + G] = d1;
    Ap[i] = 0.0;
    Ap[i + G] = 0.0;
    x[i] = x0 + alpha * d0;
    x[i + G] = x1 + alpha * d1;
    const double r0 = s0 - alpha * q0, r1 = s1 - alpha * q1;
    r[i] = r0;
    r[i + G] = r1;
    if (r32) {
      r32[i] = (float)r0;
      r32[i + G] = (float)r1;
    }
    s += r0 * r0;
    s += r1 * r1;
  }
  for (; i < len; i += G) {
    const double d = fma(beta, p[i], (double)z[i]);
    p[i] = d;
    x[i] += alpha * d;
    const double ri = r[i] - alpha * Ap[i];
    Ap[i] = 0.0;
    r[i] = ri;
    if (r32) r32[i] = (float)ri;
    s += ri * ri;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
  if (!last_block(counter)) return;
  __syncthreads();
  const double rr = sum_partials(partial, gridDim.x, sh);
  if (threadIdx.x == 0) {
    scal[5] = rr;
    *counter = 0u;
    const int k = ++(*it);
    if (!(rr > tol2 * scal[6]) || k >= max_it) {
      if (h)
        cudaGraphSetConditional(h, 0);
      else
        it[1] = 1;
    }
  }
}

// scal layout: 0 rz, 1 pAp, 2 alpha, 3 rz_new, 4 beta, 5 rr
template <typename T>
__global__ void cg_update_kernel(int64_t len, const double* __restrict__ scal, T* __restrict__ x,
                                 T* __restrict__ r, const T* __restrict__ p,
                                 const T* __restrict__ Ap) {
  const T alpha = (T)scal[2];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    r[i] -= alpha * Ap[i];
  }
}

template <typename T>
__global__ void cg_direction_kernel(int64_t len, const double* __restrict__ scal,
                                    const T* __restrict__ z, T* __restrict__ p) {
  const T beta = (T)scal[4];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}

// out = scale * in (FP64 -> FP32), and y += alpha * x (FP32 -> FP64): the
// hand-over between the FP64 outer and the FP32 inner iteration
// blockIdx.y: right-hand side j of a blocked solve, its scale at
// scale[j * sstride]; a zero scale (a right-hand side already solved)
// gives a zero vector
__global__ void scale_to_f32_kernel(int64_t len, const double* __restrict__ in,
                                    const double* __restrict__ scale, float* __restrict__ out,
                                    int sstride) {
  const size_t o = (size_t)blockIdx.y * len;
  const double v = scale[(size_t)blockIdx.y * sstride];
  const double sc = v > 0.0 ? 1.0 / sqrt(v) : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    out[o + i] = (float)(in[o + i] * sc);
}

__global__ void add_f32_kernel(int64_t len, const double* __restrict__ scale,
                               const float* __restrict__ x, double* __restrict__ y, int sstride) {
  const size_t o = (size_t)blockIdx.y * len;
  const double sc = sqrt(scale[(size_t)blockIdx.y * sstride]);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    y[o + i] += sc * (double)x[o + i];
}

__global__ void axpby_kernel(int64_t len, double a, const double* __restrict__ x, double b,
                             double* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

__global__ void cg_scalars_kernel(double* scal, int stage) {
  if (stage == 0) {            // alpha = rz / pAp
    scal[2] = scal[0] / scal[1];
  } else {                     // beta = rz_new / rz, rz = rz_new
    scal[4] = scal[3] / scal[0];
    scal[0] = scal[3];
  }
}

__global__ void copy_boundary_kernel(int n, int nd, const double* __restrict__ gD,
                                     double* __restrict__ lam) {
  const int nedge = 2 * n * (n + 1);
  const int edge = blockIdx.x * blockDim.x + threadIdx.x;
  if (edge >= nedge) return;
  const bool b = bnd_edge(n, edge);
  for (int k = 0; k < nd; ++k) {
    const size_t ix = (size_t)k * nedge + edge;
    lam[ix] = b ? (gD ? gD[ix] : 0.0) : 0.0;
  }
}

template <typename T>
__global__ void unpack_kernel(int nl, int nE, bool ns, const T* __restrict__ Ap,
                              double* __restrict__ full) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nE) return;
  for (int r = 0; r < nl; ++r)
    for (int c = 0; c < nl; ++c)
      full[(size_t)(r * nl + c) * nE + e] = (double)Ap[(size_t)(ns ? r * nl + c : pk_any(r, c)) * nE + e];
}


}  // namespace

// ---------------------------------------------------------------- launchers
#define ND_DISPATCH(nd, MACRO)  \
  switch (nd) {                 \
    case 2: MACRO(2); break;    \
    case 3: MACRO(3); break;    \
    case 4: MACRO(4); break;    \
    case 5: MACRO(5); break;    \
    case 6: MACRO(6); break;    \
    case 7: MACRO(7); break;    \
    case 8: MACRO(8); break;    \
    case 9: MACRO(9); break;    \
    default: break;             \
  }

template <typename T>
void launch_matvec(cudaStream_t s, int n, int nd, bool ns, const T* A, const T* x, T* y, T alpha,
                   const T* xadd, int k) {
#define MV(ND)                                                           \
  if (ns) launch_matvec_nd<T, ND, true>(s, n, A, x, y, alpha, xadd, k);   \
  else launch_matvec_nd<T, ND, false>(s, n, A, x, y, alpha, xadd, k)
  ND_DISPATCH(nd, MV)
#undef MV
}

void launch_cg_matvec(cudaStream_t s, int n, int nd, const double* A, const float* z32,
                      const double* z64, const double* p, double* Ap, double* scal,
                      double* partial, unsigned* counter) {
#define CGM(ND) launch_cg_matvec_nd<ND>(s, n, A, z32, z64, p, Ap, scal, partial, counter)
  ND_DISPATCH(nd, CGM)
#undef CGM
}

void launch_matvec_mf(cudaStream_t s, int n, int nd, const float* tables, const double* kap,
                      const float* x, float* y, float alpha, const float* xadd, int k) {
  switch (nd) {
#define MFC(ND) \
  case ND: launch_matvec_mf_nd<ND>(s, n, tables, kap, x, y, alpha, xadd, k); break;
    MFC(2) MFC(3) MFC(4) MFC(5) MFC(6) MFC(7)
#undef MFC
    default: break;
  }
}

void launch_bj_update_dot(cudaStream_t s, int n, int nd, const float* Dinv, const float* r,
                          float* y, float* e, float omega, const float* xadd, const double* r64,
                          double* scal, double* partial, unsigned* counter) {
#define BJD(ND) launch_bj_update_dot_nd<ND>(s, n, Dinv, r, y, e, omega, xadd, r64, scal, partial, counter)
  ND_DISPATCH(nd, BJD)
#undef BJD
}

void launch_matvec_bf16(cudaStream_t s, int n, int nd, bool ns, const __nv_bfloat16* A,
                        const float* x, float* y, float alpha, const float* xadd, int k) {
#define MVB(ND)                                                                 \
  if (ns) launch_matvec_bf16_nd<ND, true>(s, n, A, x, y, alpha, xadd, k);       \
  else launch_matvec_bf16_nd<ND, false>(s, n, A, x, y, alpha, xadd, k)
  ND_DISPATCH(nd, MVB)
#undef MVB
}

__global__ void to_bf16_kernel(int64_t len, const double* __restrict__ in,
                               __nv_bfloat16* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = __double2bfloat16(in[i]);
}

void launch_to_bf16(cudaStream_t s, int64_t len, const double* in, __nv_bfloat16* out) {
  int blocks = nblk(len, 256);
  if (blocks > 4 * 152 * 4) blocks = 4 * 152 * 4;
  note_launch();
  to_bf16_kernel<<<blocks, 256, 0, s>>>(len, in, out);
}

template <typename T>
void launch_bj_blocks(cudaStream_t s, int n, int nd, bool ns, const T* A, T* Dinv, int* err) {
#define BJ(ND)                                                \
  if (ns) launch_bj_blocks_nd<T, ND, true>(s, n, A, Dinv, err); \
  else launch_bj_blocks_nd<T, ND, false>(s, n, A, Dinv, err)
  ND_DISPATCH(nd, BJ)
#undef BJ
}

template <typename T>
void launch_bj_update(cudaStream_t s, int n, int nd, bool ns, const T* Dinv, const T* r, T* y,
                      T* e, T omega, int first, const T* xadd, int k) {
#define BU(ND)                                                                           \
  if (ns) launch_bj_update_nd<T, ND, true>(s, n, Dinv, r, y, e, omega, first, xadd, k);  \
  else launch_bj_update_nd<T, ND, false>(s, n, Dinv, r, y, e, omega, first, xadd, k)
  ND_DISPATCH(nd, BU)
#undef BU
}

template <typename T>
void launch_pcoarsen(cudaStream_t s, int nE, int ndf, bool ns, const T* Af, T* Ac) {
  note_launch();
  pcoarsen_kernel<T><<<nblk(nE, 128), 128, 0, s>>>(nE, ndf, ns, Af, Ac);
}

static void upload_jc() {
  // once per device: the constant-memory copy of the child injection
  static std::once_flag flags[64];
  int dev = 0;
  cudaGetDevice(&dev);
  std::call_once(flags[dev & 63], [] {
    double J[2][2][2];
    child_injection(J);
    cudaMemcpyToSymbol(c_Jc, J, sizeof(J));
    float Jf[2][2][2];
    for (int a = 0; a < 8; ++a) (&Jf[0][0][0])[a] = (float)(&J[0][0][0])[a];
    cudaMemcpyToSymbol(c_Jcf, Jf, sizeof(Jf));
  });
}

template <typename T>
void launch_agglomerate(cudaStream_t s, int nc, bool ns, const T* Af, T* Ac, T* AIIinv, T* Y,
                        T* Pi, T* Rt, int* err) {
  upload_jc();
  note_launch();
  if (ns)
    agglomerate_ns_warp_kernel<T, 4><<<nblk(nc * nc, 4), 128, 0, s>>>(nc, Af, Ac, AIIinv, Y, Pi, Rt,
                                                                       err);
  else
    agglomerate_warp_kernel<T, 4><<<nblk(nc * nc, 4), 128, 0, s>>>(nc, Af, Ac, AIIinv, Y, Pi, err);
}

template <typename T>
void launch_local_correction(cudaStream_t s, int nc, bool ns, const T* AIIinv, const T* Y,
                             const T* r, T* e, int k) {
  const P1Geom g = make_p1geom(2 * nc);
  const dim3 grid(nblk(8 * nc * nc, 128), k);
  note_launch();
  if (ns)
    local_correction_kernel<T, true><<<grid, 128, 0, s>>>(g, AIIinv, Y, r, e);
  else
    local_correction_kernel<T, false><<<grid, 128, 0, s>>>(g, AIIinv, Y, r, e);
}

template <typename T>
void launch_edge_p1(cudaStream_t s, int n, bool ns, const T* A, const T* Dinv, const T* r, const T* x,
                    T* out, T omega, bool sweep, int k) {
  const P1Geom g = make_p1geom(n);
  const dim3 nb(nblk(g.nedge, 128), k);
  note_launch();
  if (ns) {
    if (sweep)
      edge_p1_kernel<T, true, true><<<nb, 128, 0, s>>>(g, A, Dinv, r, x, out, omega);
    else
      edge_p1_kernel<T, true, false><<<nb, 128, 0, s>>>(g, A, Dinv, r, x, out, omega);
  } else {
    if (sweep)
      edge_p1_kernel<T, false, true><<<nb, 128, 0, s>>>(g, A, Dinv, r, x, out, omega);
    else
      edge_p1_kernel<T, false, false><<<nb, 128, 0, s>>>(g, A, Dinv, r, x, out, omega);
  }
}

template <typename T>
void launch_point_diag(cudaStream_t s, int n, int nd, bool ns, const T* A, T* Dpt) {
  note_launch();
  point_diag_kernel<T><<<nblk(2 * n * (n + 1), 128), 128, 0, s>>>(n, nd, ns, A, Dpt);
}

template <typename T>
void launch_pj_update(cudaStream_t s, int n, int nd, const T* Dpt, const T* r, T* y, T* e, T omega,
                      int first) {
  note_launch();
  pj_update_kernel<T><<<nblk(2 * n * (n + 1), 128), 128, 0, s>>>(n, nd, Dpt, r, y, e, omega, first);
}

template <typename T>
void launch_cheb_update(cudaStream_t s, int n, int nd, const T* Dpt, const T* r, T* y, T* e, T* d,
                        const double* coef, int k, int first_e, int first_d) {
  note_launch();
  cheb_update_kernel<T><<<nblk(2 * n * (n + 1), 128), 128, 0, s>>>(n, nd, Dpt, r, y, e, d, coef, k,
                                                                   first_e, first_d);
}

template <typename T>
void launch_gs_colour(cudaStream_t s, int n, int nd, bool ns, const T* A, const T* Dpt, const T* r,
                      T* e, int colour, int backward) {
  note_launch();
  gs_colour_kernel<T><<<nblk(2 * n * (n + 1), 128), 128, 0, s>>>(n, nd, ns, A, Dpt, r, e, colour,
                                                                 backward);
}

template <typename T>
void launch_power_start(cudaStream_t s, int n, int nd, T* x) {
  note_launch();
  power_start_kernel<T><<<nblk(2 * n * (n + 1), 128), 128, 0, s>>>(n, nd, x);
}

template <typename T>
void launch_scale_by(cudaStream_t s, int64_t len, const T* Dpt, T* y) {
  int blocks = nblk(len, 256);
  if (blocks > 2432) blocks = 2432;
  note_launch();
  scale_by_kernel<T><<<blocks, 256, 0, s>>>(len, Dpt, y);
}

template <typename T>
void launch_normalize(cudaStream_t s, int64_t len, const T* y, const double* nrm2, T* x) {
  int blocks = nblk(len, 256);
  if (blocks > 2432) blocks = 2432;
  note_launch();
  normalize_kernel<T><<<blocks, 256, 0, s>>>(len, y, nrm2, x);
}

template <typename T>
void launch_restrict_h(cudaStream_t s, int nc, const T* Pi, const T* r, T* y, T* rc, int k) {
  upload_jc();
  const int nedc = 2 * nc * (nc + 1);
  note_launch();
  restrict_h_kernel<T><<<dim3(nblk(2 * nedc, 128), k), 128, 0, s>>>(make_p1geom(2 * nc), Pi, r, y,
                                                                    rc);
}

template <typename T>
void launch_prolong_h(cudaStream_t s, int nc, const T* Pi, const T* ec, T* e, T* y, int k) {
  upload_jc();
  const int tot = 8 * nc * nc + 4 * nc * (nc + 1);
  note_launch();
  prolong_h_kernel<T><<<dim3(nblk(tot, 128), k), 128, 0, s>>>(make_p1geom(2 * nc), Pi, ec, e, y);
}

template <typename T>
void launch_bj_first_restrict_p(cudaStream_t s, int n, int nd0, bool ns, const T* Dinv1,
                                const T* r0, T* y0, T* r1, T* e1, T omega, int k) {
  const P1Geom g = make_p1geom(n);
  const dim3 grid(nblk(g.nedge, 128), k);
  note_launch();
  if (ns)
    bj_first_restrict_p_kernel<T, true><<<grid, 128, 0, s>>>(g, nd0, Dinv1, r0, y0, r1, e1, omega);
  else
    bj_first_restrict_p_kernel<T, false><<<grid, 128, 0, s>>>(g, nd0, Dinv1, r0, y0, r1, e1, omega);
}

template <typename T>
void launch_restrict_p(cudaStream_t s, int n, int nd, const T* r, T* y, T* rc) {
  const int ne = 2 * n * (n + 1);
  note_launch();
  restrict_p_kernel<T><<<nblk(ne, 128), 128, 0, s>>>(n, nd, r, y, rc);
}

template <typename T>
void launch_prolong_p(cudaStream_t s, int n, int nd, const T* ec, T* e) {
  (void)nd;
  const int ne = 2 * n * (n + 1);
  note_launch();
  prolong_p_kernel<T><<<nblk(ne, 128), 128, 0, s>>>(n, ec, e);
}

template <typename T>
void launch_coarse_assemble(cudaStream_t s, int n, bool ns, const T* A, const int* freeidx, int nf,
                            double* dense) {
  cudaMemsetAsync(dense, 0, sizeof(double) * (size_t)nf * nf, s);
  note_launch();
  coarse_assemble_kernel<T><<<nblk(n * n, 64), 64, 0, s>>>(n, ns, A, freeidx, nf, dense);
}

void launch_coarse_gj(cudaStream_t s, int nf, double* M, double* Ainv, int* err) {
  note_launch();
  coarse_gj_kernel<<<1, 1024, sizeof(double) * (size_t)(nf > 0 ? nf : 1), s>>>(nf, M, Ainv, err);
}

void launch_coarse_factor(cudaStream_t s, int nf, double* dense, int* err) {
  note_launch();
  coarse_factor_kernel<<<1, 1024, 0, s>>>(nf, dense, err);
}

template <typename T>
bool launch_coarse_setup_smem(cudaStream_t s, int n, bool ns, const T* A, const int* freeidx,
                              int nf, double* Ainv, int* err) {
  const size_t shm = sizeof(double) * ((size_t)nf * nf + nf);
  if (shm > 200 * 1024) return false;
  static const bool attr = [] {
    cudaFuncSetAttribute(coarse_setup_smem_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    return true;
  }();
  (void)attr;
  note_launch();
  coarse_setup_smem_kernel<T><<<1, 1024, shm, s>>>(n, ns, A, freeidx, nf, Ainv, err);
  return true;
}

void launch_coarse_inverse(cudaStream_t s, int nf, const double* L, double* Li, double* Ainv) {
  note_launch();
  chol_linv_kernel<<<nblk(nf, 64), 64, 0, s>>>(nf, L, Li);
  note_launch();
  chol_gram_kernel<<<nf, 128, 0, s>>>(nf, Li, Ainv);
}

template <typename T>
void launch_coarse_solve(cudaStream_t s, int n, const int* freeidx, const int* fedge, int nf,
                         const double* Ainv, const T* r, T* e, int k) {
  note_launch();
  coarse_solve_kernel<T><<<dim3(1, k), 256, sizeof(double) * (nf + 1), s>>>(n, freeidx, fedge, nf,
                                                                             Ainv, r, e);
}

template <typename T>
void launch_vcycle_tail(cudaStream_t s, const TailParams<T>& P) {
  // FP64 needs twice the registers per value: half the threads
  constexpr int NTHR = sizeof(T) == 8 ? 512 : 1024;
  static const bool attr = [] {
    cudaFuncSetAttribute(vcycle_tail_kernel<T, NTHR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kTailMaxSmem);
    return true;
  }();
  (void)attr;
  note_launch();
  vcycle_tail_kernel<T, NTHR><<<1, NTHR, P.smem_bytes, s>>>(P);
}

// the persistent cycle: 1024 threads per block in FP32 (at most 64 registers
// a thread), 512 in FP64; one block per SM; shared memory for the coarsest
// right-hand side (nf <= kPcMaxNf doubles)
constexpr int kPcMaxNf = 4096;
constexpr int kPcMaxSmem = 200 * 1024;
template <typename T>
constexpr int pc_nthr() {
  return sizeof(T) == 8 ? 512 : 1024;
}

template <typename T>
int pcycle_threads() {
  return pc_nthr<T>();
}

template <typename T>
static void pc_attributes() {
  static std::once_flag flags[64];
  int dev = 0;
  cudaGetDevice(&dev);
  std::call_once(flags[dev & 63], [] {
    cudaFuncSetAttribute(pcycle_kernel<T, false, pc_nthr<T>()>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, kPcMaxSmem);
    cudaFuncSetAttribute(pcycle_kernel<T, true, pc_nthr<T>()>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, kPcMaxSmem);
  });
}

template <typename T>
int pcycle_max_blocks(int smem_bytes) {
  int dev = 0, sms = 0, per_sm = 0, per_sm_ns = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  pc_attributes<T>();
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcycle_kernel<T, false, pc_nthr<T>()>,
                                                    pc_nthr<T>(), smem_bytes) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_ns, pcycle_kernel<T, true, pc_nthr<T>()>,
                                                    pc_nthr<T>(), smem_bytes) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (per_sm < per_sm_ns ? per_sm : per_sm_ns) * sms;
}

template <typename T>
cudaError_t launch_pcycle(cudaStream_t s, const PCycleParams<T>& P, int blocks) {
  if (P.nf > kPcMaxNf || blocks < 1 || P.smem_bytes > kPcMaxSmem) return cudaErrorInvalidValue;
  upload_jc();
  pc_attributes<T>();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks, 1, 1);
  cfg.blockDim = dim3(pc_nthr<T>(), 1, 1);
  cfg.dynamicSmemBytes = (size_t)P.smem_bytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  note_launch();
  if (P.ns) return cudaLaunchKernelEx(&cfg, pcycle_kernel<T, true, pc_nthr<T>()>, P);
  return cudaLaunchKernelEx(&cfg, pcycle_kernel<T, false, pc_nthr<T>()>, P);
}

template <typename T>
void launch_dot(cudaStream_t s, int64_t len, const T* a, const T* b, double* partial,
                double* out) {
  note_launch();
  dot_partial_kernel<T><<<kDotBlocks, 256, 0, s>>>(len, a, b, partial);
  note_launch();
  dot_final_kernel<<<1, 1024, 0, s>>>(kDotBlocks, partial, out);
}

template <typename T>
void launch_mask(cudaStream_t s, int n, int nd, T* x) {
  const int ne = 2 * n * (n + 1);
  note_launch();
  mask_kernel<T><<<nblk(ne, 128), 128, 0, s>>>(n, nd, x);
}

template <typename T>
void launch_unpack(cudaStream_t s, int nl, int nE, bool ns, const T* Ap, double* full) {
  note_launch();
  unpack_kernel<T><<<nblk(nE, 128), 128, 0, s>>>(nl, nE, ns, Ap, full);
}

template <typename A, typename B>
void launch_convert(cudaStream_t s, int64_t len, const A* in, B* out) {
  int blocks = nblk(len, 256);
  if (blocks > 4 * 152 * 4) blocks = 4 * 152 * 4;
  note_launch();
  convert_kernel<A, B><<<blocks, 256, 0, s>>>(len, in, out);
}

template <typename T>
void launch_cg_update(cudaStream_t s, int64_t len, const double* scal, T* x, T* r,
                      const T* p, const T* Ap) {
  int blocks = nblk(len, 256);
  if (blocks > 2432) blocks = 2432;
  note_launch();
  cg_update_kernel<T><<<blocks, 256, 0, s>>>(len, scal, x, r, p, Ap);
}

template <typename T>
void launch_cg_direction(cudaStream_t s, int64_t len, const double* scal, const T* z, T* p) {
  int blocks = nblk(len, 256);
  if (blocks > 2432) blocks = 2432;
  note_launch();
  cg_direction_kernel<T><<<blocks, 256, 0, s>>>(len, scal, z, p);
}

template <typename T>
void launch_dot_fused(cudaStream_t s, int64_t len, const T* a, const T* b, double* partial,
                      unsigned* counter, double* scal, int mode, int k) {
  note_launch();
  dot_fused_kernel<T><<<dim3(kDotBlocks, k), 256, 0, s>>>(len, a, b, partial, counter, scal, mode);
}

template <typename T>
void launch_cg_direction_zero(cudaStream_t s, int64_t len, const double* scal, const T* z, T* p,
                              T* Ap, int k) {
  int blocks = nblk(len, 256);
  if (blocks > 2432) blocks = 2432;
  note_launch();
  cg_direction_zero_kernel<T><<<dim3(blocks, k), 256, 0, s>>>(len, scal, z, p, Ap);
}

template <typename T>
void launch_cg_update_test(cudaStream_t s, int64_t len, double* scal, T* x, T* r, const T* p,
                           const T* Ap, double* partial, unsigned* counter,
                           cudaGraphConditionalHandle h, int* it, int max_it, double tol2,
                           float* r32) {
  note_launch();
  cg_update_test_kernel<T><<<kDotBlocks, 256, 0, s>>>(len, scal, x, r, p, Ap, partial, counter, h,
                                                      it, max_it, tol2, r32);
}

void launch_cg_update_dir_test(cudaStream_t s, int64_t len, double* scal, double* x, double* r,
                               double* p, double* Ap, const float* z32, const double* z64,
                               double* partial, unsigned* counter, cudaGraphConditionalHandle h,
                               int* it, int max_it, double tol2, float* r32) {
  note_launch();
  if (z32)
    cg_update_dir_test_kernel<float><<<kDotBlocks, 256, 0, s>>>(len, scal, x, r, p, Ap, z32, partial,
                                                                counter, h, it, max_it, tol2, r32);
  else
    cg_update_dir_test_kernel<double><<<kDotBlocks, 256, 0, s>>>(len, scal, x, r, p, Ap, z64, partial,
                                                                 counter, h, it, max_it, tol2, r32);
}

void launch_dot_fused_mixed(cudaStream_t s, int64_t len, const double* a, const float* b,
                            double* partial, unsigned* counter, double* scal, int mode) {
  note_launch();
  dot_fused_kernel<double, float><<<kDotBlocks, 256, 0, s>>>(len, a, b, partial, counter, scal, mode);
}

void launch_cg_direction_zero_mixed(cudaStream_t s, int64_t len, const double* scal, const float* z,
                                    double* p, double* Ap) {
  int blocks = nblk(len, 256);
  if (blocks > 2432) blocks = 2432;
  note_launch();
  cg_direction_zero_kernel<double, float><<<blocks, 256, 0, s>>>(len, scal, z, p, Ap);
}

void launch_scale_to_f32(cudaStream_t s, int64_t len, const double* in, const double* scale,
                         float* out, int k, int sstride) {
  int blocks = nblk(len, 256);
  if (blocks > 2432) blocks = 2432;
  note_launch();
  scale_to_f32_kernel<<<dim3(blocks, k), 256, 0, s>>>(len, in, scale, out, sstride);
}

void launch_add_f32(cudaStream_t s, int64_t len, const double* scale, const float* x, double* y,
                    int k, int sstride) {
  int blocks = nblk(len, 256);
  if (blocks > 2432) blocks = 2432;
  note_launch();
  add_f32_kernel<<<dim3(blocks, k), 256, 0, s>>>(len, scale, x, y, sstride);
}

template <typename T>
void launch_cg_update_test_block(cudaStream_t s, int64_t len, int k, double* scal, T* x, T* r,
                                 const T* p, const T* Ap, double* partial, unsigned* counter,
                                 cudaGraphConditionalHandle h, int* it, int max_it, double tol2) {
  note_launch();
  cg_update_test_block_kernel<T><<<dim3(kDotBlocks, k), 256, 0, s>>>(len, scal, x, r, p, Ap, partial,
                                                                     counter, h, it, max_it, tol2);
}
template void launch_cg_update_test_block<float>(cudaStream_t, int64_t, int, double*, float*,
                                                 float*, const float*, const float*, double*,
                                                 unsigned*, cudaGraphConditionalHandle, int*, int,
                                                 double);

void launch_axpby(cudaStream_t s, int64_t len, double a, const double* x, double b, double* y) {
  int blocks = nblk(len, 256);
  if (blocks > 2432) blocks = 2432;
  note_launch();
  axpby_kernel<<<blocks, 256, 0, s>>>(len, a, x, b, y);
}

void launch_cg_scalars(cudaStream_t s, double* scal, int stage) {
  note_launch();
  cg_scalars_kernel<<<1, 1, 0, s>>>(scal, stage);
}

void launch_copy_boundary(cudaStream_t s, int n, int nd, const double* gD, double* lam) {
  const int ne = 2 * n * (n + 1);
  note_launch();
  copy_boundary_kernel<<<nblk(ne, 128), 128, 0, s>>>(n, nd, gD, lam);
}

// explicit instantiations
#define INST(T)                                                                                 \
  template void launch_matvec<T>(cudaStream_t, int, int, bool, const T*, const T*, T*, T,       \
                                 const T*, int);                                                \
  template void launch_bj_blocks<T>(cudaStream_t, int, int, bool, const T*, T*, int*);          \
  template void launch_bj_update<T>(cudaStream_t, int, int, bool, const T*, const T*, T*, T*, T, \
                                    int, const T*, int);                                        \
  template void launch_bj_first_restrict_p<T>(cudaStream_t, int, int, bool, const T*, const T*, \
                                              T*, T*, T*, T, int);                              \
  template void launch_pcoarsen<T>(cudaStream_t, int, int, bool, const T*, T*);                 \
  template void launch_agglomerate<T>(cudaStream_t, int, bool, const T*, T*, T*, T*, T*, T*,    \
                                      int*);                                                    \
  template void launch_local_correction<T>(cudaStream_t, int, bool, const T*, const T*,         \
                                           const T*, T*, int);                                  \
  template void launch_restrict_h<T>(cudaStream_t, int, const T*, const T*, T*, T*, int);       \
  template void launch_point_diag<T>(cudaStream_t, int, int, bool, const T*, T*);               \
  template void launch_pj_update<T>(cudaStream_t, int, int, const T*, const T*, T*, T*, T, int); \
  template void launch_cheb_update<T>(cudaStream_t, int, int, const T*, const T*, T*, T*, T*,   \
                                      const double*, int, int, int);                            \
  template void launch_gs_colour<T>(cudaStream_t, int, int, bool, const T*, const T*, const T*, \
                                    T*, int, int);                                              \
  template void launch_power_start<T>(cudaStream_t, int, int, T*);                              \
  template void launch_scale_by<T>(cudaStream_t, int64_t, const T*, T*);                        \
  template void launch_normalize<T>(cudaStream_t, int64_t, const T*, const double*, T*);        \
  template void launch_edge_p1<T>(cudaStream_t, int, bool, const T*, const T*, const T*,       \
                                  const T*, T*, T, bool, int);                                  \
  template void launch_prolong_h<T>(cudaStream_t, int, const T*, const T*, T*, T*, int);        \
  template void launch_restrict_p<T>(cudaStream_t, int, int, const T*, T*, T*);                 \
  template void launch_prolong_p<T>(cudaStream_t, int, int, const T*, T*);                      \
  template void launch_coarse_assemble<T>(cudaStream_t, int, bool, const T*, const int*, int,   \
                                          double*);                                             \
  template void launch_coarse_solve<T>(cudaStream_t, int, const int*, const int*, int,          \
                                       const double*, const T*, T*, int);                       \
  template void launch_mask<T>(cudaStream_t, int, int, T*);                                     \
  template void launch_unpack<T>(cudaStream_t, int, int, bool, const T*, double*);
INST(double)
INST(float)
#undef INST
template void launch_convert<double, float>(cudaStream_t, int64_t, const double*, float*);
template void launch_vcycle_tail<double>(cudaStream_t, const TailParams<double>&);
template bool launch_coarse_setup_smem<double>(cudaStream_t, int, bool, const double*, const int*,
                                               int, double*, int*);
template bool launch_coarse_setup_smem<float>(cudaStream_t, int, bool, const float*, const int*, int,
                                              double*, int*);
template void launch_dot<double>(cudaStream_t, int64_t, const double*, const double*, double*, double*);
template void launch_dot_fused<double>(cudaStream_t, int64_t, const double*, const double*, double*,
                                       unsigned*, double*, int, int);
template void launch_dot_fused<float>(cudaStream_t, int64_t, const float*, const float*, double*,
                                      unsigned*, double*, int, int);
template void launch_cg_direction_zero<double>(cudaStream_t, int64_t, const double*, const double*,
                                               double*, double*, int);
template void launch_cg_direction_zero<float>(cudaStream_t, int64_t, const double*, const float*,
                                              float*, float*, int);
template void launch_cg_update_test<double>(cudaStream_t, int64_t, double*, double*, double*,
                                            const double*, const double*, double*, unsigned*,
                                            cudaGraphConditionalHandle, int*, int, double, float*);
template void launch_cg_update_test<float>(cudaStream_t, int64_t, double*, float*, float*,
                                           const float*, const float*, double*, unsigned*,
                                           cudaGraphConditionalHandle, int*, int, double, float*);
template void launch_dot<float>(cudaStream_t, int64_t, const float*, const float*, double*, double*);
template void launch_cg_update<double>(cudaStream_t, int64_t, const double*, double*, double*,
                                       const double*, const double*);
template void launch_cg_update<float>(cudaStream_t, int64_t, const double*, float*, float*,
                                      const float*, const float*);
template void launch_cg_direction<double>(cudaStream_t, int64_t, const double*, const double*, double*);
template void launch_cg_direction<float>(cudaStream_t, int64_t, const double*, const float*, float*);
template void launch_vcycle_tail<float>(cudaStream_t, const TailParams<float>&);
template int pcycle_threads<float>();
template int pcycle_threads<double>();
template int pcycle_max_blocks<float>(int);
template int pcycle_max_blocks<double>(int);
template cudaError_t launch_pcycle<float>(cudaStream_t, const PCycleParams<float>&, int);
template cudaError_t launch_pcycle<double>(cudaStream_t, const PCycleParams<double>&, int);
template void launch_convert<float, double>(cudaStream_t, int64_t, const float*, double*);
template void launch_convert<double, double>(cudaStream_t, int64_t, const double*, double*);

}  // namespace hdgmg
