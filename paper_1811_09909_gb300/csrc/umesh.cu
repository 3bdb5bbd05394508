// Unstructured-mesh path: HDG on bilinearly mapped quadrilaterals, the DtN
// multigrid of Sec. 3 on seed-point macro-elements (Sec. 3.1.2), PCG.
//
// Element condensation (Sec. 2).  With the (p+1)^2 Gauss nodes as volume
// nodes and quadrature points, every HDG form on a bilinear element is
// integrated exactly (det J is bilinear and det J grad = cofactor . ref-grad),
// the mass matrix is diagonal (m_a = w_a det J_a), and q is eliminated:
//   D_d[i][a] = (phi_a, d_d phi_i) = w_a (c_d,xi(a) l'_{i1}(xi_{a1}) [i2 == a2]
//                                        + c_d,eta(a) [i1 == a1] l'_{i2}(xi_{a2})),
//   F[i][(j,k)] = <psi_jk, phi_i>_{edge j},  C_d = n_{j,d} F,
//   G = sum_d D_d^T M^-1 D_d,  H = sum_d D_d^T M^-1 C_d,  K = sum_d C_d^T M^-1 C_d,
//   E = <phi_a, phi_b>_dK,  S = kappa G + tau E,  W = kappa H + tau F,
//   A_e = kappa K + tau I - W^T S^-1 W,  g_e = W^T S^-1 M f,
//   u = S^-1 (M f + W lambda),  q_d = kappa M^-1 (D_d u - C_d lambda).
// S is Cholesky-factored per element (its geometry differs per element);
// the factor and Z = S^-1 W stay in memory for the right-hand side and the
// recovery.
//
// Levels are element-based: level vectors hold the macro-edges that carry
// unknowns, and y = A x sums the element products of the two sides of every
// macro-edge.  Mesh levels compute the element products row by row into a
// slot buffer and then sum per edge; macro-element levels pull each
// macro-edge's rows from its two sides in one pass.  h-coarsening per coarse
// macro-element E: assemble its children's operators, Cholesky of A_II,
// Y = -A_II^-1 A_IB, S_B = A_BB + A_BI Y, A_E = J_E^T S_B J_E (eqs. n_1_Ik,
// coarse).  The V-cycle is Algorithm 1 with block-Jacobi smoothing, the
// local correction of eq. localCorrection, Q = [J^T Y^T, J^T] and
// I = [Y J; J]; it runs in FP64 or on FP32 copies of every level (the outer
// PCG, its operator and residual stay FP64).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/hdgmg_umesh.h"
#include "internal.h"
#include "umesh_plan.h"

namespace hdgmg {
namespace {

constexpr int kMaxLoc = 160;        // unknowns of one macro-element's local system
constexpr int kMaxCoarse = 1024;    // unknowns of the coarsest level

struct UTab {
  double xi[9], w[9], Dl[9][9], le[9], re[9], Pk[9][9];
};

inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

// ---------------------------------------------------------------------------
// element geometry
// ---------------------------------------------------------------------------
template <int P>
struct Geo {
  double m[(P + 1) * (P + 1)];
  double cxx[(P + 1) * (P + 1)], cxe[(P + 1) * (P + 1)];
  double cyx[(P + 1) * (P + 1)], cye[(P + 1) * (P + 1)];
  double len[4], nx[4], ny[4];
  int flip[4];
  double vx[4], vy[4];
};

// fills g (shared) for element e; needs a __syncthreads() afterwards
template <int P>
__device__ void element_geometry(const UTab& T, const double* __restrict__ xy,
                                 const int* __restrict__ quads, int e, Geo<P>& g) {
  constexpr int P1 = P + 1, NV = P1 * P1;
  const int tid = threadIdx.x;
  if (tid < 4) {
    const int v = quads[4 * e + tid];
    g.vx[tid] = xy[2 * v];
    g.vy[tid] = xy[2 * v + 1];
  }
  __syncthreads();
  if (tid < 4) {
    const int j = tid, j1 = (tid + 1) & 3;
    const double dx = g.vx[j1] - g.vx[j], dy = g.vy[j1] - g.vy[j];
    const double l = sqrt(dx * dx + dy * dy);
    g.len[j] = l;
    g.nx[j] = dy / l;
    g.ny[j] = -dx / l;
    g.flip[j] = quads[4 * e + j] > quads[4 * e + j1] ? 1 : 0;
  }
  for (int a = tid; a < NV; a += blockDim.x) {
    const int a1 = a % P1, a2 = a / P1;
    const double xi = T.xi[a1], eta = T.xi[a2];
    const double xx = 0.25 * (-(1 - eta) * g.vx[0] + (1 - eta) * g.vx[1] + (1 + eta) * g.vx[2] - (1 + eta) * g.vx[3]);
    const double xe = 0.25 * (-(1 - xi) * g.vx[0] - (1 + xi) * g.vx[1] + (1 + xi) * g.vx[2] + (1 - xi) * g.vx[3]);
    const double yx = 0.25 * (-(1 - eta) * g.vy[0] + (1 - eta) * g.vy[1] + (1 + eta) * g.vy[2] - (1 + eta) * g.vy[3]);
    const double ye = 0.25 * (-(1 - xi) * g.vy[0] - (1 + xi) * g.vy[1] + (1 + xi) * g.vy[2] + (1 - xi) * g.vy[3]);
    g.m[a] = T.w[a1] * T.w[a2] * (xx * ye - xe * yx);
    g.cxx[a] = ye;
    g.cxe[a] = -yx;
    g.cyx[a] = -xe;
    g.cye[a] = xx;
  }
}

// D_d[i][a] = (phi_a, d_d phi_i), exact by collocation at node a
template <int P>
__device__ __forceinline__ double dval(const UTab& T, const Geo<P>& g, int d, int i, int a) {
  constexpr int P1 = P + 1;
  const int i1 = i % P1, i2 = i / P1, a1 = a % P1, a2 = a / P1;
  const double cxi = d == 0 ? g.cxx[a] : g.cyx[a];
  const double ceta = d == 0 ? g.cxe[a] : g.cye[a];
  double r = 0.0;
  if (i2 == a2) r += cxi * T.Dl[i1][a1];
  if (i1 == a1) r += ceta * T.Dl[i2][a2];
  return T.w[a1] * T.w[a2] * r;
}

// F[i][(j,k)] = <psi_jk, phi_i> on edge j (Gauss quadrature on the edge at the
// volume nodes' coordinates: only the node row / column next to the edge
// contributes) = esc w[al] endv Pk[k][al], with the signed trace-basis scale
// esc = 0.5 sqrt(len_j (2k + 1)) (-1 when the edge's direction flips an odd
// mode) formed once per (edge, mode) by the caller
template <int P>
__device__ __forceinline__ double fval_scaled(const UTab& T, double esc, int i, int j, int k) {
  constexpr int P1 = P + 1;
  const int i1 = i % P1, i2 = i / P1;
  int al;
  double endv;
  switch (j) {
    case 0: al = i1; endv = T.le[i2]; break;
    case 1: al = i2; endv = T.re[i1]; break;
    case 2: al = i1; endv = T.re[i2]; break;
    default: al = i2; endv = T.le[i1]; break;
  }
  return esc * T.w[al] * endv * T.Pk[k][al];
}

// E[a][b] = <phi_a, phi_b>_dK
template <int P>
__device__ __forceinline__ double eval_E(const UTab& T, const Geo<P>& g, int a, int b) {
  constexpr int P1 = P + 1;
  const int a1 = a % P1, a2 = a / P1, b1 = b % P1, b2 = b / P1;
  double r = 0.0;
  if (a1 == b1) r += 0.5 * g.len[0] * T.w[a1] * T.le[a2] * T.le[b2]
                   + 0.5 * g.len[2] * T.w[a1] * T.re[a2] * T.re[b2];
  if (a2 == b2) r += 0.5 * g.len[1] * T.w[a2] * T.re[a1] * T.re[b1]
                   + 0.5 * g.len[3] * T.w[a2] * T.le[a1] * T.le[b1];
  return r;
}

// ---------------------------------------------------------------------------
// condensation: one element per block.  The kernel is bound by the FP64 pipe,
// so every FP64 quantity used more than once is formed once: 1/m_i, the
// trace-basis scales, and D_d[i][a] for the 2p+1 nodes i on the row and
// column of a (the only non-zeros), stored by (a, t) with
//   t < p+1:  i = (t, a2)            (the row of a)
//   t >= p+1: i = (a1, t-p-1 skipping a2)   (the column of a).
// ---------------------------------------------------------------------------
template <int P>
__device__ __forceinline__ int line_node(int a, int t) {
  constexpr int P1 = P + 1;
  const int a1 = a % P1, a2 = a / P1;
  if (t < P1) return a2 * P1 + t;
  const int r = t - P1;
  return (r < a2 ? r : r + 1) * P1 + a1;
}

// position of node i in the line list of b, or -1
template <int P>
__device__ __forceinline__ int line_pos(int b, int i) {
  constexpr int P1 = P + 1;
  const int b1 = b % P1, b2 = b / P1, i1 = i % P1, i2 = i / P1;
  if (i2 == b2) return i1;
  if (i1 == b1) return P1 + (i2 < b2 ? i2 : i2 - 1);
  return -1;
}

template <int P>
__global__ void __launch_bounds__(128) u_condense_kernel(
    UTab T, const double* __restrict__ xy, const int* __restrict__ quads,
    const double* __restrict__ logk, double tau, int E, double* __restrict__ Aout,
    double* __restrict__ Lout, double* __restrict__ Zout, double* __restrict__ Mout,
    int* __restrict__ err) {
  constexpr int P1 = P + 1, NV = P1 * P1, NT = 4 * P1, NL = 2 * P1 - 1;
  extern __shared__ double sm[];
  double* S = sm;                 // [NV][NV]
  double* W = S + NV * NV;        // [NV][NT]
  double* F = W + NV * NT;        // [NV][NT], later Z
  double* Am = F + NV * NT;       // [NT][NT]
  double* Dx = Am + NT * NT;      // [NV][NL]  D_x[line_node(a,t)][a]
  double* Dy = Dx + NV * NL;      // [NV][NL]
  __shared__ Geo<P> g;
  __shared__ double invm[NV], escale[4][P1], rdiag[NV];
  __shared__ int bad;
  const int e = blockIdx.x;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  element_geometry<P>(T, xy, quads, e, g);
  __syncthreads();
  const double kap = exp(logk[e]);
  for (int a = tid; a < NV; a += blockDim.x) {
    invm[a] = 1.0 / g.m[a];
    Mout[(size_t)e * NV + a] = g.m[a];
  }
  for (int x = tid; x < 4 * P1; x += blockDim.x) {
    const int j = x / P1, k = x % P1;
    escale[j][k] = 0.5 * sqrt(g.len[j] * (2.0 * k + 1.0));
  }
  for (int x = tid; x < NV * NL; x += blockDim.x) {
    const int a = x / NL, t = x % NL;
    const int i = line_node<P>(a, t);
    Dx[x] = dval<P>(T, g, 0, i, a);
    Dy[x] = dval<P>(T, g, 1, i, a);
  }
  __syncthreads();
  // F[i][(j,k)] = <psi_jk, phi_i>_{edge j}
  for (int x = tid; x < NV * NT; x += blockDim.x) {
    const int i = x / NT, jk = x % NT, j = jk / P1, k = jk % P1;
    const int i1 = i % P1, i2 = i / P1;
    int al, rev;
    double endv;
    switch (j) {
      case 0: al = i1; endv = T.le[i2]; rev = 0; break;
      case 1: al = i2; endv = T.re[i1]; rev = 0; break;
      case 2: al = i1; endv = T.re[i2]; rev = 1; break;
      default: al = i2; endv = T.le[i1]; rev = 1; break;
    }
    const double v = escale[j][k] * T.w[al] * endv * T.Pk[k][al];
    F[x] = (((rev ^ g.flip[j]) & k) & 1) ? -v : v;
  }
  __syncthreads();
  // S = kappa G + tau E,  G[a][b] = sum_i sum_d D_d[i][a] D_d[i][b] / m_i
  // (lower triangle: the Cholesky factorisation reads no other entry)
  for (int x = tid; x < NV * NV; x += blockDim.x) {
    const int a = x / NV, b = x % NV;
    if (b > a) continue;
    double gsum = 0.0;
    for (int t = 0; t < NL; ++t) {
      const int i = line_node<P>(a, t);
      const int tb = line_pos<P>(b, i);
      if (tb < 0) continue;
      const double pr = Dx[a * NL + t] * Dx[b * NL + tb] + Dy[a * NL + t] * Dy[b * NL + tb];
      gsum += pr * invm[i];
    }
    S[x] = kap * gsum + tau * eval_E<P>(T, g, a, b);
  }
  // W = kappa H + tau F,  H[a][(j,k)] = sum_i (D_x n_jx + D_y n_jy)[i][a] F[i][(j,k)] / m_i
  for (int x = tid; x < NV * NT; x += blockDim.x) {
    const int a = x / NT, jk = x % NT, j = jk / P1;
    double h = 0.0;
    for (int t = 0; t < NL; ++t) {
      const int i = line_node<P>(a, t);
      const double dn = (Dx[a * NL + t] * g.nx[j] + Dy[a * NL + t] * g.ny[j]) * invm[i];
      h += dn * F[i * NT + jk];
    }
    W[x] = kap * h + tau * F[x];
  }
  // kappa K + tau I,  K[r][c] = n_r . n_c sum_i F[i][r] F[i][c] / m_i (lower
  // triangle; A_e is symmetric)
  for (int x = tid; x < NT * NT; x += blockDim.x) {
    const int r = x / NT, c = x % NT;
    if (c > r) continue;
    const int jr = r / P1, jc = c / P1;
    const double nn = g.nx[jr] * g.nx[jc] + g.ny[jr] * g.ny[jc];
    double ks = 0.0;
    for (int i = 0; i < NV; ++i) ks += F[i * NT + r] * (F[i * NT + c] * invm[i]);
    Am[x] = kap * nn * ks + (r == c ? tau : 0.0);
  }
  __syncthreads();
  // Cholesky of S (lower, in place); rdiag = 1 / L_kk
  for (int k = 0; k < NV; ++k) {
    if (tid == 0) {
      double d = S[k * NV + k];
      if (!(d > 0.0)) { bad = 1; d = 1.0; }
      const double l = sqrt(d);
      S[k * NV + k] = l;
      rdiag[k] = 1.0 / l;
    }
    __syncthreads();
    const double rp = rdiag[k];
    for (int r = k + 1 + tid; r < NV; r += blockDim.x) S[r * NV + k] *= rp;
    __syncthreads();
    const int m = NV - k - 1;
    for (int x = tid; x < m * m; x += blockDim.x) {
      const int r = k + 1 + x / m, c = k + 1 + x % m;
      if (c <= r) S[r * NV + c] -= S[r * NV + k] * S[c * NV + k];
    }
    __syncthreads();
  }
  // Z = S^-1 W, one column per thread (into F)
  for (int c = tid; c < NT; c += blockDim.x) {
    for (int r = 0; r < NV; ++r) {
      double v = W[r * NT + c];
      for (int q = 0; q < r; ++q) v -= S[r * NV + q] * F[q * NT + c];
      F[r * NT + c] = v * rdiag[r];
    }
    for (int r = NV - 1; r >= 0; --r) {
      double v = F[r * NT + c];
      for (int q = r + 1; q < NV; ++q) v -= S[q * NV + r] * F[q * NT + c];
      F[r * NT + c] = v * rdiag[r];
    }
  }
  __syncthreads();
  // A_e = kappa K + tau I - W^T Z, symmetric: the lower triangle, mirrored
  double* Ag = Aout + (size_t)e * NT * NT;
  for (int x = tid; x < NT * NT; x += blockDim.x) {
    const int r = x / NT, c = x % NT;
    if (c > r) continue;
    double s = 0.0;
    for (int a = 0; a < NV; ++a) s += W[a * NT + r] * F[a * NT + c];
    const double v = Am[x] - s;
    Ag[x] = v;
    Ag[c * NT + r] = v;
  }
  double* Lg = Lout + (size_t)e * NV * NV;
  for (int x = tid; x < NV * NV; x += blockDim.x) Lg[x] = S[x];
  double* Zg = Zout + (size_t)e * NV * NT;
  for (int x = tid; x < NV * NT; x += blockDim.x) Zg[x] = F[x];
  if (tid == 0 && bad) atomicExch(err, 1);
}

// g_e = Z^T M f_e into the element slot buffer t [E][NT]
template <int P>
__global__ void u_rhs_kernel(int E, const double* __restrict__ Z, const double* __restrict__ M,
                             const double* __restrict__ f, double* __restrict__ t) {
  constexpr int P1 = P + 1, NV = P1 * P1, NT = 4 * P1;
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= (long long)E * NT) return;
  const int e = (int)(x / NT), c = (int)(x % NT);
  const double* Ze = Z + (size_t)e * NV * NT;
  double s = 0.0;
  for (int a = 0; a < NV; ++a) s += Ze[a * NT + c] * M[(size_t)e * NV + a] * f[(size_t)e * NV + a];
  t[x] = s;
}

// recovery of u and q per element (one block per element; the two
// triangular solves of S^-1 on warp 0, column by column with the reciprocal
// pivots, the rest over the block; at most 64 registers so that 8 blocks
// share an SM)
template <int P>
__global__ void __launch_bounds__(128, 8) u_recover_kernel(
    UTab T, const double* __restrict__ xy, const int* __restrict__ quads,
    const double* __restrict__ logk, const int* __restrict__ el_slot,
    const double* __restrict__ L, const double* __restrict__ Z, const double* __restrict__ f,
    const double* __restrict__ lam, double* __restrict__ u, double* __restrict__ q) {
  constexpr int P1 = P + 1, NV = P1 * P1, NT = 4 * P1;
  __shared__ Geo<P> g;
  __shared__ double le_[NT], y[NV], uu[NV], es[NT], rdg[NV];
  const int e = blockIdx.x, tid = threadIdx.x;
  element_geometry<P>(T, xy, quads, e, g);
  for (int c = tid; c < NT; c += blockDim.x) {
    const int b = el_slot[4 * e + c / P1];
    le_[c] = b < 0 ? 0.0 : lam[(size_t)b * P1 + c % P1];
  }
  __syncthreads();
  // the signed trace-basis scales of fval_scaled, one FP64 sqrt per (edge,
  // mode) instead of one per use (the flux term below uses each NV times)
  for (int c = tid; c < NT; c += blockDim.x) {
    const int j = c / P1, k = c % P1, rev = j >= 2 ? 1 : 0;
    const double sg = (((rev ^ g.flip[j]) & k) & 1) ? -1.0 : 1.0;
    es[c] = 0.5 * sqrt(g.len[j] * (2.0 * k + 1.0)) * sg;
  }
  const double* Le = L + (size_t)e * NV * NV;
  for (int a = tid; a < NV; a += blockDim.x) {
    y[a] = g.m[a] * f[(size_t)e * NV + a];
    rdg[a] = 1.0 / Le[a * NV + a];
  }
  __syncthreads();
  if (tid < 32) {                         // S^-1 (M f) = L^-T L^-1 (M f), column by column on warp 0
    for (int k = 0; k < NV; ++k) {        // forward: y_k /= L_kk, then y_i -= L_ik y_k below
      if (tid == 0) y[k] *= rdg[k];
      __syncwarp();
      const double yk = y[k];
      for (int i = k + 1 + tid; i < NV; i += 32) y[i] -= Le[i * NV + k] * yk;
      __syncwarp();
    }
    for (int k = NV - 1; k >= 0; --k) {   // backward with L^T: y_k /= L_kk, then y_i -= L_ki y_k above
      if (tid == 0) y[k] *= rdg[k];
      __syncwarp();
      const double yk = y[k];
      for (int i = tid; i < k; i += 32) y[i] -= Le[k * NV + i] * yk;
      __syncwarp();
    }
  }
  __syncthreads();
  const double* Ze = Z + (size_t)e * NV * NT;
  for (int a = tid; a < NV; a += blockDim.x) {
    double v = y[a];
    for (int c = 0; c < NT; ++c) v += Ze[a * NT + c] * le_[c];
    uu[a] = v;
    if (u) u[(size_t)e * NV + a] = v;
  }
  __syncthreads();
  if (!q) return;
  const double kap = exp(logk[e]);
  for (int x = tid; x < 2 * NV; x += blockDim.x) {
    const int d = x / NV, a = x % NV;
    const int a1 = a % P1, a2 = a / P1;
    double s = 0.0;
    for (int t = 0; t < 2 * P1 - 1; ++t) {     // (D_d u)[a] = sum_b D_d[a][b] u_b
      const int b = t < P1 ? a2 * P1 + t : (t - P1 < a2 ? t - P1 : t - P1 + 1) * P1 + a1;
      s += dval<P>(T, g, d, a, b) * uu[b];
    }
    for (int c = 0; c < NT; ++c) {
      const int j = c / P1;
      s -= (d == 0 ? g.nx[j] : g.ny[j]) * fval_scaled<P>(T, es[c], a, j, c % P1) * le_[c];
    }
    q[(size_t)e * 2 * NV + x] = kap * s / g.m[a];
  }
}

// ---------------------------------------------------------------------------
// level operators
// ---------------------------------------------------------------------------
// t[e][i] = sum_j A_e[j][i] x(slot j) on a mesh level (4 edges of ND modes per
// element), one thread per row, fully unrolled so that every load of a thread
// is in flight at once (consecutive threads read consecutive entries)
template <typename T, int ND>
__global__ void __launch_bounds__(128) u_elem_matvec_mesh_kernel(int n_el, const int* __restrict__ el_slot,
                                                                 const T* __restrict__ A,
                                                                 const T* __restrict__ x,
                                                                 T* __restrict__ t) {
  constexpr int NDM = 4 * ND;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)n_el * NDM) return;
  const int e = (int)(id / NDM), i = (int)(id % NDM);
  const T* Ae = A + (size_t)e * NDM * NDM + i;
  int b[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) b[s] = __ldg(el_slot + 4 * e + s);
  T xv[NDM];
#pragma unroll
  for (int j = 0; j < NDM; ++j) xv[j] = b[j / ND] >= 0 ? __ldg(x + (size_t)b[j / ND] * ND + j % ND) : T(0);
  T s0 = 0, s1 = 0;
#pragma unroll
  for (int j = 0; j < NDM; j += 2) {
    s0 += __ldg(Ae + (size_t)j * NDM) * xv[j];
    if (j + 1 < NDM) s1 += __ldg(Ae + (size_t)(j + 1) * NDM) * xv[j + 1];
  }
  t[id] = s0 + s1;
}

// mesh levels, second half: per edge block y = t(side 0) + t(side 1); SUM:
// out = y; RES: out = r - y; SMOOTH: out = x + omega Dinv (r - y)
template <typename T>
__global__ void u_edge_kernel(int n_blk, int nd, const int* __restrict__ t0, const int* __restrict__ t1,
                              const T* __restrict__ t, const T* __restrict__ x,
                              const T* __restrict__ r, const T* __restrict__ Dinv, double omega,
                              int mode, T* __restrict__ out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_blk) return;
  T y[9];
  const size_t o0 = (size_t)t0[b] * nd, o1 = (size_t)t1[b] * nd;
  for (int k = 0; k < nd; ++k) y[k] = t[o0 + k] + t[o1 + k];
  if (mode == 0) {
    for (int k = 0; k < nd; ++k) out[(size_t)b * nd + k] = y[k];
  } else if (mode == 1) {
    for (int k = 0; k < nd; ++k) out[(size_t)b * nd + k] = r[(size_t)b * nd + k] - y[k];
  } else {
    for (int k = 0; k < nd; ++k) y[k] = r[(size_t)b * nd + k] - y[k];
    const T* D = Dinv + (size_t)b * nd * nd;
    for (int k = 0; k < nd; ++k) {
      T s = 0;
      for (int l = 0; l < nd; ++l) s += D[k * nd + l] * y[l];
      out[(size_t)b * nd + k] = x[(size_t)b * nd + k] + (T)omega * s;
    }
  }
}

enum { U_SUM = 0, U_RES = 1, U_SMOOTH = 2 };

// The same with one thread per row (thread (b, k) walks b's two sides'
// padded columns in order, y = side 0 + side 1): the FP64 levels' form.  The
// warp form below halves the FP32 cycle's pull time but doubles the FP64
// one's (10.5 against 21.9 us per launch at 97k quadrilaterals, p = 3).
template <typename T>
__global__ void __launch_bounds__(128) u_pull_row_kernel(int n_blk, int nu, const int* __restrict__ el_slot,
                                                         const int* __restrict__ t0, const int* __restrict__ t1,
                                                         const T* __restrict__ A, const T* __restrict__ x,
                                                         const T* __restrict__ r, const T* __restrict__ Dinv,
                                                         double omega, int mode, T* __restrict__ out) {
  constexpr int ND = 2, UPB = 128 / ND;
  __shared__ T ys[UPB * ND];
  const int ndm = nu * ND;
  const int lu = threadIdx.x / ND, k = threadIdx.x % ND;
  const int b = blockIdx.x * UPB + lu;
  const bool act = b < n_blk;
  T y = 0;
  if (act) {
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int ts = side == 0 ? __ldg(t0 + b) : __ldg(t1 + b);
      const int el = ts / nu, sl = ts % nu;
      const T* Ae = A + (size_t)el * ndm * ndm + sl * ND + k;
      const int* sls = el_slot + (size_t)el * nu;
      T s = 0;
      for (int j = 0; j < ndm; ++j) {
        const int bj = __ldg(sls + j / ND);
        if (bj >= 0) s += __ldg(Ae + (size_t)j * ndm) * __ldg(x + (size_t)bj * ND + j % ND);
      }
      y += s;
    }
  }
  if (mode == U_SUM) {
    if (act) out[(size_t)b * ND + k] = y;
    return;
  }
  if (mode == U_RES) {
    if (act) out[(size_t)b * ND + k] = r[(size_t)b * ND + k] - y;
    return;
  }
  ys[lu * ND + k] = act ? r[(size_t)b * ND + k] - y : T(0);
  __syncthreads();
  if (act) {
    const T* D = Dinv + (size_t)b * ND * ND + k * ND;
    T s = 0;
#pragma unroll
    for (int l = 0; l < ND; ++l) s += D[l] * ys[lu * ND + l];
    out[(size_t)b * ND + k] = x[(size_t)b * ND + k] + (T)omega * s;
  }
}

// y = A x for one macro-element level in one pass, pulled per macro-edge
// (two modes per edge): one warp per unknown block b.  The lanes split the
// columns of b's two sides (side s, column j of its macro-element's padded
// matrix; A_e symmetric, stored column by column, so b's two rows are
// adjacent in every column) and each sums its columns' products for both rows
// in column order; a butterfly over the warp gives y_b (a fixed order).  Then
// SUM: out = y; RES: out = r - y; SMOOTH: out = x + omega Dinv (r - y) on the
// block.  out never aliases x: a smoothing step reads every neighbour's old
// value.  (One thread per row walked the padded columns serially: 10-18
// units per macro-element at the deep levels against ~5.5 on average.)
template <typename T>
__global__ void __launch_bounds__(128) u_pull_kernel(int n_blk, int nu, const int* __restrict__ el_slot,
                                                     const int* __restrict__ t0, const int* __restrict__ t1,
                                                     const T* __restrict__ A, const T* __restrict__ x,
                                                     const T* __restrict__ r, const T* __restrict__ Dinv,
                                                     double omega, int mode, T* __restrict__ out) {
  constexpr int ND = 2;
  const int b = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= n_blk) return;                   // whole warps
  const int ndm = nu * ND;
  const int ts0 = __ldg(t0 + b), ts1 = __ldg(t1 + b);
  T y0 = 0, y1 = 0;
  for (int q = lane; q < 2 * ndm; q += 32) {
    const int side = q >= ndm ? 1 : 0, j = q - side * ndm;
    const int ts = side ? ts1 : ts0;
    const int el = ts / nu, sl = ts - el * nu;
    const int bj = __ldg(el_slot + (size_t)el * nu + j / ND);
    if (bj >= 0) {
      const T xv = __ldg(x + (size_t)bj * ND + j % ND);
      const T* col = A + ((size_t)el * ndm + j) * ndm + sl * ND;
      y0 += __ldg(col) * xv;
      y1 += __ldg(col + 1) * xv;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    y0 += __shfl_xor_sync(0xffffffffu, y0, o);
    y1 += __shfl_xor_sync(0xffffffffu, y1, o);
  }
  if (lane >= ND) return;
  const int k = lane;
  const size_t o = (size_t)b * ND;
  if (mode == U_SUM) {
    out[o + k] = k == 0 ? y0 : y1;
    return;
  }
  const T r0 = r[o] - y0, r1 = r[o + 1] - y1;
  if (mode == U_RES) {
    out[o + k] = k == 0 ? r0 : r1;
    return;
  }
  const T* D = Dinv + o * ND + k * ND;
  out[o + k] = x[o + k] + (T)omega * (D[0] * r0 + D[1] * r1);
}

// per unknown block: out = t(side 0) + t(side 1) (the element-slot sums of
// the right-hand side and of the restriction)
template <typename T>
__global__ void u_unit_kernel(int n_blk, int nd, const int* __restrict__ t0, const int* __restrict__ t1,
                              const T* __restrict__ t, T* __restrict__ out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_blk) return;
  const size_t o0 = (size_t)t0[b] * nd, o1 = (size_t)t1[b] * nd;
  for (int k = 0; k < nd; ++k) out[(size_t)b * nd + k] = t[o0 + k] + t[o1 + k];
}

// e = omega Dinv r (first smoothing step from zero)
template <typename T>
__global__ void u_bj_first_kernel(int n_blk, int nd, const T* __restrict__ Dinv,
                                  const T* __restrict__ r, double omega, T* __restrict__ e) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_blk) return;
  const T* D = Dinv + (size_t)b * nd * nd;
  for (int k = 0; k < nd; ++k) {
    T s = 0;
    for (int l = 0; l < nd; ++l) s += D[k * nd + l] * r[(size_t)b * nd + l];
    e[(size_t)b * nd + k] = (T)omega * s;
  }
}

// block-Jacobi blocks: D = sum of the two sides' diagonal blocks, inverted by
// Gauss-Jordan elimination (SPD: no pivoting needed)
__global__ void u_bjinv_kernel(int n_blk, int nu, int nd, const int* __restrict__ t0,
                               const int* __restrict__ t1, const double* __restrict__ A,
                               double* __restrict__ Dinv, int* __restrict__ err) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_blk) return;
  const int ndm = nu * nd;
  double D[81], X[81];
  const int s[2] = {t0[b], t1[b]};
  for (int k = 0; k < nd * nd; ++k) { D[k] = 0.0; X[k] = 0.0; }
  for (int side = 0; side < 2; ++side) {
    const int el = s[side] / nu, sl = s[side] % nu;
    const double* Ae = A + (size_t)el * ndm * ndm;
    for (int k = 0; k < nd; ++k)
      for (int l = 0; l < nd; ++l) D[k * nd + l] += Ae[(size_t)(sl * nd + l) * ndm + sl * nd + k];
  }
  for (int k = 0; k < nd; ++k) X[k * nd + k] = 1.0;
  for (int c = 0; c < nd; ++c) {
    const double piv = D[c * nd + c];
    if (!(piv > 0.0)) { atomicExch(err, 1); return; }
    const double ip = 1.0 / piv;
    for (int l = 0; l < nd; ++l) { D[c * nd + l] *= ip; X[c * nd + l] *= ip; }
    for (int r = 0; r < nd; ++r) {
      if (r == c) continue;
      const double f = D[r * nd + c];
      for (int l = 0; l < nd; ++l) { D[r * nd + l] -= f * D[c * nd + l]; X[r * nd + l] -= f * X[c * nd + l]; }
    }
  }
  for (int k = 0; k < nd * nd; ++k) Dinv[(size_t)b * nd * nd + k] = X[k];
}

// p-coarsening (eq. ANm1): modes 0, 1 of every edge
__global__ void u_pcoarsen_kernel(int E, int P1, const double* __restrict__ A, double* __restrict__ A1) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)E * 64) return;
  const int e = (int)(id / 64), r = (int)(id % 64) / 8, c = (int)(id % 8);
  const int NT = 4 * P1;
  const int rf = (r / 2) * P1 + r % 2, cf = (c / 2) * P1 + c % 2;
  A1[id] = A[(size_t)e * NT * NT + (size_t)rf * NT + cf];
}

template <typename T>
__global__ void u_prestrict_kernel(int n_blk, int P1, const T* __restrict__ res, T* __restrict__ r1) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= 2 * n_blk) return;
  r1[id] = res[(size_t)(id / 2) * P1 + id % 2];
}

template <typename T>
__global__ void u_pprolong_kernel(int n_blk, int P1, const T* __restrict__ e1, T* __restrict__ e) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= 2 * n_blk) return;
  e[(size_t)(id / 2) * P1 + id % 2] += e1[id];
}

// ---------------------------------------------------------------------------
// h-coarsening (one block per coarse macro-element)
// ---------------------------------------------------------------------------
template <typename T>
struct UHArgs {
  int n_E, nu_f, nd_f, nu_c;
  const int *loc_ptr, *loc_blk, *nI, *own, *ch_ptr, *ch_el, *ch_map, *bs_ptr;
  const long long *J_off, *AI_off, *Y_off;
  const T* J;
  T *AIinv, *Y;
};

__global__ void __launch_bounds__(256) u_agglomerate_kernel(UHArgs<double> h, const double* __restrict__ Af,
                                                            double* __restrict__ Ac, int* __restrict__ err) {
  extern __shared__ double A[];                     // [n][n], n = 2 nloc
  const int E = blockIdx.x, tid = threadIdx.x;
  const int l0 = h.loc_ptr[E], nloc = h.loc_ptr[E + 1] - l0;
  const int n = 2 * nloc, nI2 = 2 * h.nI[E], nB2 = n - nI2;
  const int ndm_f = h.nu_f * 2, ndm_c = h.nu_c * 2;
  __shared__ int bad;
  if (tid == 0) bad = 0;
  for (int x = tid; x < n * n; x += blockDim.x) A[x] = 0.0;
  __syncthreads();
  for (int c = h.ch_ptr[E]; c < h.ch_ptr[E + 1]; ++c) {
    const int f = h.ch_el[c];
    const int* map = h.ch_map + (size_t)c * h.nu_f;
    const double* Ae = Af + (size_t)f * ndm_f * ndm_f;
    for (int x = tid; x < ndm_f * ndm_f; x += blockDim.x) {
      const int i = x / ndm_f, j = x % ndm_f;
      const int li = map[i / 2], lj = map[j / 2];
      if (li < 0 || lj < 0) continue;
      A[(2 * li + i % 2) * n + 2 * lj + j % 2] += Ae[x];
    }
    __syncthreads();
  }
  // Cholesky of A_II (lower, in place)
  for (int k = 0; k < nI2; ++k) {
    if (tid == 0) {
      double d = A[k * n + k];
      if (!(d > 0.0)) { bad = 1; d = 1.0; }
      A[k * n + k] = sqrt(d);
    }
    __syncthreads();
    const double piv = A[k * n + k];
    for (int r = k + 1 + tid; r < nI2; r += blockDim.x) A[r * n + k] /= piv;
    __syncthreads();
    const int m = nI2 - k - 1;
    for (int x = tid; x < m * m; x += blockDim.x) {
      const int r = k + 1 + x / m, c = k + 1 + x % m;
      if (c <= r) A[r * n + c] -= A[r * n + k] * A[c * n + k];
    }
    __syncthreads();
  }
  // Y = -A_II^-1 A_IB in place of the IB block, one column per thread
  for (int c = nI2 + tid; c < n; c += blockDim.x) {
    for (int r = 0; r < nI2; ++r) {
      double v = A[r * n + c];
      for (int q = 0; q < r; ++q) v -= A[r * n + q] * A[q * n + c];
      A[r * n + c] = v / A[r * n + r];
    }
    for (int r = nI2 - 1; r >= 0; --r) {
      double v = A[r * n + c];
      for (int q = r + 1; q < nI2; ++q) v -= A[q * n + r] * A[q * n + c];
      A[r * n + c] = v / A[r * n + r];
    }
    for (int r = 0; r < nI2; ++r) A[r * n + c] = -A[r * n + c];
  }
  // A_II^-1 (column-major = row-major, symmetric), one column per thread, in global memory
  double* AI = h.AIinv + h.AI_off[E];
  for (int c = tid; c < nI2; c += blockDim.x) {
    for (int r = 0; r < nI2; ++r) {
      double v = r == c ? 1.0 : 0.0;
      for (int q = 0; q < r; ++q) v -= A[r * n + q] * AI[(size_t)c * nI2 + q];
      AI[(size_t)c * nI2 + r] = v / A[r * n + r];
    }
    for (int r = nI2 - 1; r >= 0; --r) {
      double v = AI[(size_t)c * nI2 + r];
      for (int q = r + 1; q < nI2; ++q) v -= A[q * n + r] * AI[(size_t)c * nI2 + q];
      AI[(size_t)c * nI2 + r] = v / A[r * n + r];
    }
  }
  __syncthreads();
  double* Yg = h.Y + h.Y_off[E];                     // [nI2][nB2]
  for (int x = tid; x < nI2 * nB2; x += blockDim.x) {
    const int r = x / nB2, c = x % nB2;
    Yg[x] = A[r * n + nI2 + c];
  }
  // S_B = A_BB + A_BI Y in place of the BB block
  for (int x = tid; x < nB2 * nB2; x += blockDim.x) {
    const int r = nI2 + x / nB2, c = nI2 + x % nB2;
    double s = A[r * n + c];
    for (int q = 0; q < nI2; ++q) s += A[r * n + q] * A[q * n + c];
    A[r * n + c] = s;
  }
  __syncthreads();
  // A_E = J_E^T S_B J_E (J_E block-sparse: the B rows of slot s are
  // bs_ptr[s] .. bs_ptr[s+1])
  const double* J = h.J + h.J_off[E];
  const int* bs = h.bs_ptr + (size_t)E * (h.nu_c + 1);
  int nc = 0;
  while (nc < h.nu_c && bs[nc + 1] > bs[nc]) ++nc;
  const int nc2 = 2 * nc;
  double* Ace = Ac + (size_t)E * ndm_c * ndm_c;
  for (int x = tid; x < ndm_c * ndm_c; x += blockDim.x) {
    const int r = x / ndm_c, c = x % ndm_c;
    double s = 0.0;
    if (r < nc2 && c < nc2) {
      const int sr = r / 2, sc = c / 2;
      for (int b = 2 * bs[sr]; b < 2 * bs[sr + 1]; ++b) {
        const double jr = J[(size_t)b * nc2 + r];
        double t = 0.0;
        for (int b2 = 2 * bs[sc]; b2 < 2 * bs[sc + 1]; ++b2)
          t += A[(nI2 + b) * n + nI2 + b2] * J[(size_t)b2 * nc2 + c];
        s += jr * t;
      }
    }
    Ace[x] = s;
  }
  if (tid == 0 && bad) atomicExch(err, 1);
}

// e_I += A_II^-1 res_I (local correction, eq. localCorrection)
template <typename T>
__global__ void u_localcorr_kernel(UHArgs<T> h, const T* __restrict__ res, T* __restrict__ e) {
  __shared__ T rI[kMaxLoc];
  const int E = blockIdx.x, tid = threadIdx.x;
  const int l0 = h.loc_ptr[E], nI2 = 2 * h.nI[E];
  for (int i = tid; i < nI2; i += blockDim.x) rI[i] = res[(size_t)h.loc_blk[l0 + i / 2] * 2 + i % 2];
  __syncthreads();
  const T* AI = h.AIinv + h.AI_off[E];
  for (int i = tid; i < nI2; i += blockDim.x) {
    T s = 0;
    for (int j = 0; j < nI2; ++j) s += AI[(size_t)j * nI2 + i] * rI[j];
    e[(size_t)h.loc_blk[l0 + i / 2] * 2 + i % 2] += s;
  }
}

// tc[E][c] = (J_E^T (Y^T res_I + own res_B))_c: E's share of Q_{k-1} res
template <typename T>
__global__ void u_restrict_kernel(UHArgs<T> h, const T* __restrict__ res, T* __restrict__ tc) {
  __shared__ T rI[kMaxLoc], vB[kMaxLoc];
  const int E = blockIdx.x, tid = threadIdx.x;
  const int l0 = h.loc_ptr[E], nloc = h.loc_ptr[E + 1] - l0;
  const int nI2 = 2 * h.nI[E], nB2 = 2 * nloc - nI2;
  for (int i = tid; i < nI2; i += blockDim.x) rI[i] = res[(size_t)h.loc_blk[l0 + i / 2] * 2 + i % 2];
  __syncthreads();
  const T* Y = h.Y + h.Y_off[E];
  for (int b = tid; b < nB2; b += blockDim.x) {
    const int lb = h.nI[E] + b / 2;
    T s = h.own[l0 + lb] ? res[(size_t)h.loc_blk[l0 + lb] * 2 + b % 2] : T(0);
    for (int i = 0; i < nI2; ++i) s += Y[(size_t)i * nB2 + b] * rI[i];
    vB[b] = s;
  }
  __syncthreads();
  const int* bs = h.bs_ptr + (size_t)E * (h.nu_c + 1);
  int nc = 0;
  while (nc < h.nu_c && bs[nc + 1] > bs[nc]) ++nc;
  const int nc2 = 2 * nc, ndm_c = 2 * h.nu_c;
  const T* J = h.J + h.J_off[E];
  for (int c = tid; c < ndm_c; c += blockDim.x) {
    T s = 0;
    if (c < nc2)
      for (int b = 2 * bs[c / 2]; b < 2 * bs[c / 2 + 1]; ++b) s += J[(size_t)b * nc2 + c] * vB[b];
    tc[(size_t)E * ndm_c + c] = s;
  }
}

// w = J_E e_c;  e_I += Y w;  e_B += w on the blocks E owns (eq. n_1_Ik)
template <typename T>
__global__ void u_prolong_kernel(UHArgs<T> h, const int* __restrict__ el_slot_c, const T* __restrict__ ec,
                                 T* __restrict__ e) {
  __shared__ T ecl[2 * 64], w[kMaxLoc];
  const int E = blockIdx.x, tid = threadIdx.x;
  const int l0 = h.loc_ptr[E], nloc = h.loc_ptr[E + 1] - l0;
  const int nI2 = 2 * h.nI[E], nB2 = 2 * nloc - nI2;
  const int* bs = h.bs_ptr + (size_t)E * (h.nu_c + 1);
  int nc = 0;
  while (nc < h.nu_c && bs[nc + 1] > bs[nc]) ++nc;
  const int nc2 = 2 * nc;
  for (int c = tid; c < nc2; c += blockDim.x)
    ecl[c] = ec[(size_t)el_slot_c[(size_t)E * h.nu_c + c / 2] * 2 + c % 2];
  __syncthreads();
  const T* J = h.J + h.J_off[E];
  for (int b = tid; b < nB2; b += blockDim.x) {
    int s = 0;
    while (b >= 2 * bs[s + 1]) ++s;
    T v = 0;
    for (int c = 2 * s; c < 2 * s + 2; ++c) v += J[(size_t)b * nc2 + c] * ecl[c];
    w[b] = v;
    const int lb = h.nI[E] + b / 2;
    if (h.own[l0 + lb]) e[(size_t)h.loc_blk[l0 + lb] * 2 + b % 2] += v;
  }
  __syncthreads();
  const T* Y = h.Y + h.Y_off[E];
  for (int i = tid; i < nI2; i += blockDim.x) {
    T s = 0;
    for (int b = 0; b < nB2; ++b) s += Y[(size_t)i * nB2 + b] * w[b];
    e[(size_t)h.loc_blk[l0 + i / 2] * 2 + i % 2] += s;
  }
}

// ---------------------------------------------------------------------------
// coarsest level: dense assembly, Cholesky, explicit inverse (one block)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) u_coarse_setup_kernel(int n, int n_el, int nu, const int* __restrict__ el_slot,
                                                              const double* __restrict__ A, double* __restrict__ D,
                                                              double* __restrict__ Dinv, int* __restrict__ err) {
  const int tid = threadIdx.x, ndm = 2 * nu;
  __shared__ int bad;
  if (tid == 0) bad = 0;
  for (int x = tid; x < n * n; x += blockDim.x) D[x] = 0.0;
  __syncthreads();
  for (int e = 0; e < n_el; ++e) {
    for (int x = tid; x < ndm * ndm; x += blockDim.x) {
      const int i = x / ndm, j = x % ndm;
      const int bi = el_slot[(size_t)e * nu + i / 2], bj = el_slot[(size_t)e * nu + j / 2];
      if (bi < 0 || bj < 0) continue;
      D[(size_t)(2 * bi + i % 2) * n + 2 * bj + j % 2] += A[(size_t)e * ndm * ndm + x];
    }
    __syncthreads();
  }
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      double d = D[(size_t)k * n + k];
      if (!(d > 0.0)) { bad = 1; d = 1.0; }
      D[(size_t)k * n + k] = sqrt(d);
    }
    __syncthreads();
    const double piv = D[(size_t)k * n + k];
    for (int r = k + 1 + tid; r < n; r += blockDim.x) D[(size_t)r * n + k] /= piv;
    __syncthreads();
    const int m = n - k - 1;
    for (long long x = tid; x < (long long)m * m; x += blockDim.x) {
      const int r = k + 1 + (int)(x / m), c = k + 1 + (int)(x % m);
      if (c <= r) D[(size_t)r * n + c] -= D[(size_t)r * n + k] * D[(size_t)c * n + k];
    }
    __syncthreads();
  }
  for (int c = tid; c < n; c += blockDim.x) {
    for (int r = 0; r < n; ++r) {
      double v = r == c ? 1.0 : 0.0;
      for (int q = 0; q < r; ++q) v -= D[(size_t)r * n + q] * Dinv[(size_t)c * n + q];
      Dinv[(size_t)c * n + r] = v / D[(size_t)r * n + r];
    }
    for (int r = n - 1; r >= 0; --r) {
      double v = Dinv[(size_t)c * n + r];
      for (int q = r + 1; q < n; ++q) v -= D[(size_t)q * n + r] * Dinv[(size_t)c * n + q];
      Dinv[(size_t)c * n + r] = v / D[(size_t)r * n + r];
    }
  }
  if (tid == 0 && bad) atomicExch(err, 1);
}

template <typename T>
__global__ void u_dense_matvec_kernel(int n, const T* __restrict__ M, const T* __restrict__ x,
                                      T* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T s = 0;
  for (int j = 0; j < n; ++j) s += M[(size_t)j * n + i] * x[j];
  y[i] = s;
}

// lambda over all edges [n_edges][P1] from the interior unknowns
__global__ void u_scatter_trace_kernel(int ne, int P1, const int* __restrict__ unit_blk,
                                       const double* __restrict__ x, double* __restrict__ lam) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)ne * P1) return;
  const int m = (int)(id / P1), k = (int)(id % P1);
  const int b = unit_blk[m];
  lam[id] = b < 0 ? 0.0 : x[(size_t)b * P1 + k];
}

// host: 1-D tables of the Gauss-node Lagrange basis and the Legendre traces
UTab make_tables(int p) {
  UTab T;
  std::memset(&T, 0, sizeof(T));
  std::vector<double> x, w;
  gauss_legendre(p + 1, x, w);
  const int m = p + 1;
  for (int i = 0; i < m; ++i) { T.xi[i] = x[i]; T.w[i] = w[i]; }
  auto lag = [&](int j, double s) {
    double v = 1.0;
    for (int k = 0; k < m; ++k)
      if (k != j) v *= (s - x[k]) / (x[j] - x[k]);
    return v;
  };
  auto dlag = [&](int j, double s) {                 // product rule
    double tot = 0.0;
    for (int k = 0; k < m; ++k) {
      if (k == j) continue;
      double t = 1.0 / (x[j] - x[k]);
      for (int l = 0; l < m; ++l)
        if (l != j && l != k) t *= (s - x[l]) / (x[j] - x[l]);
      tot += t;
    }
    return tot;
  };
  for (int j = 0; j < m; ++j) {
    T.le[j] = lag(j, -1.0);
    T.re[j] = lag(j, 1.0);
    for (int i = 0; i < m; ++i) T.Dl[j][i] = dlag(j, x[i]);
  }
  for (int t = 0; t < m; ++t) {
    double p0 = 1.0, p1 = x[t];
    T.Pk[0][t] = 1.0;
    if (m > 1) T.Pk[1][t] = x[t];
    for (int k = 2; k < m; ++k) {
      const double pk = ((2.0 * k - 1.0) * x[t] * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = pk;
      T.Pk[k][t] = pk;
    }
  }
  return T;
}

}  // namespace
}  // namespace hdgmg

// ===========================================================================
// context and C ABI
// ===========================================================================
using namespace hdgmg;

namespace {

struct ULevelDev {
  int nd = 0, n_el = 0, nu = 0, ndm = 0, n_blk = 0, m = 1;
  int *el_slot = nullptr, *blk_t0 = nullptr, *blk_t1 = nullptr;
  double *A = nullptr, *Dinv = nullptr;
  double *r = nullptr, *e = nullptr, *res = nullptr, *t = nullptr, *tmp = nullptr;
  // FP32 copies for the FP32 V-cycle (PREC_FP32 only)
  float *A32 = nullptr, *Dinv32 = nullptr;
  float *r32 = nullptr, *e32 = nullptr, *res32 = nullptr, *t32 = nullptr, *tmp32 = nullptr;
  long long n() const { return (long long)n_blk * nd; }
};

// the buffers of one level in the V-cycle's precision
template <typename T>
struct LV {
  T *A, *Dinv, *r, *e, *res, *t, *tmp;
};
template <typename T>
LV<T> lv(ULevelDev& L);
template <>
LV<double> lv<double>(ULevelDev& L) { return {L.A, L.Dinv, L.r, L.e, L.res, L.t, L.tmp}; }
template <>
LV<float> lv<float>(ULevelDev& L) { return {L.A32, L.Dinv32, L.r32, L.e32, L.res32, L.t32, L.tmp32}; }

struct UHDev {
  UHArgs<double> a{};
  UHArgs<float> a32{};
  int nloc_max = 0;
  size_t jn = 0, ain = 0, yn = 0;
};
template <typename T>
UHArgs<T>& ha(UHDev& h);
template <>
UHArgs<double>& ha<double>(UHDev& h) { return h.a; }
template <>
UHArgs<float>& ha<float>(UHDev& h) { return h.a32; }

hdgmg_status fail_u(hdgmg_status st, const std::string& msg) {
  set_last_error(msg);
  return st;
}

}  // namespace

struct hdgmg_umesh {
  UPlan plan;
  hdgmg_opts opts{};
  cudaStream_t s = nullptr;
  int p = 0, nv = 0, nt = 0, E = 0;
  UTab tab{};
  std::vector<void*> bufs;
  double* xy = nullptr;
  int* quads = nullptr;
  int* unit_blk0 = nullptr;
  double *logk = nullptr, *Lf = nullptr, *Z = nullptr, *M = nullptr;
  std::vector<ULevelDev> L;
  std::vector<UHDev> H;
  double *cD = nullptr, *cInv = nullptr;
  float* cInv32 = nullptr;
  int n_coarse = 0;
  double *x = nullptr, *b = nullptr, *pd = nullptr, *Ap = nullptr, *z = nullptr, *rr = nullptr;
  double *scal = nullptr, *partial = nullptr, *hbuf = nullptr;
  int* err = nullptr;
  bool ready = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, ev3 = nullptr;
  size_t condense_smem = 0, agg_smem = 0;
  // one outer iteration (PCG or fixed point) captured as a CUDA graph on a
  // private stream at the first solve; replayed per iteration
  cudaStream_t cap = nullptr;
  cudaGraphExec_t g_iter[2] = {nullptr, nullptr};
  long long g_nodes[2] = {0, 0};
};

namespace {

template <typename T>
bool dalloc(hdgmg_umesh* c, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc((void**)p, count * sizeof(T)) != cudaSuccess) return false;
  c->bufs.push_back(*p);
  return true;
}

template <typename T>
bool upload(hdgmg_umesh* c, T** p, const std::vector<T>& v) {
  if (!dalloc(c, p, v.size())) return false;
  if (!v.empty() && cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return false;
  return true;
}

hdgmg_status cuda_status(const char* where) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_u(HDGMG_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return HDGMG_OK;
}

template <int P>
void launch_condense_p(hdgmg_umesh* c) {
  note_launch();
  u_condense_kernel<P><<<c->E, 128, c->condense_smem, c->s>>>(c->tab, c->xy, c->quads, c->logk, c->plan.tau,
                                                               c->E, c->L[0].A, c->Lf, c->Z, c->M, c->err);
}

template <int P>
bool set_condense_attr(size_t smem) {
  return cudaFuncSetAttribute(u_condense_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
         cudaSuccess;
}

#define U_DISPATCH(p, F, ...)         \
  switch (p) {                        \
    case 1: F<1>(__VA_ARGS__); break; \
    case 2: F<2>(__VA_ARGS__); break; \
    case 3: F<3>(__VA_ARGS__); break; \
    case 4: F<4>(__VA_ARGS__); break; \
    case 5: F<5>(__VA_ARGS__); break; \
    case 6: F<6>(__VA_ARGS__); break; \
    case 7: F<7>(__VA_ARGS__); break; \
    default: F<8>(__VA_ARGS__); break; \
  }

template <int P>
void launch_rhs_p(hdgmg_umesh* c, const double* f, double* t) {
  constexpr int NT = 4 * (P + 1);
  note_launch();
  u_rhs_kernel<P><<<nblk((long long)c->E * NT, 128), 128, 0, c->s>>>(c->E, c->Z, c->M, f, t);
}

template <int P>
void launch_recover_p(hdgmg_umesh* c, const double* lam, const double* f, double* u, double* q) {
  note_launch();
  u_recover_kernel<P><<<c->E, 128, 0, c->s>>>(c->tab, c->xy, c->quads, c->logk, c->L[0].el_slot, c->Lf, c->Z, f,
                                               lam, u, q);
}

template <typename T>
T* coarse_inverse(hdgmg_umesh* c);
template <>
double* coarse_inverse<double>(hdgmg_umesh* c) { return c->cInv; }
template <>
float* coarse_inverse<float>(hdgmg_umesh* c) { return c->cInv32; }

template <typename T, int ND>
void mesh_matvec(hdgmg_umesh* c, ULevelDev& L, const T* x) {
  const LV<T> v = lv<T>(L);
  u_elem_matvec_mesh_kernel<T, ND><<<nblk((long long)L.n_el * 4 * ND, 128), 128, 0, c->s>>>(L.n_el, L.el_slot, v.A,
                                                                                          x, v.t);
}

// y = A_k x (SUM), y = r - A_k x (RES) or y = x + omega Dinv (r - A_k x)
// (SMOOTH; y never aliases x), in precision T.  Mesh levels stream their
// element operators from HBM: one thread per element row (coalesced) into the
// slot buffer, then the edge sums.  Macro-element levels are small and
// latency-bound: one pass pulled per macro-edge.
template <typename T>
void level_matvec(hdgmg_umesh* c, int k, const T* x, T* y, int mode, const T* r) {
  ULevelDev& L = c->L[k];
  if (L.n_blk == 0) return;
  const LV<T> v = lv<T>(L);
  if (k <= c->plan.first_h && L.nu == 4) {
    note_launch();
    switch (L.nd) {
      case 2: mesh_matvec<T, 2>(c, L, x); break;
      case 3: mesh_matvec<T, 3>(c, L, x); break;
      case 4: mesh_matvec<T, 4>(c, L, x); break;
      case 5: mesh_matvec<T, 5>(c, L, x); break;
      case 6: mesh_matvec<T, 6>(c, L, x); break;
      case 7: mesh_matvec<T, 7>(c, L, x); break;
      case 8: mesh_matvec<T, 8>(c, L, x); break;
      default: mesh_matvec<T, 9>(c, L, x); break;
    }
    note_launch();
    u_edge_kernel<T><<<nblk(L.n_blk, 128), 128, 0, c->s>>>(L.n_blk, L.nd, L.blk_t0, L.blk_t1, v.t, x, r, v.Dinv,
                                                           c->opts.omega, mode, y);
  } else {
    note_launch();
    if (std::is_same<T, float>::value)
      u_pull_kernel<T><<<nblk(L.n_blk, 4), 128, 0, c->s>>>(L.n_blk, L.nu, L.el_slot, L.blk_t0, L.blk_t1, v.A,
                                                            x, r, v.Dinv, c->opts.omega, mode, y);
    else
      u_pull_row_kernel<T><<<nblk(L.n_blk, 64), 128, 0, c->s>>>(L.n_blk, L.nu, L.el_slot, L.blk_t0, L.blk_t1,
                                                                 v.A, x, r, v.Dinv, c->opts.omega, mode, y);
  }
}

// e = B_k r (Algorithm 1) in precision T
template <typename T>
void vcycle(hdgmg_umesh* c, int k, const T* r, T* e) {
  ULevelDev& L = c->L[k];
  const int nl = (int)c->L.size();
  if (k == nl - 1) {
    if (c->n_coarse == 0) return;
    note_launch();
    u_dense_matvec_kernel<T><<<nblk(c->n_coarse, 128), 128, 0, c->s>>>(c->n_coarse, coarse_inverse<T>(c), r, e);
    return;
  }
  const double om = c->opts.omega;
  if (L.n_blk == 0) return;
  const LV<T> v = lv<T>(L);
  // step 2: pre-smoothing from zero; the steps alternate between e and tmp
  // and end in e
  T* cur = ((L.m - 1) % 2 == 1) ? v.tmp : e;
  note_launch();
  u_bj_first_kernel<T><<<nblk(L.n_blk, 128), 128, 0, c->s>>>(L.n_blk, L.nd, v.Dinv, r, om, cur);
  for (int it = 1; it < L.m; ++it) {
    T* nxt = cur == e ? v.tmp : e;
    level_matvec<T>(c, k, cur, nxt, U_SMOOTH, r);
    cur = nxt;
  }
  const bool hlev = k >= c->plan.first_h;
  const int lc = c->opts.local_corr;
  UHDev* H = hlev ? &c->H[k - c->plan.first_h] : nullptr;
  if (hlev && (lc == HDGMG_LC_PRE || lc == HDGMG_LC_BOTH)) {      // step 3
    level_matvec<T>(c, k, e, v.res, U_RES, r);
    note_launch();
    u_localcorr_kernel<T><<<H->a.n_E, 64, 0, c->s>>>(ha<T>(*H), v.res, e);
  }
  level_matvec<T>(c, k, e, v.res, U_RES, r);                      // step 4
  ULevelDev& C = c->L[k + 1];
  const LV<T> cv = lv<T>(C);
  if (hlev) {
    note_launch();
    u_restrict_kernel<T><<<H->a.n_E, 64, 0, c->s>>>(ha<T>(*H), v.res, cv.t);
    if (C.n_blk > 0) {
      note_launch();
      u_unit_kernel<T><<<nblk(C.n_blk, 128), 128, 0, c->s>>>(C.n_blk, 2, C.blk_t0, C.blk_t1, cv.t, cv.r);
    }
  } else {
    note_launch();
    u_prestrict_kernel<T><<<nblk(2LL * L.n_blk, 128), 128, 0, c->s>>>(L.n_blk, L.nd, v.res, cv.r);
  }
  vcycle<T>(c, k + 1, cv.r, cv.e);
  if (hlev) {
    note_launch();
    u_prolong_kernel<T><<<H->a.n_E, 64, 0, c->s>>>(ha<T>(*H), C.el_slot, cv.e, e);
  } else {
    note_launch();
    u_pprolong_kernel<T><<<nblk(2LL * L.n_blk, 128), 128, 0, c->s>>>(L.n_blk, L.nd, cv.e, e);
  }
  if (hlev && lc == HDGMG_LC_BOTH) {                              // step 5
    level_matvec<T>(c, k, e, v.res, U_RES, r);
    note_launch();
    u_localcorr_kernel<T><<<H->a.n_E, 64, 0, c->s>>>(ha<T>(*H), v.res, e);
  }
  cur = e;                                                        // step 6
  if (L.m % 2 == 1) {
    cudaMemcpyAsync(v.tmp, e, (size_t)L.n() * sizeof(T), cudaMemcpyDeviceToDevice, c->s);
    cur = v.tmp;
  }
  for (int it = 0; it < L.m; ++it) {
    T* nxt = cur == e ? v.tmp : e;
    level_matvec<T>(c, k, cur, nxt, U_SMOOTH, r);
    cur = nxt;
  }
}

// z = B r on the finest level (FP64 in and out), the cycle in the context's
// precision: FP32 levels behind an FP64 -> FP32 -> FP64 hand-over
void apply_B(hdgmg_umesh* c, const double* r, double* z) {
  if (c->opts.precision == HDGMG_PREC_FP32) {
    ULevelDev& L0 = c->L[0];
    launch_convert<double, float>(c->s, L0.n(), r, L0.r32);
    vcycle<float>(c, 0, L0.r32, L0.e32);
    launch_convert<float, double>(c->s, L0.n(), L0.e32, z);
  } else {
    vcycle<double>(c, 0, r, z);
  }
}

hdgmg_status read_err(hdgmg_umesh* c, const char* what) {
  int h = 0;
  if (cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->s) != cudaSuccess ||
      cudaStreamSynchronize(c->s) != cudaSuccess)
    return cuda_status(what);
  if (h) {
    cudaMemsetAsync(c->err, 0, sizeof(int), c->s);
    return fail_u(HDGMG_EBREAKDOWN, std::string(what) + ": non-positive pivot");
  }
  return HDGMG_OK;
}

double read_scalar(hdgmg_umesh* c, const double* d) {
  cudaMemcpyAsync(c->hbuf, d, sizeof(double), cudaMemcpyDeviceToHost, c->s);
  cudaStreamSynchronize(c->s);
  return *c->hbuf;
}

// one PCG iteration: alpha, x, r, |r|^2 (scal[5]), z = B r, beta, p
void pcg_body(hdgmg_umesh* c) {
  const long long n = c->L[0].n();
  level_matvec<double>(c, 0, c->pd, c->Ap, U_SUM, nullptr);
  launch_dot(c->s, n, c->pd, c->Ap, c->partial, c->scal + 1);
  launch_cg_scalars(c->s, c->scal, 0);
  launch_cg_update(c->s, n, c->scal, c->x, c->rr, c->pd, c->Ap);
  launch_dot(c->s, n, c->rr, c->rr, c->partial, c->scal + 5);
  apply_B(c, c->rr, c->z);
  launch_dot(c->s, n, c->rr, c->z, c->partial, c->scal + 3);
  launch_cg_scalars(c->s, c->scal, 1);
  launch_cg_direction(c->s, n, c->scal, c->z, c->pd);
}

// one fixed-point iteration x += B (b - A x), then |b - A x|^2 (scal[5])
void fp_body(hdgmg_umesh* c) {
  const long long n = c->L[0].n();
  level_matvec<double>(c, 0, c->x, c->rr, U_RES, c->b);
  apply_B(c, c->rr, c->z);
  launch_axpby(c->s, n, 1.0, c->z, 1.0, c->x);
  level_matvec<double>(c, 0, c->x, c->rr, U_RES, c->b);
  launch_dot(c->s, n, c->rr, c->rr, c->partial, c->scal + 5);
}

// captures body k (0 PCG, 1 fixed point) once; false if capture failed
bool ensure_graph(hdgmg_umesh* c, int k) {
  if (c->g_iter[k]) return true;
  cudaStream_t saved = c->s;
  c->s = c->cap;
  const long long l0 = launch_count();
  if (cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    c->s = saved;
    return false;
  }
  if (k == 0) pcg_body(c);
  else fp_body(c);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->cap, &g);
  c->s = saved;
  c->g_nodes[k] = launch_count() - l0;
  if (e != cudaSuccess || !g) return false;
  const bool ok = cudaGraphInstantiate(&c->g_iter[k], g, 0) == cudaSuccess;
  cudaGraphDestroy(g);
  return ok;
}

}  // namespace

extern "C" {

void hdgmg_umesh_default_opts(hdgmg_opts* o) {
  if (!o) return;
  hdgmg_default_opts(o);
  o->omega = 0.8;
  o->m_fine = 2;
  o->m_max = 4;
}

hdgmg_status hdgmg_umesh_create(hdgmg_umesh** out, const hdgmg_umesh_problem* pr, const hdgmg_opts* opts,
                                void* stream) {
  if (!out || !pr) return fail_u(HDGMG_EINVAL, "null argument");
  *out = nullptr;
  hdgmg_opts o;
  if (opts) {
    o = *opts;
  } else {
    hdgmg_umesh_default_opts(&o);
  }
  if (o.precision != HDGMG_PREC_FP64 && o.precision != HDGMG_PREC_FP32)
    return fail_u(HDGMG_EINVAL, "the unstructured path runs the V-cycle in FP64 or FP32");
  if (o.smoother != HDGMG_SMOOTH_BLOCK_JACOBI) return fail_u(HDGMG_EINVAL, "the unstructured path smooths by block-Jacobi");
  if (o.krylov != HDGMG_KRYLOV_NONE && o.krylov != HDGMG_KRYLOV_CG)
    return fail_u(HDGMG_EINVAL, "the unstructured path supports krylov NONE or CG");
  if (o.m_fine < 1 || o.m_growth < 1 || o.m_max < 0 || o.max_it < 1 || !(o.rtol > 0.0) || !(o.omega > 0.0) ||
      o.local_corr < HDGMG_LC_NONE || o.local_corr > HDGMG_LC_BOTH)
    return fail_u(HDGMG_EINVAL, "invalid options");
  auto* c = new (std::nothrow) hdgmg_umesh;
  if (!c) return fail_u(HDGMG_ENOMEM, "host allocation failed");
  std::string err;
  if (!build_uplan(*pr, c->plan, err)) {
    delete c;
    return fail_u(HDGMG_EINVAL, err);
  }
  c->opts = o;
  c->s = (cudaStream_t)stream;
  UPlan& P = c->plan;
  c->p = P.p;
  c->nv = (P.p + 1) * (P.p + 1);
  c->nt = 4 * (P.p + 1);
  c->E = P.E;
  c->tab = make_tables(P.p);
  const UPlanLevel& Lcoarse = P.levels.back();
  c->n_coarse = Lcoarse.n_blk * Lcoarse.nd;
  auto bail = [&](hdgmg_status st, const std::string& m) {
    hdgmg_umesh_destroy(c);
    return fail_u(st, m);
  };
  if (c->n_coarse > kMaxCoarse)
    return bail(HDGMG_EINVAL, "coarsest level has " + std::to_string(c->n_coarse) + " unknowns (> 1024): use fewer seeds");
  for (const UPlanH& h : P.hc)
    if (2 * h.nloc_max > kMaxLoc)
      return bail(HDGMG_EINVAL, "a macro-element's local system has " + std::to_string(2 * h.nloc_max) +
                                    " unknowns (> 160): use more seeds");
  for (size_t k = 0; k < P.levels.size(); ++k)
    if (k > 0 && P.levels[k].nu > 64)
      return bail(HDGMG_EINVAL, "a macro-element has more than 64 macro-edges: use more seeds");
  const size_t E = (size_t)P.E;
  bool ok = upload(c, &c->xy, P.xy) && upload(c, &c->quads, P.quads) &&
            dalloc(c, &c->logk, E) && dalloc(c, &c->Lf, E * c->nv * c->nv) &&
            dalloc(c, &c->Z, E * c->nv * c->nt) && dalloc(c, &c->M, E * c->nv) && dalloc(c, &c->err, 1);
  // levels
  int m = o.m_fine;
  for (size_t k = 0; ok && k < P.levels.size(); ++k) {
    const UPlanLevel& pl = P.levels[k];
    ULevelDev d;
    d.nd = pl.nd;
    d.n_el = pl.n_el;
    d.nu = pl.nu;
    d.ndm = pl.nu * pl.nd;
    d.n_blk = pl.n_blk;
    d.m = m;
    m *= o.m_growth;
    if (o.m_max > 0) m = std::min(m, o.m_max);
    ok = upload(c, &d.el_slot, pl.el_slot) && upload(c, &d.blk_t0, pl.blk_t0) && upload(c, &d.blk_t1, pl.blk_t1) &&
         dalloc(c, &d.A, (size_t)d.n_el * d.ndm * d.ndm) && dalloc(c, &d.Dinv, (size_t)d.n_blk * d.nd * d.nd) &&
         dalloc(c, &d.r, (size_t)d.n()) && dalloc(c, &d.e, (size_t)d.n()) && dalloc(c, &d.res, (size_t)d.n()) &&
         dalloc(c, &d.tmp, (size_t)d.n()) &&
         dalloc(c, &d.t, (size_t)d.n_el * d.ndm);
    if (ok && o.precision == HDGMG_PREC_FP32)
      ok = dalloc(c, &d.A32, (size_t)d.n_el * d.ndm * d.ndm) && dalloc(c, &d.Dinv32, (size_t)d.n_blk * d.nd * d.nd) &&
           dalloc(c, &d.r32, (size_t)d.n()) && dalloc(c, &d.e32, (size_t)d.n()) &&
           dalloc(c, &d.res32, (size_t)d.n()) && dalloc(c, &d.tmp32, (size_t)d.n()) &&
           dalloc(c, &d.t32, (size_t)d.n_el * d.ndm);
    c->L.push_back(d);
  }
  ok = ok && upload(c, &c->unit_blk0, P.levels[0].unit_blk);
  for (size_t i = 0; ok && i < P.hc.size(); ++i) {
    const UPlanH& h = P.hc[i];
    const UPlanLevel& lf = P.levels[P.first_h + i];
    const UPlanLevel& lc = P.levels[P.first_h + i + 1];
    UHDev d;
    d.a.n_E = h.n_E;
    d.a.nu_f = lf.nu;
    d.a.nd_f = lf.nd;
    d.a.nu_c = lc.nu;
    d.nloc_max = h.nloc_max;
    // per E, the B rows of each coarse slot (blocks, cumulative), padded to nu_c + 1
    std::vector<int> blk_chain(lc.n_blk, -1);
    for (size_t q = 0; q < P.chains[lc.t].size(); ++q)
      if (lc.unit_blk[q] >= 0) blk_chain[lc.unit_blk[q]] = (int)q;
    std::vector<int> bs((size_t)h.n_E * (lc.nu + 1), 0);
    for (int Ei = 0; Ei < h.n_E; ++Ei) {
      int* row = &bs[(size_t)Ei * (lc.nu + 1)];
      int cnt = 0;
      for (int s = 0; s < lc.nu; ++s) {
        const int cb = lc.el_slot[(size_t)Ei * lc.nu + s];
        if (cb >= 0)      // units of this macro-edge carrying unknowns on the finer level
          for (int u : P.chains[lc.t][blk_chain[cb]].units)
            if (lf.unit_blk[u] >= 0) ++cnt;
        row[s + 1] = cnt;
      }
    }
    const int *lp, *lb, *nI, *own, *cp, *ce, *cm, *bsp;
    const long long *jo, *ao, *yo;
    const double* J;
    double *AI, *Y;
    ok = upload(c, (int**)&lp, h.loc_ptr) && upload(c, (int**)&lb, h.loc_blk) && upload(c, (int**)&nI, h.nI) &&
         upload(c, (int**)&own, h.own) && upload(c, (int**)&cp, h.ch_ptr) && upload(c, (int**)&ce, h.ch_el) &&
         upload(c, (int**)&cm, h.ch_map) && upload(c, (int**)&bsp, bs) &&
         upload(c, (long long**)&jo, h.J_off) && upload(c, (long long**)&ao, h.AI_off) &&
         upload(c, (long long**)&yo, h.Y_off) && upload(c, (double**)&J, h.J) &&
         dalloc(c, &AI, (size_t)h.AI_off.back()) && dalloc(c, &Y, (size_t)h.Y_off.back());
    if (!ok) break;
    d.a.loc_ptr = lp; d.a.loc_blk = lb; d.a.nI = nI; d.a.own = own; d.a.ch_ptr = cp; d.a.ch_el = ce;
    d.a.ch_map = cm; d.a.bs_ptr = bsp; d.a.J_off = jo; d.a.AI_off = ao; d.a.Y_off = yo; d.a.J = J;
    d.a.AIinv = AI; d.a.Y = Y;
    d.jn = h.J.size();
    d.ain = (size_t)h.AI_off.back();
    d.yn = (size_t)h.Y_off.back();
    d.a32.n_E = d.a.n_E; d.a32.nu_f = d.a.nu_f; d.a32.nd_f = d.a.nd_f; d.a32.nu_c = d.a.nu_c;
    d.a32.loc_ptr = lp; d.a32.loc_blk = lb; d.a32.nI = nI; d.a32.own = own; d.a32.ch_ptr = cp; d.a32.ch_el = ce;
    d.a32.ch_map = cm; d.a32.bs_ptr = bsp; d.a32.J_off = jo; d.a32.AI_off = ao; d.a32.Y_off = yo;
    if (o.precision == HDGMG_PREC_FP32) {
      float *J32, *AI32, *Y32;
      ok = dalloc(c, &J32, d.jn) && dalloc(c, &AI32, d.ain) && dalloc(c, &Y32, d.yn);
      if (!ok) break;
      d.a32.J = J32; d.a32.AIinv = AI32; d.a32.Y = Y32;
    }
    c->H.push_back(d);
    c->agg_smem = std::max(c->agg_smem, (size_t)4 * h.nloc_max * h.nloc_max * sizeof(double));
  }
  const long long nf = c->L[0].n();
  if (ok && o.precision == HDGMG_PREC_FP32) ok = dalloc(c, &c->cInv32, (size_t)c->n_coarse * c->n_coarse);
  ok = ok && dalloc(c, &c->cD, (size_t)c->n_coarse * c->n_coarse) &&
       dalloc(c, &c->cInv, (size_t)c->n_coarse * c->n_coarse) && dalloc(c, &c->x, nf) && dalloc(c, &c->b, nf) &&
       dalloc(c, &c->pd, nf) && dalloc(c, &c->Ap, nf) && dalloc(c, &c->z, nf) && dalloc(c, &c->rr, nf) &&
       dalloc(c, &c->scal, 16) && dalloc(c, &c->partial, kDotBlocks);
  if (!ok) return bail(HDGMG_ENOMEM, "device allocation failed");
  if (cudaMallocHost((void**)&c->hbuf, 64) != cudaSuccess) return bail(HDGMG_ENOMEM, "pinned allocation failed");
  cudaMemset(c->err, 0, sizeof(int));
  const int nv = c->nv, nt = c->nt;
  c->condense_smem = (size_t)(nv * nv + 2 * nv * nt + nt * nt + 2 * nv * (2 * c->p + 1)) * sizeof(double);
  bool attr = true;
  switch (c->p) {
    case 1: attr = set_condense_attr<1>(c->condense_smem); break;
    case 2: attr = set_condense_attr<2>(c->condense_smem); break;
    case 3: attr = set_condense_attr<3>(c->condense_smem); break;
    case 4: attr = set_condense_attr<4>(c->condense_smem); break;
    case 5: attr = set_condense_attr<5>(c->condense_smem); break;
    case 6: attr = set_condense_attr<6>(c->condense_smem); break;
    case 7: attr = set_condense_attr<7>(c->condense_smem); break;
    default: attr = set_condense_attr<8>(c->condense_smem); break;
  }
  if (c->agg_smem > 0)
    attr = attr && cudaFuncSetAttribute(u_agglomerate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)c->agg_smem) == cudaSuccess;
  if (!attr) return bail(HDGMG_ECUDA, "shared-memory attribute refused");
  if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess)
    return bail(HDGMG_ECUDA, "stream creation failed");
  if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess ||
      cudaEventCreate(&c->ev2) != cudaSuccess || cudaEventCreate(&c->ev3) != cudaSuccess)
    return bail(HDGMG_ECUDA, "event creation failed");
  *out = c;
  return HDGMG_OK;
}

hdgmg_status hdgmg_umesh_setup(hdgmg_umesh* c, const double* log_kappa) {
  if (!c || !log_kappa) return fail_u(HDGMG_EINVAL, "null argument");
  cudaMemcpyAsync(c->logk, log_kappa, (size_t)c->E * sizeof(double), cudaMemcpyDeviceToDevice, c->s);
  cudaEventRecord(c->ev0, c->s);
  cudaEventRecord(c->ev2, c->s);
  U_DISPATCH(c->p, launch_condense_p, c);
  cudaEventRecord(c->ev3, c->s);
  UPlan& P = c->plan;
  if (P.p > 1) {
    note_launch();
    u_pcoarsen_kernel<<<nblk((long long)c->E * 64, 128), 128, 0, c->s>>>(c->E, P.p + 1, c->L[0].A, c->L[1].A);
  }
  for (size_t i = 0; i < c->H.size(); ++i) {
    ULevelDev& Lf = c->L[P.first_h + i];
    ULevelDev& Lc = c->L[P.first_h + i + 1];
    note_launch();
    u_agglomerate_kernel<<<c->H[i].a.n_E, 256, (size_t)4 * c->H[i].nloc_max * c->H[i].nloc_max * sizeof(double),
                           c->s>>>(c->H[i].a, Lf.A, Lc.A, c->err);
  }
  for (size_t k = 0; k + 1 < c->L.size(); ++k) {
    ULevelDev& L = c->L[k];
    if (L.n_blk == 0) continue;
    note_launch();
    u_bjinv_kernel<<<nblk(L.n_blk, 64), 64, 0, c->s>>>(L.n_blk, L.nu, L.nd, L.blk_t0, L.blk_t1, L.A, L.Dinv,
                                                       c->err);
  }
  ULevelDev& C = c->L.back();
  if (c->n_coarse > 0) note_launch();
  if (c->n_coarse > 0)
    u_coarse_setup_kernel<<<1, 1024, 0, c->s>>>(c->n_coarse, C.n_el, C.nu, C.el_slot, C.A, c->cD, c->cInv, c->err);
  if (c->opts.precision == HDGMG_PREC_FP32) {     // the FP32 V-cycle's copies
    for (size_t k = 0; k < c->L.size(); ++k) {
      ULevelDev& L = c->L[k];
      launch_convert<double, float>(c->s, (int64_t)L.n_el * L.ndm * L.ndm, L.A, L.A32);
      if (k + 1 < c->L.size() && L.n_blk > 0)
        launch_convert<double, float>(c->s, (int64_t)L.n_blk * L.nd * L.nd, L.Dinv, L.Dinv32);
    }
    for (UHDev& h : c->H) {
      if (h.jn) launch_convert<double, float>(c->s, (int64_t)h.jn, h.a.J, const_cast<float*>(h.a32.J));
      if (h.ain) launch_convert<double, float>(c->s, (int64_t)h.ain, h.a.AIinv, h.a32.AIinv);
      if (h.yn) launch_convert<double, float>(c->s, (int64_t)h.yn, h.a.Y, h.a32.Y);
    }
    if (c->n_coarse > 0)
      launch_convert<double, float>(c->s, (int64_t)c->n_coarse * c->n_coarse, c->cInv, c->cInv32);
  }
  cudaEventRecord(c->ev1, c->s);
  hdgmg_status st = cuda_status("set-up");
  if (st != HDGMG_OK) return st;
  st = read_err(c, "set-up");
  if (st != HDGMG_OK) return st;
  c->ready = true;
  return HDGMG_OK;
}

hdgmg_status hdgmg_umesh_vcycle(hdgmg_umesh* c, const double* r, double* z) {
  if (!c || !r || !z) return fail_u(HDGMG_EINVAL, "null argument");
  if (!c->ready) return fail_u(HDGMG_EINVAL, "set-up required");
  apply_B(c, r, z);
  hdgmg_status st = cuda_status("vcycle");
  if (st == HDGMG_OK && cudaStreamSynchronize(c->s) != cudaSuccess) st = cuda_status("vcycle");
  return st;
}

hdgmg_status hdgmg_umesh_apply(hdgmg_umesh* c, int32_t level, const double* x, double* y) {
  if (!c || !x || !y) return fail_u(HDGMG_EINVAL, "null argument");
  if (!c->ready) return fail_u(HDGMG_EINVAL, "set-up required");
  if (level < 0 || level >= (int32_t)c->L.size()) return fail_u(HDGMG_EINVAL, "level out of range");
  level_matvec<double>(c, level, x, y, U_SUM, nullptr);
  hdgmg_status st = cuda_status("apply");
  if (st == HDGMG_OK && cudaStreamSynchronize(c->s) != cudaSuccess) st = cuda_status("apply");
  return st;
}

hdgmg_status hdgmg_umesh_level_sizes(const hdgmg_umesh* c, int32_t level, int64_t* out) {
  if (!c || !out) return fail_u(HDGMG_EINVAL, "null argument");
  if (level < 0 || level >= (int32_t)c->L.size()) return fail_u(HDGMG_EINVAL, "level out of range");
  const ULevelDev& L = c->L[level];
  out[0] = L.n();
  out[1] = L.n_el;
  out[2] = L.nd;
  out[3] = L.ndm;
  return HDGMG_OK;
}

hdgmg_status hdgmg_umesh_element_matrices(const hdgmg_umesh* c, int32_t level, double* A, int32_t* dofs) {
  if (!c) return fail_u(HDGMG_EINVAL, "null argument");
  if (A && !c->ready) return fail_u(HDGMG_EINVAL, "set-up required");
  if (level < 0 || level >= (int32_t)c->L.size()) return fail_u(HDGMG_EINVAL, "level out of range");
  const ULevelDev& L = c->L[level];
  const UPlanLevel& pl = c->plan.levels[level];
  if (A) {
    if (cudaMemcpyAsync(A, L.A, (size_t)L.n_el * L.ndm * L.ndm * sizeof(double), cudaMemcpyDeviceToDevice,
                        c->s) != cudaSuccess ||
        cudaStreamSynchronize(c->s) != cudaSuccess)
      return cuda_status("element matrices");
  }
  if (dofs)
    for (int e = 0; e < L.n_el; ++e)
      for (int i = 0; i < L.ndm; ++i) {
        const int b = pl.el_slot[(size_t)e * L.nu + i / L.nd];
        dofs[(size_t)e * L.ndm + i] = b < 0 ? -1 : b * L.nd + i % L.nd;
      }
  return HDGMG_OK;
}

hdgmg_status hdgmg_umesh_solve(hdgmg_umesh* c, const double* f, double* lam, double* u, double* q,
                               hdgmg_info* info) {
  if (!c || !f || !lam) return fail_u(HDGMG_EINVAL, "null argument");
  if (!c->ready) return fail_u(HDGMG_EINVAL, "set-up required");
  ULevelDev& L0 = c->L[0];
  const long long n = L0.n();
  float t_setup = 0.0f, t_cond = 0.0f;
  cudaEventElapsedTime(&t_setup, c->ev0, c->ev1);
  cudaEventElapsedTime(&t_cond, c->ev2, c->ev3);
  const long long launches0 = launch_count();
  cudaEventRecord(c->ev0, c->s);
  // b = sum_e g_e on the interior edges
  U_DISPATCH(c->p, launch_rhs_p, c, f, L0.t);
  if (L0.n_blk > 0) {
    note_launch();
    u_unit_kernel<<<nblk(L0.n_blk, 128), 128, 0, c->s>>>(L0.n_blk, L0.nd, L0.blk_t0, L0.blk_t1, L0.t, c->b);
  }
  launch_dot(c->s, n, c->b, c->b, c->partial, c->scal + 6);
  const double bb = read_scalar(c, c->scal + 6);
  cudaMemsetAsync(c->x, 0, n * sizeof(double), c->s);
  int it = 0;
  bool conv = bb == 0.0;
  double rel = 0.0;
  bool broke = false;
  const int gk = c->opts.krylov == HDGMG_KRYLOV_CG ? 0 : 1;
  long long captured = 0, replayed = 0;
  if (!conv) {
    // the iteration body as one graph (captured at the first solve)
    const bool had = c->g_iter[gk] != nullptr;
    const bool use_graph = ensure_graph(c, gk);
    if (!had) captured = c->g_nodes[gk];
    if (gk == 0) {
      cudaMemcpyAsync(c->rr, c->b, n * sizeof(double), cudaMemcpyDeviceToDevice, c->s);   // r = b
      apply_B(c, c->rr, c->z);
      cudaMemcpyAsync(c->pd, c->z, n * sizeof(double), cudaMemcpyDeviceToDevice, c->s);
      launch_dot(c->s, n, c->rr, c->z, c->partial, c->scal + 0);
    }
    while (it < c->opts.max_it) {
      if (use_graph) {
        cudaGraphLaunch(c->g_iter[gk], c->s);
        replayed += c->g_nodes[gk];
      } else if (gk == 0) {
        pcg_body(c);
      } else {
        fp_body(c);
      }
      ++it;
      rel = std::sqrt(read_scalar(c, c->scal + 5) / bb);
      if (!std::isfinite(rel) || (gk == 1 && rel > 1e8)) { broke = true; break; }
      if (rel <= c->opts.rtol) { conv = true; break; }
    }
  }
  // true residual
  level_matvec<double>(c, 0, c->x, c->rr, U_RES, c->b);
  launch_dot(c->s, n, c->rr, c->rr, c->partial, c->scal + 5);
  rel = bb > 0 ? std::sqrt(read_scalar(c, c->scal + 5) / bb) : 0.0;
  note_launch();
  u_scatter_trace_kernel<<<nblk((long long)c->plan.ne * (c->p + 1), 128), 128, 0, c->s>>>(
      c->plan.ne, c->p + 1, c->unit_blk0, c->x, lam);
  if (u || q) U_DISPATCH(c->p, launch_recover_p, c, c->x, f, u, q);
  cudaEventRecord(c->ev1, c->s);
  hdgmg_status st = cuda_status("solve");
  if (st == HDGMG_OK && cudaStreamSynchronize(c->s) != cudaSuccess) st = cuda_status("solve");
  if (st != HDGMG_OK) return st;
  float t_solve = 0.0f;
  cudaEventElapsedTime(&t_solve, c->ev0, c->ev1);
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iters = it;
    info->converged = conv ? 1 : 0;
    info->rel_res = rel;
    info->t_setup_ms = t_setup;
    info->t_solve_ms = t_solve;
    info->n_levels = (int32_t)c->L.size();
    info->trace_dofs = c->plan.trace_dofs;
    info->kernel_launches = launch_count() - launches0 - captured + replayed;
    info->t_condense_ms = t_cond;
    info->condense_threads = 128;
    info->condense_elements_per_block = 1;
    info->condense_kind = HDGMG_CONDENSE_FACTOR;
  }
  if (broke) return fail_u(HDGMG_EBREAKDOWN, "the iteration broke down (NaN/Inf or divergence)");
  if (!conv) return fail_u(HDGMG_ENOCONV, "max_it reached");
  return HDGMG_OK;
}

void hdgmg_umesh_destroy(hdgmg_umesh* c) {
  if (!c) return;
  if (c->s) cudaStreamSynchronize(c->s);
  for (void* p : c->bufs) cudaFree(p);
  if (c->hbuf) cudaFreeHost(c->hbuf);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->ev2) cudaEventDestroy(c->ev2);
  for (auto& g : c->g_iter)
    if (g) cudaGraphExecDestroy(g);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->ev3) cudaEventDestroy(c->ev3);
  delete c;
}

}  // extern "C"
