// Internal declarations of the hdgmg library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/hdgmg.h"

namespace hdgmg {

// ---------------------------------------------------------------------------
// Reference element (host, FP64).  Uniform rectangle hx x hy, volume space Q_p
// with Lagrange basis at the (p+1)^2 Gauss-Legendre nodes, trace space P_p
// per edge in the orthonormal Legendre basis.  With Gauss quadrature on the
// nodes every bilinear form of the scheme is integrated exactly, so the mass
// matrix is diagonal.  Matrices are row-major.
//   M      [nv]        diagonal mass  (phi_a, phi_a)
//   G      [nv][nv]    sum_d B_d M^-1 B_d^T          (q eliminated)
//   E      [nv][nv]    <phi_a, phi_b>_dK
//   H      [nv][nt]    sum_d B_d M^-1 C_d
//   F      [nv][nt]    <psi_k, phi_a>_dK
//   K      [nt][nt]    sum_d C_d^T M^-1 C_d
//   BxT,ByT [nv][nv]   B_d^T  (BdT[a][b] = (phi_b, d_d phi_a)), recovery of q
//   Cx, Cy [nv][nt]    <psi_k, phi_a n_d>, recovery of q
// ---------------------------------------------------------------------------
struct RefElement {
  int p = 0, nv = 0, nt = 0;
  double hx = 0, hy = 0;
  std::vector<double> nodes, weights;
  std::vector<double> M, G, E, H, F, K, BxT, ByT, Cx, Cy;
};
RefElement build_ref_element(int p, double hx, double hy);

// Gauss-Legendre rule on [-1, 1] (ascending nodes) by Newton iteration on P_m.
void gauss_legendre(int m, std::vector<double>& x, std::vector<double>& w);

// Closed-form P1 child injection J_c [child][fine mode][coarse mode] for a
// macro-edge split into two halves (orthonormal Legendre on both).
void child_injection(double J[2][2][2]);

// ---------------------------------------------------------------------------
// Device-side level data.  Vectors are [nd][n_edges] (mode-major, edge
// fastest).  Element operators are symmetric, stored packed (lower triangle,
// row-major: (r,c), r >= c -> r(r+1)/2 + c) in structure-of-arrays form
// [entry][element] so that a warp of consecutive elements loads one entry of
// 32 consecutive matrices in one coalesced access.
// ---------------------------------------------------------------------------
template <typename T>
struct LevelData {
  T* A = nullptr;        // [nl(nl+1)/2][nE]
  T* Dinv = nullptr;     // [nd(nd+1)/2][nEdge]  inverse edge blocks, packed
  // transfer to the next coarser level when it is an h-transfer (per coarse
  // macro-element C of the next level, nC = nE/4):
  T* AIIinv = nullptr;   // [36][nC]   A_II^-1 (8x8, packed)
  T* Y = nullptr;        // [128][nC]  -A_II^-1 A_IB  (8x16, row-major)
  T* Pi = nullptr;       // [64][nC]   -A_II^-1 A_IB J (8x8, row-major)
  T* r = nullptr;        // level right-hand side   [nd][nEdge]
  T* e = nullptr;        // level correction        [nd][nEdge]
  T* y = nullptr;        // matvec accumulator      [nd][nEdge] (kept zero)
};

struct Level {
  int n = 0;       // macro-elements per side
  int nd = 0;      // trace modes per edge
  int nl = 0;      // 4*nd
  int nsym = 0;    // nl(nl+1)/2
  int nE = 0, nEdge = 0;
  int m = 1;       // smoothing steps
  int transfer = 0;   // 0 none (coarsest), 1 p-transfer, 2 h-transfer
  LevelData<double> d64;
  LevelData<float> d32;
};

// ---------------------------------------------------------------------------
// kernel launchers (k_condense.cu, k_mg.cu, k_blas.cu)
// ---------------------------------------------------------------------------
struct RefDevice {     // device copies of RefElement tables (FP64)
  double *M, *G, *E, *H, *F, *K, *BxT, *ByT, *Cx, *Cy;
};

void launch_condense(cudaStream_t s, const RefDevice& ref, int p, int nE,
                     const double* logk, int tau_mode, double tau_c, double hmin,
                     double* A, double* Lfac, int* err);
void launch_rhs(cudaStream_t s, const RefDevice& ref, int p, int n,
                const double* logk, int tau_mode, double tau_c, double hmin,
                const double* Lfac, const double* f, double* b);
void launch_recover(cudaStream_t s, const RefDevice& ref, int p, int n,
                    const double* logk, int tau_mode, double tau_c, double hmin,
                    const double* Lfac, const double* f, const double* lam,
                    double* u, double* q);

template <typename T>
void launch_matvec(cudaStream_t s, int n, int nd, const T* A, const T* x, T* y, T alpha);
// per-ND instantiations (k_edge_inst.cu, one translation unit per type and ND)
template <typename T, int ND>
void launch_matvec_nd(cudaStream_t s, int n, const T* A, const T* x, T* y, T alpha);
template <typename T, int ND>
void launch_bj_blocks_nd(cudaStream_t s, int n, const T* A, T* Dinv, int* err);
template <typename T, int ND>
void launch_bj_update_nd(cudaStream_t s, int n, const T* Dinv, const T* r, T* y, T* e, T omega,
                         int first);
template <typename T>
void launch_bj_blocks(cudaStream_t s, int n, int nd, const T* A, T* Dinv, int* err);
template <typename T>
void launch_bj_update(cudaStream_t s, int n, int nd, const T* Dinv, const T* r, T* y,
                      T* e, T omega, int first);
template <typename T>
void launch_pcoarsen(cudaStream_t s, int nE, int ndf, const T* Af, T* Ac);
template <typename T>
void launch_agglomerate(cudaStream_t s, int nc, const T* Af, T* Ac, T* AIIinv, T* Y,
                        T* Pi, int* err);
template <typename T>
void launch_local_correction(cudaStream_t s, int nc, const T* AIIinv, const T* Y,
                             const T* r, T* e);
template <typename T>
void launch_restrict_h(cudaStream_t s, int nc, const T* Pi, const T* r, T* y, T* rc);
template <typename T>
void launch_prolong_h(cudaStream_t s, int nc, const T* Pi, const T* ec, T* e, T* y);
template <typename T>
void launch_restrict_p(cudaStream_t s, int n, int nd, const T* r, T* y, T* rc);
template <typename T>
void launch_prolong_p(cudaStream_t s, int n, int nd, const T* ec, T* e);

// coarsest level: dense FP64 Cholesky of the interior operator
template <typename T>
void launch_coarse_assemble(cudaStream_t s, int n, const T* A, const int* freeidx, int nf,
                            double* dense);
void launch_coarse_factor(cudaStream_t s, int nf, double* dense, int* err);
template <typename T>
void launch_coarse_solve(cudaStream_t s, int n, const int* freeidx, int nf, const double* L,
                         const T* r, T* e, double* work);

// vector kernels (FP64 unless templated)
void launch_dot(cudaStream_t s, int64_t len, const double* a, const double* b, double* partial,
                double* out);
template <typename T>
void launch_mask(cudaStream_t s, int n, int nd, T* x);   // zero Dirichlet entries
template <typename T>
void launch_unpack(cudaStream_t s, int nl, int nE, const T* Ap, double* full);
template <typename A, typename B>
void launch_convert(cudaStream_t s, int64_t len, const A* in, B* out);
void launch_cg_update(cudaStream_t s, int64_t len, const double* scal, double* x, double* r,
                      const double* p, const double* Ap);
void launch_cg_direction(cudaStream_t s, int64_t len, const double* scal, const double* z,
                         double* p);
void launch_cg_scalars(cudaStream_t s, double* scal, int stage);
void launch_axpby(cudaStream_t s, int64_t len, double a, const double* x, double b, double* y);
void launch_copy_boundary(cudaStream_t s, int n, int nd, const double* gD, double* lam);

// host-side count of kernel launches issued by the library (all threads)
void note_launch();
long long launch_count();

constexpr int kDotBlocks = 608;   // 4 x 152 SMs; fixed for a deterministic sum

}  // namespace hdgmg
