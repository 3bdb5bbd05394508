// Internal declarations of the hdgmg library (not part of the C ABI).
#pragma once

#include <cuda_bf16.h>
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
//                      and the convection term -(beta u, grad w)
//   Cx, Cy [nv][nt]    <psi_k, phi_a n_d>, recovery of q
//   Ef  [4][nv][nv]    <phi_a, phi_b> on face f alone (E = sum_f Ef), for
//                      face-dependent tau (convection-diffusion)
// ---------------------------------------------------------------------------
struct RefElement {
  int p = 0, nv = 0, nt = 0;
  double hx = 0, hy = 0;
  std::vector<double> nodes, weights;
  std::vector<double> M, G, E, H, F, K, BxT, ByT, Cx, Cy, Ef;
  // the kappa-proportional part of the left factor V of a non-symmetric
  // element (A_e = ... - V^T S^-1 W); equal to H except for the primal schemes
  std::vector<double> Hv;
};
RefElement build_ref_element(int p, double hx, double hy);

// Replace the tables of R by those of the hybridized interior penalty element
// of eq. IPG_H with the given s_f (1 SIPG-H, -1 NIPG-H, 0 IIPG-H):
//   G = Kst - s_f N - N^T,  H = -s_f Hn,  Hv = -Hn,  K = 0,
//   BxT[a][b] = -M_a d_x phi_b(x_a), ByT alike, Cx = Cy = 0,
// with Kst[a][b] = (grad phi_b, grad phi_a), N[a][b] = <phi_b, grad phi_a.n>,
// Hn[a][k] = <psi_k, grad phi_a.n>; E, F, M unchanged.  The element kernels
// then compute S = kappa G + tau E, W = kappa H + tau F, V = kappa Hv + tau F,
// A_e = kappa K + tau I - V^T S^-1 W and q = kappa M^-1 (B^T u - C lambda)
// = -kappa grad u, i.e. exactly the primal scheme.
void make_ipdg_tables(RefElement& R, double sf);

// Basis of the volume space that diagonalises G and E together (eigbasis.cpp):
// Phi^T (G + r0 E) Phi = I, Phi^T G Phi = diag(g), Phi^T E Phi = diag(e),
// P = Phi^T H, Q = Phi^T F ([nv][nt], row i = basis vector i).  r0 >= the
// given value, grown until G + r0 E is positive definite; false if it never is.
struct EigBasis {
  std::vector<double> Phi, g, e, P, Q;   // Phi [nv][nv], column i = phi_i
  double r0 = 0.0;
};
bool build_eig_basis(const RefElement& R, double r0, double hmin, EigBasis& out);

// Non-symmetric volume blocks S(eps) = eps G + S0 (eigbasis.cpp): with
// B = S(eps0), B^-1 G = X Lambda X^-1 in real block form (kind 0: real
// eigenvalue la; kind 1, 2: the two columns xr, xi of a pair la +- i lb), so
// S(eps)^-1 = X (I + (eps - eps0) Lambda)^-1 R with R = X^-1 B^-1, and
//   A_e = eps K + diag - (eps Pv1 + Pv0)^T (I + d Lambda)^-1 (eps Pw1 + Pw0),
// Pv1 = X^T Hv, Pv0 = X^T V0, Pw1 = R H, Pw0 = R W0 ([nv][nt]).
struct EigBasisNS {
  std::vector<double> X, R, Pv1, Pv0, Pw1, Pw0, la, lb;
  std::vector<int> kind;
  double eps0 = 1.0;
};
bool real_eigen_decomposition(const std::vector<double>& M, int n, std::vector<double>& X,
                              std::vector<double>& la, std::vector<double>& lb,
                              std::vector<int>& kind);
bool build_eig_basis_ns(const RefElement& R, const std::vector<double>& S0,
                        const std::vector<double>& W0, const std::vector<double>& V0, double eps0,
                        EigBasisNS& out);
// relative difference of A_e(eps) through the basis against a direct solve
double check_eig_basis_ns(const RefElement& R, const std::vector<double>& S0,
                          const std::vector<double>& W0, const std::vector<double>& V0,
                          const std::vector<double>& adiag, const EigBasisNS& E, double eps);

// tau_e = t kappa_e: move tau into the kappa-proportional tables
// (G += t E, H += t F, Hv += t F, K += t I); the kernels then add no tau.
void fold_kappa_tau(RefElement& R, double t);

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
  T* Rt = nullptr;       // [64][nC]   (-J^T A_BI A_II^-1)^T, the interior part of
                         //            Q_{k-1} transposed; aliases Pi when A is symmetric
  T* r = nullptr;        // level right-hand side   [nd][nEdge]
  T* e = nullptr;        // level correction        [nd][nEdge]
  T* y = nullptr;        // matvec accumulator      [nd][nEdge] (kept zero)
  // point smoothers: 1 / A_aa per dof and the Chebyshev direction
  T* Dpt = nullptr;      // [nd][nEdge]
  T* cd = nullptr;       // [nd][nEdge]
};

struct Level {
  int n = 0;       // macro-elements per side
  int nd = 0;      // trace modes per edge
  int nl = 0;      // 4*nd
  int nsym = 0;    // entries per element operator: nl(nl+1)/2 packed, nl*nl non-symmetric
  int nE = 0, nEdge = 0;
  int m = 1;       // smoothing steps
  int transfer = 0;   // 0 none (coarsest), 1 p-transfer, 2 h-transfer
  LevelData<double> d64;
  LevelData<float> d32;
  __nv_bfloat16* A16 = nullptr;   // BF16 copy of A (finest level, PREC_BF16)
  // Chebyshev smoother: Lambda_max of D^-1 A and the step coefficients
  // [c1_k, c2_k] of d_k = c1_k d_{k-1} + c2_k D^-1 (r - A e), k < m (device)
  double lmax = 0.0;
  double* cheb = nullptr;
};

// ---------------------------------------------------------------------------
// kernel launchers (k_condense.cu, k_mg.cu, k_blas.cu)
// ---------------------------------------------------------------------------
struct RefDevice {     // device copies of RefElement tables (FP64)
  double *M, *G, *E, *H, *F, *K, *BxT, *ByT, *Cx, *Cy, *Ef, *Hv;
  double *Phi, *eg, *ee, *P, *Q;   // EigBasis (symmetric volume blocks only), with the
                                   // element-independent tau applied: ee = tau e, Q = tau Q
};

// kap = exp(log kappa) per element; the element kernels take kap
void launch_kappa(cudaStream_t s, int nE, const double* logk, double* kap);
// returns the autotuned launch shape, threads per element * 16 + elements per
// block; tune_only: only make sure the choice for this (kernel, p) is made
// (times the candidates on a sample)
// symmetric volume blocks S = kappa G + tau E through the EigBasis tables
// (no stored factors): A_e = kappa K + tau I - U^T U,
// U = diag(kappa g + tau e)^-1/2 (kappa P + tau Q)
int launch_condense(cudaStream_t s, const RefDevice& ref, int p, int nE,
                    const double* kap, double tau, double* A, int* err, bool tune_only = false);
void launch_rhs(cudaStream_t s, const RefDevice& ref, int p, int n,
                const double* kap, double tau, const double* f, double* b);
void launch_recover(cudaStream_t s, const RefDevice& ref, int p, int n,
                    const double* kap, double tau, const double* f, const double* lam,
                    double* u, double* q);
// symmetric S by local Cholesky (HDGMG_CONDENSE_FACTOR): packed factor
// Lfac [nv(nv+1)/2][nE] kept for the right-hand side and recovery
int launch_condense_factor(cudaStream_t s, const RefDevice& ref, int p, int nE,
                           const double* kap, double tau, double* A, double* Lfac, int* err,
                           bool tune_only = false);
void launch_rhs_factor(cudaStream_t s, const RefDevice& ref, int p, int n, const double* kap,
                       double tau, const double* Lfac, const double* f, double* b);
void launch_recover_factor(cudaStream_t s, const RefDevice& ref, int p, int n, const double* kap,
                           double tau, const double* Lfac, const double* f, const double* lam,
                           double* u, double* q);

// convection-diffusion element (non-symmetric A_e, full [nt*nt][nE]; LU
// factors of the volume block, full [nv*nv][nE]).  The element-independent
// tables (tau and beta are the same on every element):
//   S0 [nv][nv] = -beta_x BxT - beta_y ByT + sum_f tau_f E_f
//   W0 [nv][nt] = (tau_f - beta.n_f) F,   V0 [nv][nt] = tau_f F
//   adiag [nt]  = tau_f - beta.n_f        (f = the face of trace dof c)
// with tau_f = tau + max(beta.n_f, 0), normals 0: -x, 1: +x, 2: -y, 3: +y.
struct CdTables {
  double *S0 = nullptr, *W0 = nullptr, *V0 = nullptr, *adiag = nullptr;
};
// device copy of an EigBasisNS (X, R [nv][nv]; P* [nv][nt]; la, lb, kind [nv])
struct PencilDevice {
  double *X = nullptr, *R = nullptr, *Pv1 = nullptr, *Pv0 = nullptr, *Pw1 = nullptr,
         *Pw0 = nullptr, *la = nullptr, *lb = nullptr;
  int* kind = nullptr;
  double eps0 = 0.0;
};
// non-symmetric S through the pencil basis (no stored factor)
int launch_condense_cdeig(cudaStream_t s, const RefDevice& ref, const CdTables& cd,
                          const PencilDevice& pb, int p, int nE, const double* kap, double* A,
                          int* err, bool tune_only = false);
void launch_rhs_cdeig(cudaStream_t s, const RefDevice& ref, const PencilDevice& pb, int p, int n,
                      const double* kap, const double* f, double* b);
void launch_recover_cdeig(cudaStream_t s, const RefDevice& ref, const CdTables& cd,
                          const PencilDevice& pb, int p, int n, const double* kap, const double* f,
                          const double* lam, double* u, double* q);
void build_cd_tables(const RefElement& R, double tau, double bx, double by,
                     std::vector<double>& S0, std::vector<double>& W0, std::vector<double>& V0,
                     std::vector<double>& adiag);
int launch_condense_cd(cudaStream_t s, const RefDevice& ref, const CdTables& cd, int p, int nE,
                       const double* kap, double* A, double* LU, int* err, bool tune_only = false);
void launch_rhs_cd(cudaStream_t s, const RefDevice& ref, const CdTables& cd, int p, int n,
                   const double* kap, const double* LU, const double* f, double* b);
void launch_recover_cd(cudaStream_t s, const RefDevice& ref, const CdTables& cd, int p, int n,
                       const double* kap, const double* LU, const double* f, const double* lam,
                       double* u, double* q);

// adjoint: per-element derivative contraction (K13), adjoint source, misfit
void launch_grad_contract(cudaStream_t s, const RefDevice& ref, int p, int n, const double* kap,
                          const double* lam, const double* u, const double* mu, const double* w,
                          double* dlogk, double* df);
void launch_adjoint_source(cudaStream_t s, const RefDevice& ref, int nv, int nE, const double* g,
                           double* fadj);
void launch_misfit(cudaStream_t s, const RefDevice& ref, int nv, int nE, const double* u,
                   const double* uobs, double* d, double* gu);

// ns: operators stored non-symmetric (full row-major) instead of packed.
// xadd (nullable): the P1 correction of the next level, added to modes 0
// and 1 of x (matvec) or of e (block-Jacobi update) on the fly -- the
// p-prolongation J_N fused into the first post-smoothing step.
// k: right-hand sides of a blocked solve, vectors [k][...] contiguous per
// right-hand side (every V-cycle launcher below takes it, default 1)
template <typename T>
void launch_matvec(cudaStream_t s, int n, int nd, bool ns, const T* A, const T* x, T* y, T alpha,
                   const T* xadd = nullptr, int k = 1);
// per-ND instantiations (k_edge_inst.cu, one translation unit per type and ND)
template <typename T, int ND, bool NS>
void launch_matvec_nd(cudaStream_t s, int n, const T* A, const T* x, T* y, T alpha, const T* xadd,
                      int k);
template <typename T, int ND, bool NS>
void launch_bj_blocks_nd(cudaStream_t s, int n, const T* A, T* Dinv, int* err);
// the PCG iteration's direction update, FP64 matvec and p.Ap in one launch
// (symmetric storage; z32 or z64 is the preconditioned residual, the other
// null); partial holds kDotBlocks doubles
void launch_cg_matvec(cudaStream_t s, int n, int nd, const double* A, const float* z32,
                      const double* z64, const double* p, double* Ap, double* scal,
                      double* partial, unsigned* counter);
template <int ND>
void launch_cg_matvec_nd(cudaStream_t s, int n, const double* A, const float* z32,
                         const double* z64, const double* p, double* Ap, double* scal,
                         double* partial, unsigned* counter);
// matrix-free FP32 finest-level apply through the eigenbasis (k_mf.cuh;
// symmetric basis route, nd <= 7): tables is a host array of
// mf_table_size(nd) floats (K [nt][nt], P [nv][nt], tau Q, g [nv], tau e,
// tau), kap the FP64 element coefficients
constexpr int mf_table_size(int nd) { return 16 * nd * nd + 8 * nd * nd * nd + 2 * nd * nd + 1; }
constexpr int kMfMaxNd = 7;
void launch_matvec_mf(cudaStream_t s, int n, int nd, const float* tables, const double* kap,
                      const float* x, float* y, float alpha, const float* xadd, int k);
template <int ND>
void launch_matvec_mf_nd(cudaStream_t s, int n, const float* tables, const double* kap,
                         const float* x, float* y, float alpha, const float* xadd, int k);
// the finest FP32 level's last post-smoothing step with r64 . z (z the new
// e) and the beta recurrence of the FP64 PCG (symmetric storage, one
// right-hand side); partial holds kDotBlocks doubles
void launch_bj_update_dot(cudaStream_t s, int n, int nd, const float* Dinv, const float* r,
                          float* y, float* e, float omega, const float* xadd, const double* r64,
                          double* scal, double* partial, unsigned* counter);
template <int ND>
void launch_bj_update_dot_nd(cudaStream_t s, int n, const float* Dinv, const float* r, float* y,
                             float* e, float omega, const float* xadd, const double* r64,
                             double* scal, double* partial, unsigned* counter);
// x += alpha p+, r -= alpha Ap, Ap = 0, p = p+ (= fma(beta, p, z)), r.r and
// the loop test of cg_update_test (r32: FP32 copy of r, nullable)
void launch_cg_update_dir_test(cudaStream_t s, int64_t len, double* scal, double* x, double* r,
                               double* p, double* Ap, const float* z32, const double* z64,
                               double* partial, unsigned* counter, cudaGraphConditionalHandle h,
                               int* it, int max_it, double tol2, float* r32);
template <typename T, int ND, bool NS>
void launch_bj_update_nd(cudaStream_t s, int n, const T* Dinv, const T* r, T* y, T* e, T omega,
                         int first, const T* xadd, int k);
// y += alpha A x with A stored in BF16, x, y and the accumulation in FP32
void launch_matvec_bf16(cudaStream_t s, int n, int nd, bool ns, const __nv_bfloat16* A,
                        const float* x, float* y, float alpha, const float* xadd = nullptr,
                        int k = 1);
template <int ND, bool NS>
void launch_matvec_bf16_nd(cudaStream_t s, int n, const __nv_bfloat16* A, const float* x, float* y,
                           float alpha, const float* xadd, int k);
void launch_to_bf16(cudaStream_t s, int64_t len, const double* in, __nv_bfloat16* out);
template <typename T>
void launch_bj_blocks(cudaStream_t s, int n, int nd, bool ns, const T* A, T* Dinv, int* err);
template <typename T>
void launch_bj_update(cudaStream_t s, int n, int nd, bool ns, const T* Dinv, const T* r, T* y,
                      T* e, T omega, int first, const T* xadd = nullptr, int k = 1);
// p-restriction fused into the first sweep of the P1 level below the
// p-level: r1 = (r0 - y0) on modes 0, 1 (written), y0 := 0 on all nd0
// modes, e1 = omega D1^-1 r1
template <typename T>
void launch_bj_first_restrict_p(cudaStream_t s, int n, int nd0, bool ns, const T* Dinv1,
                                const T* r0, T* y0, T* r1, T* e1, T omega, int k = 1);
template <typename T>
void launch_pcoarsen(cudaStream_t s, int nE, int ndf, bool ns, const T* Af, T* Ac);
// ns: also writes Rt = Z^T J with Z = -A_BI A_II^-1 (the restriction block);
// symmetric operators use Rt = Pi
template <typename T>
void launch_agglomerate(cudaStream_t s, int nc, bool ns, const T* Af, T* Ac, T* AIIinv, T* Y,
                        T* Pi, T* Rt, int* err);
template <typename T>
void launch_local_correction(cudaStream_t s, int nc, bool ns, const T* AIIinv, const T* Y,
                             const T* r, T* e, int k = 1);
template <typename T>
void launch_restrict_h(cudaStream_t s, int nc, const T* Pi, const T* r, T* y, T* rc, int k = 1);
// P1 level, one thread per edge gathering both elements' rows (no atomics):
// sweep: out = x + omega D^-1 (r - A x); else out = A x.  x != out.
template <typename T>
void launch_edge_p1(cudaStream_t s, int n, bool ns, const T* A, const T* Dinv, const T* r, const T* x,
                    T* out, T omega, bool sweep, int k = 1);
template <typename T>
void launch_prolong_h(cudaStream_t s, int nc, const T* Pi, const T* ec, T* e, T* y, int k = 1);
template <typename T>
void launch_restrict_p(cudaStream_t s, int n, int nd, const T* r, T* y, T* rc);
template <typename T>
void launch_prolong_p(cudaStream_t s, int n, int nd, const T* ec, T* e);

// fused V-cycle over the P1 tail of the hierarchy (one thread block)
constexpr int kMaxTail = 8;
constexpr int kTailMaxSmem = 224 * 1024;
template <typename T>
struct TailLevel {
  int n = 0, m = 1, nEdge = 0;
  // shared-memory offsets (T units) of [r|e|y] and of the staged operators
  int voff = 0, a_off = 0, dinv_off = 0, aii_off = 0, y_off = 0, pi_off = 0, rt_off = 0;
  int staged = 0;              // operators copied to shared memory (else read from L2)
  const T* A = nullptr;
  const T* Dinv = nullptr;
  const T* AIIinv = nullptr;
  const T* Y = nullptr;
  const T* Pi = nullptr;
  const T* Rt = nullptr;
};
template <typename T>
struct TailParams {
  int nlev = 0;
  TailLevel<T> lv[kMaxTail];
  const T* r_in = nullptr;      // right-hand side of the first tail level (global)
  T* e_out = nullptr;           // its correction (global)
  const double* Ainv = nullptr; // coarsest dense inverse (FP64)
  const int* fidx = nullptr;    // coarsest edge -> free edge number (-1: Dirichlet)
  const int* fedge = nullptr;   // free edge number -> coarsest edge
  int nf = 0;
  T omega = T(1);
  int lc = 0;
  int ns = 0;                   // non-symmetric (full) operators
  int ainv_off = 0, w_off = 0;  // byte offsets of the staged inverse (-1: read from global)
                                // and of the workspace
  int smem_bytes = 0;
};
template <typename T>
void launch_vcycle_tail(cudaStream_t s, const TailParams<T>& P);

// fused V-cycle over the P1 tail on one thread-block cluster (k_ctail.cu)
template <typename T>
struct CTailLevel {
  int n = 0, m = 1, nEdge = 0;
  int echunk = 0, edchunk = 0, cchunk = 0;   // elements / edges / macro-elements per CTA
  // shared-memory offsets (T units): vectors [r|e|y] x [2][edchunk]; staged
  // operators ([stride][chunk]) or -1 when they are read from global memory
  int off_v = 0, off_A = -1, off_D = -1, off_AII = -1, off_Y = -1, off_Pi = -1;
  const T* A = nullptr;
  const T* Dinv = nullptr;
  const T* AIIinv = nullptr;
  const T* Y = nullptr;
  const T* Pi = nullptr;
};
template <typename T>
struct CTailParams {
  int nlev = 0, cl = 0;
  CTailLevel<T> lv[kMaxTail];
  const T* r_in = nullptr;
  T* e_out = nullptr;
  const double* Ainv = nullptr;
  const int* fidx = nullptr;
  const int* fedge = nullptr;
  int nf = 0;
  int w_off = 0;                // byte offset of the coarse-solve workspace
  T omega = T(1);
  int lc = 0;
  double Jc[2][2][2] = {};
  int smem_bytes = 0;
};
template <typename T>
int ctail_max_clusters(int cluster, int smem_bytes);
template <typename T>
void launch_ctail(cudaStream_t s, const CTailParams<T>& P);

// Persistent V-cycle over the P1 levels (k_mg.cu): one cooperative launch
// runs Algorithm 1 from the first P1 level to the coarsest and back, every
// step a grid-stride loop over its work items, the steps separated by grid
// barriers (bounded waits) instead of kernel launches.  Levels from `tail`
// on run on block 0 alone (block barriers), while the other blocks wait at
// one grid barrier.  Vectors stay in global memory (L2-resident).
constexpr int kMaxPLev = 14;
// floor(x / d) for 0 <= x < 2^31 by a multiply-high and a shift (the
// round-up method of Granlund and Montgomery): s = ceil(log2 d),
// m = floor(2^(32+s) / d) + 1 - 2^32, floor(x / d) = (mulhi(x, m) + x) >> s.
// m / 2^(32+s) exceeds 1/d by less than 2^-(32+s), so for x < 2^31 the
// error stays below 2^-(s+1) <= 1/(2d) and never reaches the next integer.
struct FastDiv {
  unsigned m = 1, s = 0;
};
inline FastDiv make_fastdiv(int d) {
  FastDiv f;
  unsigned s = 0;
  while ((1ull << s) < (unsigned long long)d) ++s;
  f.s = s;
  f.m = (unsigned)(((1ull << (32 + s)) / (unsigned long long)d) + 1ull - (1ull << 32));
  return f;
}
// Sizes of a P1 level with n macro-elements per side and, when n is even, of
// the next coarser level nc = n / 2, with the divisors the work items need.
struct P1Geom {
  int n = 0, nE = 0, nvert = 0, nedge = 0;
  int nc = 0, nC = 0, nvc = 0, nedc = 0;
  FastDiv dn, dn1, dnc, dnc1, dnC;
  // item counts of the cycle's steps (blocked solves: item j = rhs * count + t)
  FastDiv dne, dlc, dc1, dc2, dpro;   // nedge, 8 nC, nedc, 2 nedc, 8 nC + 2 nedc
};
inline P1Geom make_p1geom(int n) {
  P1Geom g;
  g.n = n;
  g.nE = n * n;
  g.nvert = n * (n + 1);
  g.nedge = 2 * n * (n + 1);
  g.dn = make_fastdiv(n);
  g.dn1 = make_fastdiv(n + 1);
  g.nc = n / 2;
  if (g.nc > 0) {
    g.nC = g.nc * g.nc;
    g.nvc = g.nc * (g.nc + 1);
    g.nedc = 2 * g.nc * (g.nc + 1);
    g.dnc = make_fastdiv(g.nc);
    g.dnc1 = make_fastdiv(g.nc + 1);
    g.dnC = make_fastdiv(g.nC);
    g.dlc = make_fastdiv(8 * g.nC);
    g.dc1 = make_fastdiv(g.nedc);
    g.dc2 = make_fastdiv(2 * g.nedc);
    g.dpro = make_fastdiv(8 * g.nC + 2 * g.nedc);
  }
  g.dne = make_fastdiv(g.nedge);
  return g;
}
template <typename T>
struct PLevel {
  int n = 0, m = 1;
  P1Geom g;
  const T* A = nullptr;
  const T* Dinv = nullptr;
  const T* AIIinv = nullptr;
  const T* Y = nullptr;
  const T* Pi = nullptr;
  const T* Rt = nullptr;        // restriction block (= Pi when symmetric)
  T* r = nullptr;
  T* e = nullptr;
  T* y = nullptr;
  // levels of the block-0 tail: byte offsets of their shared-memory copies
  // (operators, and the vectors [r | e | y]); -1 when not staged
  int so_A = -1, so_D = -1, so_AII = -1, so_Y = -1, so_Pi = -1, so_Rt = -1, so_v = -1;
};
template <typename T>
struct PCycleParams {
  int nlev = 0;                 // lv[0] first P1 level ... lv[nlev-1] coarsest
  int tail = 0;                 // first level run by block 0 alone (nlev: none)
  PLevel<T> lv[kMaxPLev];
  // pending p-restriction J_N^T (r0 - y0) of the level above lv[0] (r0 null:
  // lv[0].r is the given right-hand side)
  const T* rp_r0 = nullptr;
  T* rp_y0 = nullptr;
  int rp_nd0 = 0;
  const double* Ainv = nullptr; // coarsest dense inverse (FP64)
  const int* fidx = nullptr;
  const int* fedge = nullptr;
  int nf = 0;
  FastDiv dco;                  // n_edges(coarsest) + nf: items of the coarse step
  int nrhs = 1;                 // right-hand sides of a blocked solve (vectors [k][...])
  T omega = T(1);
  int lc = 0;
  int ns = 0;
  unsigned long long* bar = nullptr;   // grid barrier: monotonic arrival count
  int* err = nullptr;           // bit 0: a barrier wait expired, bit 1: the wait for the
                                // tail's bulk copies expired (both HDGMG_ETIMEOUT)
  unsigned long long wait_ns = 1000000000ull;   // limit of one barrier wait
  int withhold = 0;             // testing: no block arrives at the first barrier
  // profiling: (global timer ns, step tag) pairs written by block 0 after each
  // barrier, at most trace_cap pairs (null: no trace)
  unsigned long long* trace = nullptr;
  int trace_cap = 0;
  // dynamic shared memory: the block-0 tail's staged levels (staged = 1), the
  // coarsest inverse at so_Ainv and the coarse workspace at so_w (bytes)
  int staged = 0;
  int stage_bytes = 0;          // bytes of the staged operators and inverse (bulk copies)
  int so_Ainv = -1, so_w = 0;
  int smem_bytes = 0;
};
template <typename T>
int pcycle_max_blocks(int smem_bytes);   // co-resident blocks of the kernel on this device
template <typename T>
int pcycle_threads();
template <typename T>
cudaError_t launch_pcycle(cudaStream_t s, const PCycleParams<T>& P, int blocks);

// coarsest level: dense FP64 Cholesky of the interior operator
template <typename T>
void launch_coarse_assemble(cudaStream_t s, int n, bool ns, const T* A, const int* freeidx, int nf,
                            double* dense);
// in-place Gauss-Jordan inverse of a dense matrix with positive-definite
// symmetric part (one block, global memory): Ainv = M^-1
void launch_coarse_gj(cudaStream_t s, int nf, double* M, double* Ainv, int* err);
void launch_coarse_factor(cudaStream_t s, int nf, double* dense, int* err);
void launch_coarse_inverse(cudaStream_t s, int nf, const double* L, double* Li, double* Ainv);
// assemble + invert in one block when A_1 fits in shared memory; false if not
template <typename T>
bool launch_coarse_setup_smem(cudaStream_t s, int n, bool ns, const T* A, const int* freeidx,
                              int nf, double* Ainv, int* err);
template <typename T>
void launch_coarse_solve(cudaStream_t s, int n, const int* freeidx, const int* fedge, int nf,
                         const double* Ainv, const T* r, T* e, int k = 1);

// vector kernels (FP64 unless templated)
template <typename T>
void launch_dot(cudaStream_t s, int64_t len, const T* a, const T* b, double* partial,
                double* out);
template <typename T>
void launch_mask(cudaStream_t s, int n, int nd, T* x);   // zero Dirichlet entries
template <typename T>
void launch_unpack(cudaStream_t s, int nl, int nE, bool ns, const T* Ap, double* full);
template <typename A, typename B>
void launch_convert(cudaStream_t s, int64_t len, const A* in, B* out);
template <typename T>
void launch_cg_update(cudaStream_t s, int64_t len, const double* scal, T* x, T* r, const T* p,
                      const T* Ap);
template <typename T>
void launch_cg_direction(cudaStream_t s, int64_t len, const double* scal, const T* z, T* p);
// fused PCG kernels (scal layout: 0 rz, 1 pAp, 2 alpha, 3 rz_new, 4 beta,
// 5 rr, 6 reference norm^2); counter: a zeroed unsigned reset by the kernel
// k > 1: blocked over k right-hand sides (vectors [k][len], scalars
// scal[8 j ...], partials [k][blocks], counters [k])
template <typename T>
void launch_dot_fused(cudaStream_t s, int64_t len, const T* a, const T* b, double* partial,
                      unsigned* counter, double* scal, int mode, int k = 1);
template <typename T>
void launch_cg_direction_zero(cudaStream_t s, int64_t len, const double* scal, const T* z, T* p,
                              T* Ap, int k = 1);
// blocked PCG update and loop test (see k_mg.cu): counters [k + 1]
template <typename T>
void launch_cg_update_test_block(cudaStream_t s, int64_t len, int k, double* scal, T* x, T* r,
                                 const T* p, const T* Ap, double* partial, unsigned* counter,
                                 cudaGraphConditionalHandle h, int* it, int max_it, double tol2);
// r32 (nullable): also receives the updated r rounded to FP32
template <typename T>
void launch_cg_update_test(cudaStream_t s, int64_t len, double* scal, T* x, T* r, const T* p,
                           const T* Ap, double* partial, unsigned* counter,
                           cudaGraphConditionalHandle h, int* it, int max_it, double tol2,
                           float* r32);
// FP64 CG vectors with the FP32 V-cycle output z read directly
void launch_dot_fused_mixed(cudaStream_t s, int64_t len, const double* a, const float* b,
                            double* partial, unsigned* counter, double* scal, int mode);
void launch_cg_direction_zero_mixed(cudaStream_t s, int64_t len, const double* scal, const float* z,
                                    double* p, double* Ap);
// FP64 -> FP32 with 1/sqrt(*scale), and y += sqrt(*scale) x (FP32 -> FP64)
// k right-hand sides, the scale of j at scale[j * sstride]
void launch_scale_to_f32(cudaStream_t s, int64_t len, const double* in, const double* scale,
                         float* out, int k = 1, int sstride = 0);
void launch_add_f32(cudaStream_t s, int64_t len, const double* scale, const float* x, double* y,
                    int k = 1, int sstride = 0);
void launch_cg_scalars(cudaStream_t s, double* scal, int stage);
void launch_axpby(cudaStream_t s, int64_t len, double a, const double* x, double b, double* y);
void launch_copy_boundary(cudaStream_t s, int n, int nd, const double* gD, double* lam);

// flexible GMRES (k_krylov.cu); jp: device Arnoldi index
int gm_partial_blocks();
void launch_gm_select(cudaStream_t s, int64_t len, const double* base, const int* jp, int shift,
                      double* out);
void launch_gm_store(cudaStream_t s, int64_t len, const double* in, double* base, const int* jp,
                     int shift);
void launch_gm_orthogonalize(cudaStream_t s, int64_t len, const double* V, const int* jp,
                             double* w, double* partial, int ldh, double* H, double* h,
                             int max_k, int accumulate);
void launch_gm_normalize(cudaStream_t s, int64_t len, const double* w, const double* nrm2, double* V,
                         const int* jp);
void launch_gm_givens(cudaStream_t s, double* H, int ldh, double* cs, double* sn, double* g, int* jp,
                      int m, const double* tolp, const double* nrm2, cudaGraphConditionalHandle hdl,
                      int* total, int max_total);
void launch_gm_update(cudaStream_t s, int64_t len, const double* Z, int nk, const double* y,
                      double* x);

// condensation autotuning of one context, synchronously (hdgmg_api.cu)
hdgmg_status tune_condensation(hdgmg_ctx* c, const double* log_kappa);
bool condensation_kind(const hdgmg_ctx* c, int* p, int* ns);

// point smoothers (k_mg.cu); generic in nd, element operators packed or full
template <typename T>
void launch_point_diag(cudaStream_t s, int n, int nd, bool ns, const T* A, T* Dpt);
// e = omega Dpt r (first) or e += omega Dpt (r - y), y := 0
template <typename T>
void launch_pj_update(cudaStream_t s, int n, int nd, const T* Dpt, const T* r, T* y, T* e, T omega,
                      int first);
// d = c1_k d + c2_k Dpt (r - y) (first_d: d = c2_k Dpt (r - y)), e += d
// (first_e: e = d; y is then not read), y := 0
template <typename T>
void launch_cheb_update(cudaStream_t s, int n, int nd, const T* Dpt, const T* r, T* y, T* e, T* d,
                        const double* coef, int k, int first_e, int first_d);
// one colour of a point Gauss-Seidel sweep, in place on e
template <typename T>
void launch_gs_colour(cudaStream_t s, int n, int nd, bool ns, const T* A, const T* Dpt, const T* r,
                      T* e, int colour, int backward);
// power iteration helpers: x = start vector; y *= Dpt; x = y / sqrt(*nrm2)
template <typename T>
void launch_power_start(cudaStream_t s, int n, int nd, T* x);
template <typename T>
void launch_scale_by(cudaStream_t s, int64_t len, const T* Dpt, T* y);
template <typename T>
void launch_normalize(cudaStream_t s, int64_t len, const T* y, const double* nrm2, T* x);

// set the calling thread's hdgmg_last_error() message
void set_last_error(const std::string& msg);

// host-side count of kernel launches issued by the library (all threads)
void note_launch();
long long launch_count();

constexpr int kDotBlocks = 608;   // 4 x 152 SMs; fixed for a deterministic sum

}  // namespace hdgmg
