// Host: a basis that diagonalises the two reference matrices of the volume
// block at once.
//
// On a uniform mesh the volume block of every element is S = kappa G + tau E
// with the same G and E (Sec. 2; kappa and tau are scalars per element).  For
// B = G + r0 E symmetric positive definite, Cholesky B = L L^T and the
// symmetric eigen-decomposition L^-1 G L^-T = Z diag(lambda) Z^T give
// Phi = L^-T Z with
//   Phi^T B Phi = I,  Phi^T G Phi = diag(g),  Phi^T E Phi = diag(e),
// so S = Phi^-T diag(kappa g + tau e) Phi^-1 for every kappa and tau, and S
// is positive definite exactly when every s_i = kappa g_i + tau e_i > 0.
// The eigen-decomposition is the cyclic Jacobi method (rotations chosen to
// annihilate one off-diagonal pair at a time, sweeps until the off-diagonal
// part is at rounding level; Golub & Van Loan, Matrix Computations, 4th ed.,
// Sec. 8.5).
#include <cmath>

#include "internal.h"

namespace hdgmg {
namespace {

// in-place Cholesky of the n x n row-major matrix (lower triangle); false if
// a pivot is not positive
bool cholesky(std::vector<double>& A, int n) {
  for (int j = 0; j < n; ++j) {
    double d = A[j * n + j];
    for (int k = 0; k < j; ++k) d -= A[j * n + k] * A[j * n + k];
    if (!(d > 0.0) || !std::isfinite(d)) return false;
    d = std::sqrt(d);
    A[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double s = A[i * n + j];
      for (int k = 0; k < j; ++k) s -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = s / d;
    }
  }
  return true;
}

// cyclic Jacobi on the symmetric C (n x n): C -> diag, Z accumulates the
// rotations (C_in = Z diag Z^T)
void jacobi_eigen(std::vector<double>& C, std::vector<double>& Z, int n) {
  Z.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Z[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i) {
      diag += C[i * n + i] * C[i * n + i];
      for (int j = i + 1; j < n; ++j) off += C[i * n + j] * C[i * n + j];
    }
    if (off <= 1e-32 * diag) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = C[p * n + q];
        const double app = C[p * n + p], aqq = C[q * n + q];
        if (std::fabs(apq) <= 1e-18 * (std::fabs(app) + std::fabs(aqq)) || std::fabs(apq) < 1e-300) {
          C[p * n + q] = C[q * n + p] = 0.0;     // negligible against the diagonal
          continue;
        }
        // rotation angle: tan(theta) = t solves t^2 + 2 t zeta - 1 = 0,
        // zeta = (aqq - app) / (2 apq), smaller root for stability
        const double zeta = (aqq - app) / (2.0 * apq);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = t * cs;
        for (int k = 0; k < n; ++k) {        // columns p, q
          const double ckp = C[k * n + p], ckq = C[k * n + q];
          C[k * n + p] = cs * ckp - sn * ckq;
          C[k * n + q] = sn * ckp + cs * ckq;
        }
        for (int k = 0; k < n; ++k) {        // rows p, q
          const double cpk = C[p * n + k], cqk = C[q * n + k];
          C[p * n + k] = cs * cpk - sn * cqk;
          C[q * n + k] = sn * cpk + cs * cqk;
        }
        C[p * n + q] = C[q * n + p] = 0.0;
        for (int k = 0; k < n; ++k) {
          const double zkp = Z[k * n + p], zkq = Z[k * n + q];
          Z[k * n + p] = cs * zkp - sn * zkq;
          Z[k * n + q] = sn * zkp + cs * zkq;
        }
      }
  }
}

}  // namespace

bool build_eig_basis(const RefElement& R, double r0, double hmin, EigBasis& out) {
  const int nv = R.nv, nt = R.nt;
  std::vector<double> G(nv * nv), E(nv * nv);
  for (int i = 0; i < nv; ++i)
    for (int j = 0; j < nv; ++j) {
      G[i * nv + j] = 0.5 * (R.G[i * nv + j] + R.G[j * nv + i]);
      E[i * nv + j] = 0.5 * (R.E[i * nv + j] + R.E[j * nv + i]);
    }
  // B = G + r0 E must be positive definite; grow r0 until it is
  std::vector<double> L;
  bool ok = false;
  for (int attempt = 0; attempt < 64 && !ok; ++attempt) {
    L.resize((size_t)nv * nv);
    for (int t = 0; t < nv * nv; ++t) L[t] = G[t] + r0 * E[t];
    ok = cholesky(L, nv);
    if (!ok) r0 = r0 > 0.0 ? 2.0 * r0 : 1.0 / hmin;
  }
  if (!ok) return false;
  // C = L^-1 G L^-T: X = L^-1 G (forward substitution per column), C = X L^-T
  std::vector<double> X(G), C((size_t)nv * nv);
  for (int col = 0; col < nv; ++col)
    for (int i = 0; i < nv; ++i) {
      double s = X[i * nv + col];
      for (int k = 0; k < i; ++k) s -= L[i * nv + k] * X[k * nv + col];
      X[i * nv + col] = s / L[i * nv + i];
    }
  for (int row = 0; row < nv; ++row)        // C[row][:] = L^-1 X[row][:]^T
    for (int i = 0; i < nv; ++i) {
      double s = X[row * nv + i];
      for (int k = 0; k < i; ++k) s -= L[i * nv + k] * C[row * nv + k];
      C[row * nv + i] = s / L[i * nv + i];
    }
  for (int i = 0; i < nv; ++i)
    for (int j = i + 1; j < nv; ++j) C[i * nv + j] = C[j * nv + i] = 0.5 * (C[i * nv + j] + C[j * nv + i]);
  std::vector<double> Z;
  jacobi_eigen(C, Z, nv);
  // Phi = L^-T Z (back substitution per column)
  out.Phi.assign((size_t)nv * nv, 0.0);
  for (int col = 0; col < nv; ++col)
    for (int i = nv - 1; i >= 0; --i) {
      double s = Z[i * nv + col];
      for (int k = i + 1; k < nv; ++k) s -= L[k * nv + i] * out.Phi[k * nv + col];
      out.Phi[i * nv + col] = s / L[i * nv + i];
    }
  // g_i = phi_i^T G phi_i, e_i = phi_i^T E phi_i; P = Phi^T H, Q = Phi^T F
  out.g.assign(nv, 0.0);
  out.e.assign(nv, 0.0);
  for (int i = 0; i < nv; ++i) {
    double sg = 0.0, se = 0.0;
    for (int a = 0; a < nv; ++a) {
      double ga = 0.0, ea = 0.0;
      for (int b = 0; b < nv; ++b) {
        ga += G[a * nv + b] * out.Phi[b * nv + i];
        ea += E[a * nv + b] * out.Phi[b * nv + i];
      }
      sg += out.Phi[a * nv + i] * ga;
      se += out.Phi[a * nv + i] * ea;
    }
    out.g[i] = sg;
    out.e[i] = se;
  }
  out.P.assign((size_t)nv * nt, 0.0);
  out.Q.assign((size_t)nv * nt, 0.0);
  for (int i = 0; i < nv; ++i)
    for (int c = 0; c < nt; ++c) {
      double sp = 0.0, sq = 0.0;
      for (int a = 0; a < nv; ++a) {
        sp += out.Phi[a * nv + i] * R.H[a * nt + c];
        sq += out.Phi[a * nv + i] * R.F[a * nt + c];
      }
      out.P[i * nt + c] = sp;
      out.Q[i * nt + c] = sq;
    }
  out.r0 = r0;
  return true;
}

}  // namespace hdgmg
