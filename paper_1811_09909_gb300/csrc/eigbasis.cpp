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

// ---------------------------------------------------------------------------
// Non-symmetric volume blocks S(eps) = eps G + S0 (convection-diffusion,
// NIPG-H, IIPG-H): with B = S(eps0) and M = B^-1 G,
//   S(eps) = B (I + (eps - eps0) M),
// so an eigen-decomposition M = X Lambda X^-1, kept real (a complex pair
// a +- ib with eigenvector xr +- i xi becomes the columns xr, xi and the block
// [[a, b], [-b, a]]), gives S(eps)^-1 = X (I + d Lambda)^-1 X^-1 B^-1 with
// d = eps - eps0 and a block-diagonal (I + d Lambda).
// Eigenvalues: reduction to upper Hessenberg form by Householder reflections,
// then Francis' implicit double-shift QR iteration with deflation (Golub & Van
// Loan, Matrix Computations, 4th ed., Sec. 7.4-7.5).  Eigenvectors: inverse
// iteration with each eigenvalue on M itself in complex arithmetic (complex
// LU with partial pivoting), vectors of a repeated eigenvalue kept independent
// by orthogonalising against the earlier ones.  The caller checks the whole
// decomposition against direct solves before using it.
#include <complex>
#include <random>

namespace hdgmg {
namespace {

using cplx = std::complex<double>;

void to_hessenberg(std::vector<double>& A, int n) {
  std::vector<double> v(n);
  for (int k = 0; k + 2 < n; ++k) {
    double alpha = 0.0;
    for (int i = k + 1; i < n; ++i) alpha += A[i * n + k] * A[i * n + k];
    alpha = std::sqrt(alpha);
    if (alpha == 0.0) continue;
    if (A[(k + 1) * n + k] > 0) alpha = -alpha;
    // v = x - alpha e1 over rows k+1..n-1
    for (int i = 0; i < n; ++i) v[i] = 0.0;
    v[k + 1] = A[(k + 1) * n + k] - alpha;
    for (int i = k + 2; i < n; ++i) v[i] = A[i * n + k];
    double vv = 0.0;
    for (int i = k + 1; i < n; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    // A <- (I - 2 v v^T / vv) A (I - 2 v v^T / vv)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int i = k + 1; i < n; ++i) s += v[i] * A[i * n + j];
      s *= 2.0 / vv;
      for (int i = k + 1; i < n; ++i) A[i * n + j] -= s * v[i];
    }
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int j = k + 1; j < n; ++j) s += A[i * n + j] * v[j];
      s *= 2.0 / vv;
      for (int j = k + 1; j < n; ++j) A[i * n + j] -= s * v[j];
    }
    for (int i = k + 2; i < n; ++i) A[i * n + k] = 0.0;
  }
}

// eigenvalues of the upper Hessenberg H (destroyed); false if the iteration
// does not converge
bool hessenberg_eigenvalues(std::vector<double>& H, int n, std::vector<cplx>& ev) {
  ev.clear();
  double anorm = 0.0;
  for (double x : H) anorm = std::max(anorm, std::fabs(x));
  if (anorm == 0.0) anorm = 1.0;
  const double eps = 2.2e-16;
  int hi = n - 1, iter = 0;
  auto h = [&](int i, int j) -> double& { return H[i * n + j]; };
  while (hi >= 0) {
    int lo = hi;
    while (lo > 0) {
      double s = std::fabs(h(lo - 1, lo - 1)) + std::fabs(h(lo, lo));
      if (s == 0.0) s = anorm;
      if (std::fabs(h(lo, lo - 1)) <= eps * s) {
        h(lo, lo - 1) = 0.0;
        break;
      }
      --lo;
    }
    if (lo == hi) {                               // 1 x 1 block
      ev.push_back(cplx(h(hi, hi), 0.0));
      --hi;
      iter = 0;
      continue;
    }
    if (lo == hi - 1) {                           // 2 x 2 block
      const double a = h(hi - 1, hi - 1), b = h(hi - 1, hi), c = h(hi, hi - 1), d = h(hi, hi);
      const double tr = a + d, det = a * d - b * c;
      const double disc = 0.25 * tr * tr - det;
      if (disc >= 0.0) {
        const double sq = std::sqrt(disc);
        const double l1 = 0.5 * tr + (tr >= 0 ? sq : -sq);
        const double l2 = l1 != 0.0 ? det / l1 : 0.5 * tr - (tr >= 0 ? sq : -sq);
        ev.push_back(cplx(l1, 0.0));
        ev.push_back(cplx(l2, 0.0));
      } else {
        const double sq = std::sqrt(-disc);
        ev.push_back(cplx(0.5 * tr, sq));
        ev.push_back(cplx(0.5 * tr, -sq));
      }
      hi -= 2;
      iter = 0;
      continue;
    }
    if (++iter > 60 * n) return false;
    // shifts: the eigenvalues of the trailing 2 x 2 (trace s, determinant t),
    // or an ad hoc pair every tenth iteration to break cycles
    double s = h(hi - 1, hi - 1) + h(hi, hi);
    double t = h(hi - 1, hi - 1) * h(hi, hi) - h(hi - 1, hi) * h(hi, hi - 1);
    if (iter % 10 == 0) {
      const double w = std::fabs(h(hi, hi - 1)) + std::fabs(h(hi - 1, hi - 2));
      s = 1.5 * w;
      t = w * w;
    }
    // first column of (H - s1 I)(H - s2 I) restricted to rows lo..lo+2
    double x = h(lo, lo) * h(lo, lo) + h(lo, lo + 1) * h(lo + 1, lo) - s * h(lo, lo) + t;
    double y = h(lo + 1, lo) * (h(lo, lo) + h(lo + 1, lo + 1) - s);
    double z = h(lo + 2, lo + 1) * h(lo + 1, lo);
    for (int k = lo; k <= hi - 1; ++k) {
      const int m = (k < hi - 1) ? 3 : 2;         // reflector size
      double v0 = x, v1 = y, v2 = (m == 3) ? z : 0.0;
      double alpha = std::sqrt(v0 * v0 + v1 * v1 + v2 * v2);
      if (alpha != 0.0) {
        if (v0 > 0) alpha = -alpha;
        v0 -= alpha;
        const double vv = v0 * v0 + v1 * v1 + v2 * v2;
        if (vv != 0.0) {
          const double f = 2.0 / vv;
          const int c0 = std::max(lo, k - 1);
          for (int j = c0; j <= hi; ++j) {          // rows k..k+m-1
            double sum = v0 * h(k, j) + v1 * h(k + 1, j) + (m == 3 ? v2 * h(k + 2, j) : 0.0);
            sum *= f;
            h(k, j) -= sum * v0;
            h(k + 1, j) -= sum * v1;
            if (m == 3) h(k + 2, j) -= sum * v2;
          }
          const int r1 = std::min(hi, k + 3);
          for (int i = lo; i <= r1; ++i) {          // columns k..k+m-1
            double sum = v0 * h(i, k) + v1 * h(i, k + 1) + (m == 3 ? v2 * h(i, k + 2) : 0.0);
            sum *= f;
            h(i, k) -= sum * v0;
            h(i, k + 1) -= sum * v1;
            if (m == 3) h(i, k + 2) -= sum * v2;
          }
        }
      }
      if (k + 1 <= hi - 1) {
        x = h(k + 1, k);
        y = h(k + 2, k);
        z = (k + 3 <= hi) ? h(k + 3, k) : 0.0;
      }
      if (k > lo) {
        h(k + 1, k - 1) = 0.0;
        if (m == 3) h(k + 2, k - 1) = 0.0;
      }
    }
  }
  return true;
}

// solve (A) x = b in place, A complex n x n (destroyed), partial pivoting;
// a zero pivot is replaced by a tiny one (inverse iteration on a nearly
// singular shifted matrix is the intent)
void complex_lu_solve(std::vector<cplx>& A, int n, std::vector<cplx>& b, double tiny) {
  std::vector<int> piv(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::abs(A[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (std::abs(A[i * n + k]) > best) {
        best = std::abs(A[i * n + k]);
        p = i;
      }
    piv[k] = p;
    // swap the not yet eliminated columns only: the multipliers of earlier
    // steps stay in their rows, matching the interleaved solve below
    if (p != k)
      for (int j = k; j < n; ++j) std::swap(A[k * n + j], A[p * n + j]);
    if (std::abs(A[k * n + k]) < tiny) A[k * n + k] = tiny;
    for (int i = k + 1; i < n; ++i) {
      const cplx l = A[i * n + k] / A[k * n + k];
      A[i * n + k] = l;
      for (int j = k + 1; j < n; ++j) A[i * n + j] -= l * A[k * n + j];
    }
  }
  for (int k = 0; k < n; ++k) {
    if (piv[k] != k) std::swap(b[k], b[piv[k]]);
    for (int i = k + 1; i < n; ++i) b[i] -= A[i * n + k] * b[k];
  }
  for (int i = n - 1; i >= 0; --i) {
    cplx s = b[i];
    for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * b[j];
    b[i] = s / A[i * n + i];
  }
}

// inverse of the real n x n A by Gauss-Jordan with partial pivoting
bool real_inverse(const std::vector<double>& A_in, int n, std::vector<double>& Ainv) {
  std::vector<double> A(A_in);
  Ainv.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Ainv[i * n + i] = 1.0;
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[i * n + k]) > std::fabs(A[p * n + k])) p = i;
    if (A[p * n + k] == 0.0) return false;
    if (p != k)
      for (int j = 0; j < n; ++j) {
        std::swap(A[k * n + j], A[p * n + j]);
        std::swap(Ainv[k * n + j], Ainv[p * n + j]);
      }
    const double d = 1.0 / A[k * n + k];
    for (int j = 0; j < n; ++j) {
      A[k * n + j] *= d;
      Ainv[k * n + j] *= d;
    }
    for (int i = 0; i < n; ++i) {
      if (i == k) continue;
      const double f = A[i * n + k];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        A[i * n + j] -= f * A[k * n + j];
        Ainv[i * n + j] -= f * Ainv[k * n + j];
      }
    }
  }
  return true;
}

// least-squares eigenvalue of the real column col of X: x^T M x / x^T x
double rayleigh_real(const std::vector<double>& M, int n, const std::vector<double>& X, int col) {
  double num = 0.0, den = 0.0;
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += M[i * n + j] * X[j * n + col];
    num += X[i * n + col] * s;
    den += X[i * n + col] * X[i * n + col];
  }
  return num / den;
}

}  // namespace

bool real_eigen_decomposition(const std::vector<double>& M, int n, std::vector<double>& X,
                              std::vector<double>& la, std::vector<double>& lb,
                              std::vector<int>& kind) {
  std::vector<double> H(M);
  to_hessenberg(H, n);
  std::vector<cplx> ev;
  if (!hessenberg_eigenvalues(H, n, ev) || (int)ev.size() != n) return false;
  double mnorm = 0.0;
  for (double x : M) mnorm = std::max(mnorm, std::fabs(x));
  if (mnorm == 0.0) mnorm = 1.0;
  // one representative per conjugate pair (positive imaginary part)
  std::vector<cplx> reps;
  const double imtol = 1e-13 * mnorm;
  for (const cplx& l : ev)
    if (l.imag() >= -imtol) reps.push_back(std::fabs(l.imag()) <= imtol ? cplx(l.real(), 0.0) : l);
  X.assign((size_t)n * n, 0.0);
  la.assign(n, 0.0);
  lb.assign(n, 0.0);
  kind.assign(n, 0);
  std::mt19937_64 rng(12345);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  std::vector<std::vector<cplx>> done;           // eigenvectors found so far
  std::vector<cplx> done_l;
  int col = 0;
  for (const cplx& l : reps) {
    const bool real = l.imag() == 0.0;
    if (col + (real ? 1 : 2) > n) return false;
    // inverse iteration on (M - mu I), mu = l moved by a relative 1e-9 so
    // that the shifted matrix is invertible in practice, then Rayleigh
    // quotient steps (mu = x^H M x / x^H x) that refine the pair together
    cplx mu = l + cplx(1e-9 * mnorm, real ? 0.0 : 1e-9 * mnorm);
    std::vector<cplx> x(n), Mx(n);
    for (int i = 0; i < n; ++i) x[i] = cplx(U(rng), real ? 0.0 : U(rng));
    for (int it = 0; it < 6; ++it) {
      // remove the components along earlier vectors of the same eigenvalue
      for (size_t q = 0; q < done.size(); ++q) {
        if (std::abs(done_l[q] - l) > 1e-7 * mnorm) continue;
        cplx dot = 0.0, nn = 0.0;
        for (int i = 0; i < n; ++i) {
          dot += std::conj(done[q][i]) * x[i];
          nn += std::conj(done[q][i]) * done[q][i];
        }
        for (int i = 0; i < n; ++i) x[i] -= dot / nn * done[q][i];
      }
      std::vector<cplx> A((size_t)n * n);
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) A[i * n + j] = cplx(M[i * n + j], 0.0) - (i == j ? mu : cplx(0.0));
      complex_lu_solve(A, n, x, 1e-200 * mnorm);
      double nrm = 0.0;
      for (const cplx& v : x) nrm = std::max(nrm, std::abs(v));
      if (!(nrm > 0.0) || !std::isfinite(nrm)) return false;
      for (cplx& v : x) v /= nrm;
      if (it >= 2) {                                   // Rayleigh quotient
        cplx num = 0.0, den = 0.0;
        for (int i = 0; i < n; ++i) {
          cplx s = 0.0;
          for (int j = 0; j < n; ++j) s += M[i * n + j] * x[j];
          Mx[i] = s;
          num += std::conj(x[i]) * s;
          den += std::conj(x[i]) * x[i];
        }
        const cplx rq = num / den;
        if (std::abs(rq - l) > 1e-6 * mnorm) break;    // wandered off: keep the last vector
        double r = 0.0;
        for (int i = 0; i < n; ++i) r = std::max(r, std::abs(Mx[i] - rq * x[i]));
        if (real) mu = cplx(rq.real(), 0.0); else mu = rq;
        if (r <= 4e-16 * mnorm) break;
        // shift slightly off the refined value so the solve stays finite
        mu += cplx(1e-13 * mnorm, 0.0);
      }
    }
    const cplx lfin = real ? cplx(mu.real() - 0.0, 0.0) : mu;
    if (real) {
      // a real eigenvector: rotate x so its largest entry is real
      int imax = 0;
      for (int i = 1; i < n; ++i)
        if (std::abs(x[i]) > std::abs(x[imax])) imax = i;
      const cplx ph = std::abs(x[imax]) / x[imax];
      for (int i = 0; i < n; ++i) X[i * n + col] = (x[i] * ph).real();
      la[col] = rayleigh_real(M, n, X, col);
      kind[col] = 0;
      col += 1;
    } else {
      for (int i = 0; i < n; ++i) {
        X[i * n + col] = x[i].real();
        X[i * n + col + 1] = x[i].imag();
      }
      la[col] = la[col + 1] = lfin.real();
      lb[col] = lfin.imag();
      lb[col + 1] = -lfin.imag();
      kind[col] = 1;
      kind[col + 1] = 2;
      col += 2;
    }
    done.push_back(x);
    done_l.push_back(l);
  }
  return col == n;
}

bool build_eig_basis_ns(const RefElement& R, const std::vector<double>& S0,
                        const std::vector<double>& W0, const std::vector<double>& V0, double eps0,
                        EigBasisNS& out) {
  const int nv = R.nv, nt = R.nt;
  std::vector<double> B((size_t)nv * nv), Binv, M((size_t)nv * nv, 0.0);
  for (int t = 0; t < nv * nv; ++t) B[t] = eps0 * R.G[t] + S0[t];
  if (!real_inverse(B, nv, Binv)) return false;
  for (int i = 0; i < nv; ++i)
    for (int k = 0; k < nv; ++k) {
      const double b = Binv[i * nv + k];
      if (b == 0.0) continue;
      for (int j = 0; j < nv; ++j) M[i * nv + j] += b * R.G[k * nv + j];
    }
  std::vector<double> X, Xinv;
  if (!real_eigen_decomposition(M, nv, X, out.la, out.lb, out.kind)) return false;
  if (!real_inverse(X, nv, Xinv)) return false;
  // R = X^-1 B^-1; Pw1 = R H, Pw0 = R W0; Pv1 = X^T Hv, Pv0 = X^T V0
  out.X = X;
  out.R.assign((size_t)nv * nv, 0.0);
  for (int i = 0; i < nv; ++i)
    for (int k = 0; k < nv; ++k) {
      const double a = Xinv[i * nv + k];
      for (int j = 0; j < nv; ++j) out.R[i * nv + j] += a * Binv[k * nv + j];
    }
  out.Pw1.assign((size_t)nv * nt, 0.0);
  out.Pw0.assign((size_t)nv * nt, 0.0);
  out.Pv1.assign((size_t)nv * nt, 0.0);
  out.Pv0.assign((size_t)nv * nt, 0.0);
  for (int i = 0; i < nv; ++i)
    for (int c = 0; c < nt; ++c) {
      double w1 = 0.0, w0 = 0.0, v1 = 0.0, v0 = 0.0;
      for (int a = 0; a < nv; ++a) {
        w1 += out.R[i * nv + a] * R.H[a * nt + c];
        w0 += out.R[i * nv + a] * W0[a * nt + c];
        v1 += X[a * nv + i] * R.Hv[a * nt + c];
        v0 += X[a * nv + i] * V0[a * nt + c];
      }
      out.Pw1[i * nt + c] = w1;
      out.Pw0[i * nt + c] = w0;
      out.Pv1[i * nt + c] = v1;
      out.Pv0[i * nt + c] = v0;
    }
  out.eps0 = eps0;
  return true;
}

// A_e(eps) through the decomposition and by a direct dense solve; the
// largest entry difference relative to max |A_e|
double check_eig_basis_ns(const RefElement& R, const std::vector<double>& S0,
                          const std::vector<double>& W0, const std::vector<double>& V0,
                          const std::vector<double>& adiag, const EigBasisNS& E, double eps) {
  const int nv = R.nv, nt = R.nt;
  const double d = eps - E.eps0;
  // direct: S^-1 W by Gauss-Jordan
  std::vector<double> S((size_t)nv * nv), Sinv;
  for (int t = 0; t < nv * nv; ++t) S[t] = eps * R.G[t] + S0[t];
  if (!real_inverse(S, nv, Sinv)) return 1e300;
  std::vector<double> A1((size_t)nt * nt), A2((size_t)nt * nt);
  std::vector<double> X((size_t)nv * nt, 0.0), Y((size_t)nv * nt, 0.0);
  for (int i = 0; i < nv; ++i)
    for (int c = 0; c < nt; ++c) {
      double s = 0.0;
      for (int a = 0; a < nv; ++a) s += Sinv[i * nv + a] * (eps * R.H[a * nt + c] + W0[a * nt + c]);
      X[i * nt + c] = s;
    }
  // basis: Y = blocks(d) (eps Pw1 + Pw0)
  for (int i = 0; i < nv; ++i) {
    const double a = 1.0 + d * E.la[i];
    for (int c = 0; c < nt; ++c) {
      const double w = eps * E.Pw1[i * nt + c] + E.Pw0[i * nt + c];
      if (E.kind[i] == 0) {
        Y[i * nt + c] = w / a;
      } else {
        const int i0 = E.kind[i] == 1 ? i : i - 1;
        const double ar = 1.0 + d * E.la[i0], bi = d * E.lb[i0];
        const double det = ar * ar + bi * bi;
        const double w0 = eps * E.Pw1[i0 * nt + c] + E.Pw0[i0 * nt + c];
        const double w1 = eps * E.Pw1[(i0 + 1) * nt + c] + E.Pw0[(i0 + 1) * nt + c];
        Y[i * nt + c] = E.kind[i] == 1 ? (ar * w0 - bi * w1) / det : (bi * w0 + ar * w1) / det;
      }
    }
  }
  double amax = 0.0, dmax = 0.0;
  for (int r = 0; r < nt; ++r)
    for (int c = 0; c < nt; ++c) {
      double s1 = 0.0, s2 = 0.0;
      for (int a = 0; a < nv; ++a) s1 += (eps * R.Hv[a * nt + r] + V0[a * nt + r]) * X[a * nt + c];
      for (int i = 0; i < nv; ++i)
        s2 += (eps * E.Pv1[i * nt + r] + E.Pv0[i * nt + r]) * Y[i * nt + c];
      const double base = eps * R.K[r * nt + c] + (r == c ? adiag[r] : 0.0);
      amax = std::max(amax, std::fabs(base - s1));
      dmax = std::max(dmax, std::fabs(s1 - s2));
    }
  return amax > 0.0 ? dmax / amax : dmax;
}

}  // namespace hdgmg
