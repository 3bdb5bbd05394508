// Host construction of the reference-element tables (FP64).
//
// Bilinear forms of the HDG local problem (arXiv:1811.09909, Sec. 2, eqs.
// HDG_local1, HDG_local2 with the flux HDG_flux), with K = kappa I:
//   (kappa^-1 q, v) - (u, div v) + <lambda, v.n> = 0
//   (div q, w) + <tau (u - lambda), w>            = (f, w)
// (the second one after integrating the paper's -(q, grad w) + <q.n, w> by
// parts back).  Eliminating q with the diagonal Gauss-point mass matrix M:
//   (kappa G + tau E) u = M f + (kappa H + tau F) lambda
// and the element contribution to the conservation condition gives the trace
// operator  A_e = kappa K + tau I - W^T S^-1 W,  S = kappa G + tau E,
// W = kappa H + tau F  (I = trace mass matrix in the orthonormal basis).
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace hdgmg {

void gauss_legendre(int m, std::vector<double>& x, std::vector<double>& w) {
  x.assign(m, 0.0);
  w.assign(m, 0.0);
  for (int i = 0; i < m; ++i) {
    // Newton on P_m from the Chebyshev-like first guess, root index m-1-i so
    // that the nodes come out ascending
    double z = std::cos(M_PI * (m - 1 - i + 0.75) / (m + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      if (m == 0) break;
      for (int k = 2; k <= m; ++k) {
        double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      double pm = (m == 1) ? z : p1;
      double pm1 = (m == 1) ? 1.0 : p0;
      dp = m * (z * pm - pm1) / (z * z - 1.0);
      double dz = pm / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    // derivative at the converged root
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= m; ++k) {
      double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = pk;
    }
    double pm = (m == 1) ? z : p1;
    double pm1 = (m == 1) ? 1.0 : p0;
    dp = m * (z * pm - pm1) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

static double legendre_p(int k, double s) {
  if (k == 0) return 1.0;
  double p0 = 1.0, p1 = s;
  for (int j = 2; j <= k; ++j) {
    double pj = ((2.0 * j - 1.0) * s * p1 - (j - 1.0) * p0) / j;
    p0 = p1;
    p1 = pj;
  }
  return p1;
}

void child_injection(double J[2][2][2]) {
  // macro-edge P1 function c0 psi0 + c1 psi1 restricted to a half: the half
  // parameter s maps to t = (s -+ 1)/2; in the half's orthonormal basis
  //   mode 0: c0 / sqrt(2) -+ c1 sqrt(3) / (2 sqrt(2)),   mode 1: c1 / (2 sqrt(2))
  const double r2 = std::sqrt(2.0), r3 = std::sqrt(3.0);
  for (int c = 0; c < 2; ++c) {
    double sg = (c == 0) ? -1.0 : 1.0;
    J[c][0][0] = 1.0 / r2;
    J[c][0][1] = sg * r3 / (2.0 * r2);
    J[c][1][0] = 0.0;
    J[c][1][1] = 1.0 / (2.0 * r2);
  }
}

RefElement build_ref_element(int p, double hx, double hy) {
  RefElement R;
  const int p1 = p + 1;
  const int nv = p1 * p1, nt = 4 * p1;
  R.p = p;
  R.nv = nv;
  R.nt = nt;
  R.hx = hx;
  R.hy = hy;
  gauss_legendre(p1, R.nodes, R.weights);
  const std::vector<double>& xi = R.nodes;
  const std::vector<double>& w = R.weights;
  // barycentric weights and the derivative matrix D[i][j] = l_j'(xi_i)
  std::vector<double> bw(p1, 1.0), D(p1 * p1, 0.0), lm(p1), lp(p1);
  for (int j = 0; j < p1; ++j)
    for (int k = 0; k < p1; ++k)
      if (k != j) bw[j] /= (xi[j] - xi[k]);
  for (int i = 0; i < p1; ++i) {
    double diag = 0.0;
    for (int j = 0; j < p1; ++j)
      if (j != i) {
        D[i * p1 + j] = (bw[j] / bw[i]) / (xi[i] - xi[j]);
        diag -= D[i * p1 + j];
      }
    D[i * p1 + i] = diag;
  }
  // l_j(-1), l_j(+1)
  for (int j = 0; j < p1; ++j) {
    double a = 1.0, b = 1.0;
    for (int k = 0; k < p1; ++k)
      if (k != j) {
        a *= (-1.0 - xi[k]) / (xi[j] - xi[k]);
        b *= (1.0 - xi[k]) / (xi[j] - xi[k]);
      }
    lm[j] = a;
    lp[j] = b;
  }
  const double Jac = hx * hy / 4.0;
  R.M.assign(nv, 0.0);
  for (int b2 = 0; b2 < p1; ++b2)
    for (int b1 = 0; b1 < p1; ++b1) R.M[b2 * p1 + b1] = w[b1] * w[b2] * Jac;
  // B_x[b][a] = (phi_b, d_x phi_a) = w_b J (2/hx) D[b1][a1] delta(b2,a2)
  std::vector<double> Bx(nv * nv, 0.0), By(nv * nv, 0.0);
  for (int b2 = 0; b2 < p1; ++b2)
    for (int b1 = 0; b1 < p1; ++b1) {
      int b = b2 * p1 + b1;
      double wb = w[b1] * w[b2] * Jac;
      for (int a1 = 0; a1 < p1; ++a1) Bx[b * nv + (b2 * p1 + a1)] = wb * (2.0 / hx) * D[b1 * p1 + a1];
      for (int a2 = 0; a2 < p1; ++a2) By[b * nv + (a2 * p1 + b1)] = wb * (2.0 / hy) * D[b2 * p1 + a2];
    }
  R.BxT.assign(nv * nv, 0.0);
  R.ByT.assign(nv * nv, 0.0);
  for (int a = 0; a < nv; ++a)
    for (int b = 0; b < nv; ++b) {
      R.BxT[a * nv + b] = Bx[b * nv + a];
      R.ByT[a * nv + b] = By[b * nv + a];
    }
  // edge terms: local edge 0 left (xi=-1, n=-x), 1 right, 2 bottom (eta=-1,
  // n=-y), 3 top.  Edge quadrature at the Gauss nodes of the tangential
  // direction, measure |e|/2.
  R.E.assign(nv * nv, 0.0);
  R.Ef.assign(4 * nv * nv, 0.0);
  R.F.assign(nv * nt, 0.0);
  R.Cx.assign(nv * nt, 0.0);
  R.Cy.assign(nv * nt, 0.0);
  for (int edge = 0; edge < 4; ++edge) {
    const bool vert = edge < 2;
    const double len = vert ? hy : hx;
    const std::vector<double>& lend = (edge == 0 || edge == 2) ? lm : lp;
    const double nrm = (edge == 0 || edge == 2) ? -1.0 : 1.0;
    for (int q = 0; q < p1; ++q) {          // tangential quadrature node
      const double wq = w[q] * len / 2.0;
      for (int na = 0; na < p1; ++na) {     // normal-direction node of phi_a
        const int a = vert ? (q * p1 + na) : (na * p1 + q);
        const double phia = lend[na];
        for (int nb = 0; nb < p1; ++nb) {
          const int b = vert ? (q * p1 + nb) : (nb * p1 + q);
          R.E[a * nv + b] += wq * phia * lend[nb];
          R.Ef[(size_t)edge * nv * nv + a * nv + b] += wq * phia * lend[nb];
        }
        for (int k = 0; k < p1; ++k) {
          const double psi = std::sqrt((2.0 * k + 1.0) / len) * legendre_p(k, xi[q]);
          const double val = wq * phia * psi;
          R.F[a * nt + edge * p1 + k] += val;
          if (vert)
            R.Cx[a * nt + edge * p1 + k] += nrm * val;
          else
            R.Cy[a * nt + edge * p1 + k] += nrm * val;
        }
      }
    }
  }
  // G = sum_d B_d M^-1 B_d^T, H = sum_d B_d M^-1 C_d, K = sum_d C_d^T M^-1 C_d
  R.G.assign(nv * nv, 0.0);
  R.H.assign(nv * nt, 0.0);
  R.K.assign(nt * nt, 0.0);
  for (int a = 0; a < nv; ++a) {
    const double mi = 1.0 / R.M[a];
    for (int b = 0; b < nv; ++b) {
      const double bxa = Bx[b * nv + a], bya = By[b * nv + a];
      if (bxa == 0.0 && bya == 0.0) continue;
      for (int c = 0; c < nv; ++c) R.G[b * nv + c] += (bxa * Bx[c * nv + a] + bya * By[c * nv + a]) * mi;
      for (int k = 0; k < nt; ++k) R.H[b * nt + k] += (bxa * R.Cx[a * nt + k] + bya * R.Cy[a * nt + k]) * mi;
    }
    for (int k = 0; k < nt; ++k) {
      const double cxk = R.Cx[a * nt + k], cyk = R.Cy[a * nt + k];
      if (cxk == 0.0 && cyk == 0.0) continue;
      for (int l = 0; l < nt; ++l) R.K[k * nt + l] += (cxk * R.Cx[a * nt + l] + cyk * R.Cy[a * nt + l]) * mi;
    }
  }
  R.Hv = R.H;
  return R;
}

// Primal hybridized interior penalty element (Sec. 2, eqs. IPDG_flux, IPG_H).
// Every integrand is a polynomial of degree <= 2p per direction, so the
// (p+1)-point Gauss rule at the nodes integrates it exactly; at the nodes
// l_a(xi_q) = delta_aq, which collapses the quadrature sums below.
void make_ipdg_tables(RefElement& R, double sf) {
  const int p1 = R.p + 1, nv = R.nv, nt = R.nt;
  const std::vector<double>& xi = R.nodes;
  const std::vector<double>& w = R.weights;
  const double hx = R.hx, hy = R.hy, Jac = hx * hy / 4.0;
  // D[i][j] = l_j'(xi_i) (barycentric), le[s][j] = l_j(-+1), dl[s][j] = l_j'(-+1)
  std::vector<double> bw(p1, 1.0), D(p1 * p1, 0.0), le(2 * p1), dl(2 * p1);
  for (int j = 0; j < p1; ++j)
    for (int k = 0; k < p1; ++k)
      if (k != j) bw[j] /= (xi[j] - xi[k]);
  for (int i = 0; i < p1; ++i) {
    double diag = 0.0;
    for (int j = 0; j < p1; ++j)
      if (j != i) {
        D[i * p1 + j] = (bw[j] / bw[i]) / (xi[i] - xi[j]);
        diag -= D[i * p1 + j];
      }
    D[i * p1 + i] = diag;
  }
  for (int s = 0; s < 2; ++s) {
    const double x = s == 0 ? -1.0 : 1.0;     // not a Gauss node
    for (int j = 0; j < p1; ++j) {
      double l = 1.0, sum = 0.0;
      for (int k = 0; k < p1; ++k)
        if (k != j) {
          l *= (x - xi[k]) / (xi[j] - xi[k]);
          sum += 1.0 / (x - xi[k]);
        }
      le[s * p1 + j] = l;
      dl[s * p1 + j] = l * sum;
    }
  }
  auto idx = [p1](int a1, int a2) { return a2 * p1 + a1; };
  // stiffness: x-part couples equal y indices, y-part equal x indices
  std::vector<double> Kst(nv * nv, 0.0);
  const double cx = Jac * (2.0 / hx) * (2.0 / hx), cy = Jac * (2.0 / hy) * (2.0 / hy);
  for (int a2 = 0; a2 < p1; ++a2)
    for (int a1 = 0; a1 < p1; ++a1)
      for (int b1 = 0; b1 < p1; ++b1) {
        double s = 0.0;
        for (int q = 0; q < p1; ++q) s += w[q] * D[q * p1 + a1] * D[q * p1 + b1];
        Kst[idx(a1, a2) * nv + idx(b1, a2)] += cx * w[a2] * s;
      }
  for (int a1 = 0; a1 < p1; ++a1)
    for (int a2 = 0; a2 < p1; ++a2)
      for (int b2 = 0; b2 < p1; ++b2) {
        double s = 0.0;
        for (int q = 0; q < p1; ++q) s += w[q] * D[q * p1 + a2] * D[q * p1 + b2];
        Kst[idx(a1, a2) * nv + idx(a1, b2)] += cy * w[a1] * s;
      }
  // boundary terms, edge 0 left (n = -x), 1 right, 2 bottom (n = -y), 3 top;
  // on a vertical edge the tangential node is a2, on a horizontal one a1
  std::vector<double> N(nv * nv, 0.0), Hn(nv * nt, 0.0);
  for (int edge = 0; edge < 4; ++edge) {
    const bool vert = edge < 2;
    const int s = (edge == 0 || edge == 2) ? 0 : 1;
    const double sg = s == 0 ? -1.0 : 1.0;
    const double len = vert ? hy : hx;
    const double dnorm = sg * 2.0 / (vert ? hx : hy);   // d/dn of the normal coordinate
    for (int t = 0; t < p1; ++t)            // tangential node (= quadrature point)
      for (int na = 0; na < p1; ++na) {     // normal-direction index of phi_a
        const int a = vert ? idx(na, t) : idx(t, na);
        const double dna = w[t] * (len / 2.0) * dnorm * dl[s * p1 + na];
        for (int nb = 0; nb < p1; ++nb) {
          const int b = vert ? idx(nb, t) : idx(t, nb);
          N[a * nv + b] += dna * le[s * p1 + nb];
        }
        for (int k = 0; k < p1; ++k) {
          const double psi = std::sqrt((2.0 * k + 1.0) / len) * legendre_p(k, xi[t]);
          Hn[a * nt + edge * p1 + k] += dna * psi;
        }
      }
  }
  for (int a = 0; a < nv; ++a)
    for (int b = 0; b < nv; ++b) R.G[a * nv + b] = Kst[a * nv + b] - sf * N[a * nv + b] - N[b * nv + a];
  for (int t = 0; t < nv * nt; ++t) {
    R.H[t] = -sf * Hn[t];
    R.Hv[t] = -Hn[t];
  }
  std::fill(R.K.begin(), R.K.end(), 0.0);
  std::fill(R.Cx.begin(), R.Cx.end(), 0.0);
  std::fill(R.Cy.begin(), R.Cy.end(), 0.0);
  std::fill(R.BxT.begin(), R.BxT.end(), 0.0);
  std::fill(R.ByT.begin(), R.ByT.end(), 0.0);
  for (int a2 = 0; a2 < p1; ++a2)
    for (int a1 = 0; a1 < p1; ++a1) {
      const int a = idx(a1, a2);
      for (int b = 0; b < p1; ++b) {
        R.BxT[a * nv + idx(b, a2)] = -R.M[a] * (2.0 / hx) * D[a1 * p1 + b];
        R.ByT[a * nv + idx(a1, b)] = -R.M[a] * (2.0 / hy) * D[a2 * p1 + b];
      }
    }
}

void fold_kappa_tau(RefElement& R, double t) {
  const int nv = R.nv, nt = R.nt;
  for (int i = 0; i < nv * nv; ++i) R.G[i] += t * R.E[i];
  for (int i = 0; i < nv * nt; ++i) {
    R.H[i] += t * R.F[i];
    R.Hv[i] += t * R.F[i];
  }
  for (int c = 0; c < nt; ++c) R.K[c * nt + c] += t;
}

void build_cd_tables(const RefElement& R, double tau, double bx, double by,
                     std::vector<double>& S0, std::vector<double>& W0, std::vector<double>& V0,
                     std::vector<double>& adiag) {
  const int nv = R.nv, nt = R.nt, p1 = R.p + 1;
  const double bn[4] = {-bx, bx, -by, by};
  double tf[4];
  for (int f = 0; f < 4; ++f) tf[f] = tau + (bn[f] > 0.0 ? bn[f] : 0.0);
  S0.assign((size_t)nv * nv, 0.0);
  for (int t = 0; t < nv * nv; ++t) {
    double s = -bx * R.BxT[t] - by * R.ByT[t];
    for (int f = 0; f < 4; ++f) s += tf[f] * R.Ef[(size_t)f * nv * nv + t];
    S0[t] = s;
  }
  W0.assign((size_t)nv * nt, 0.0);
  V0.assign((size_t)nv * nt, 0.0);
  for (int a = 0; a < nv; ++a)
    for (int c = 0; c < nt; ++c) {
      const int f = c / p1;
      W0[(size_t)a * nt + c] = (tf[f] - bn[f]) * R.F[(size_t)a * nt + c];
      V0[(size_t)a * nt + c] = tf[f] * R.F[(size_t)a * nt + c];
    }
  adiag.assign(nt, 0.0);
  for (int c = 0; c < nt; ++c) adiag[c] = tf[c / p1] - bn[c / p1];
}

}  // namespace hdgmg
