"""Reference-element building blocks for the oracle (test infrastructure only).

Bases (readings of the paper, Sec. 2, where P^p is written for every element but
Example I runs quadrilaterals):

* volume space on a square element: tensor-product Q_p, Lagrange basis at the
  (p+1) Gauss-Legendre points per direction, node (a, b) -> index b*(p+1)+a
  (x index fastest);
* trace space on an edge: P_p with the L2-orthonormal Legendre basis
  psi_k(s) = sqrt((2k+1)/|e|) P_k(s), s in [-1, 1] running along +x for
  horizontal and +y for vertical edges.

Everything here is evaluated directly from its definition (Lagrange products,
the Legendre recurrence); quadrature points come from numpy's Gauss-Legendre
routine, which serves as a library primitive.  Pins: tests/test_oracle_refelem.py
(partition of unity, exact polynomial integration, orthonormality).
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def gauss(m):
    """m-point Gauss-Legendre rule on [-1, 1] (nodes ascending, weights)."""
    x, w = npleg.leggauss(m)
    return np.asarray(x, dtype=np.float64), np.asarray(w, dtype=np.float64)


def lagrange(nodes, x):
    """Values L[j, q] = l_j(x_q) of the Lagrange polynomials on ``nodes``."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    m = len(nodes)
    L = np.ones((m, len(x)))
    for j in range(m):
        for k in range(m):
            if k != j:
                L[j] *= (x - nodes[k]) / (nodes[j] - nodes[k])
    return L


def lagrange_deriv(nodes, x):
    """Derivatives D[j, q] = l_j'(x_q), by the product rule applied term by term."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    m = len(nodes)
    D = np.zeros((m, len(x)))
    for j in range(m):
        for k in range(m):
            if k == j:
                continue
            term = np.full(len(x), 1.0 / (nodes[j] - nodes[k]))
            for l in range(m):
                if l != j and l != k:
                    term = term * (x - nodes[l]) / (nodes[j] - nodes[l])
            D[j] += term
    return D


def legendre(p, s):
    """P[k, q] = P_k(s_q), k = 0..p (classical Legendre polynomials)."""
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    P = np.zeros((p + 1, len(s)))
    for k in range(p + 1):
        c = np.zeros(k + 1)
        c[k] = 1.0
        P[k] = npleg.legval(s, c)
    return P


def trace_basis(p, s, length):
    """Orthonormal trace basis psi_k(s) = sqrt((2k+1)/length) P_k(s) on an edge."""
    P = legendre(p, s)
    scale = np.sqrt((2.0 * np.arange(p + 1) + 1.0) / length)
    return P * scale[:, None]


class RefQuad:
    """Volume and edge quadrature plus basis tables for a rectangle hx x hy.

    ``nq`` quadrature points per direction; the default p+3 over-integrates
    every bilinear form of the HDG scheme (all are polynomials of degree <= 2p
    per direction), so the oracle's integrals are exact and do not depend on
    the Gauss-Lobatto/Gauss choice of the CUDA path.
    """

    def __init__(self, p, hx, hy, nq=None):
        self.p = p
        self.hx = float(hx)
        self.hy = float(hy)
        self.nq = nq if nq is not None else p + 3
        self.nodes, self.wnodes = gauss(p + 1)           # volume nodal points
        self.xq, self.wq = gauss(self.nq)                 # quadrature points
        nv1 = p + 1
        self.nv = nv1 * nv1
        # 1-D tables at quadrature points and at the end points -1, +1
        self.l_q = lagrange(self.nodes, self.xq)          # [nv1, nq]
        self.dl_q = lagrange_deriv(self.nodes, self.xq)   # [nv1, nq]
        self.l_end = lagrange(self.nodes, np.array([-1.0, 1.0]))  # [nv1, 2]
        self.dl_end = lagrange_deriv(self.nodes, np.array([-1.0, 1.0]))

    # --- 2-D volume basis at the tensor quadrature grid ------------------
    def volume_tables(self):
        """phi[a, q], dphidx[a, q], dphidy[a, q], weights wJ[q] on the element.

        q runs over the tensor grid (qx, qy) with qx fastest; derivatives are
        physical (d/dx = (2/hx) d/dxi)."""
        p1 = self.p + 1
        nq = self.nq
        phi = np.zeros((self.nv, nq * nq))
        dx = np.zeros((self.nv, nq * nq))
        dy = np.zeros((self.nv, nq * nq))
        for b in range(p1):
            for a in range(p1):
                idx = b * p1 + a
                phi[idx] = np.outer(self.l_q[b], self.l_q[a]).ravel()
                dx[idx] = np.outer(self.l_q[b], self.dl_q[a]).ravel() * (2.0 / self.hx)
                dy[idx] = np.outer(self.dl_q[b], self.l_q[a]).ravel() * (2.0 / self.hy)
        wJ = np.outer(self.wq, self.wq).ravel() * (self.hx * self.hy / 4.0)
        return phi, dx, dy, wJ

    # --- edge tables ------------------------------------------------------
    def edge_tables(self, edge):
        """For local edge 0=left, 1=right, 2=bottom, 3=top return
        (phi_on_edge[a, q], psi[k, q], w_ds[q], normal (nx, ny)).

        The edge parameter s runs along +y on vertical and +x on horizontal
        edges; w_ds includes the edge Jacobian |e|/2."""
        p1 = self.p + 1
        nq = self.nq
        phi = np.zeros((self.nv, nq))
        if edge in (0, 1):
            end = 0 if edge == 0 else 1
            for b in range(p1):
                for a in range(p1):
                    phi[b * p1 + a] = self.l_end[a, end] * self.l_q[b]
            length = self.hy
            normal = (-1.0, 0.0) if edge == 0 else (1.0, 0.0)
        else:
            end = 0 if edge == 2 else 1
            for b in range(p1):
                for a in range(p1):
                    phi[b * p1 + a] = self.l_q[a] * self.l_end[b, end]
            length = self.hx
            normal = (0.0, -1.0) if edge == 2 else (0.0, 1.0)
        psi = trace_basis(self.p, self.xq, length)
        w_ds = self.wq * (length / 2.0)
        return phi, psi, w_ds, normal

    def edge_normal_derivative(self, edge):
        """dn[a, q] = (grad phi_a . n)(s_q) on local edge ``edge`` at the same
        quadrature points as ``edge_tables`` (physical derivative)."""
        p1 = self.p + 1
        dn = np.zeros((self.nv, self.nq))
        end = 0 if edge in (0, 2) else 1
        sign = -1.0 if edge in (0, 2) else 1.0
        for b in range(p1):
            for a in range(p1):
                if edge in (0, 1):      # n = -+x: d/dx of l_a(xi) at xi = -+1, times l_b(eta)
                    dn[b * p1 + a] = sign * (2.0 / self.hx) * self.dl_end[a, end] * self.l_q[b]
                else:                   # n = -+y
                    dn[b * p1 + a] = sign * (2.0 / self.hy) * self.l_q[a] * self.dl_end[b, end]
        return dn

    def nodal_gradient(self):
        """(Gx, Gy): [n_v, n_v] matrices taking nodal values of a Q_p function
        to its physical x- and y-derivatives at the nodes."""
        p1 = self.p + 1
        D = lagrange_deriv(self.nodes, self.nodes)      # D[j, i] = l_j'(xi_i)
        Gx = np.zeros((self.nv, self.nv))
        Gy = np.zeros((self.nv, self.nv))
        for a2 in range(p1):
            for a1 in range(p1):
                for b in range(p1):
                    Gx[a2 * p1 + a1, a2 * p1 + b] = (2.0 / self.hx) * D[b, a1]
                    Gy[a2 * p1 + a1, b * p1 + a1] = (2.0 / self.hy) * D[b, a2]
        return Gx, Gy
