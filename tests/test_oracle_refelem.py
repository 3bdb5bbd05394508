"""Pins of the oracle's reference-element tables against closed forms."""
import numpy as np
import pytest

from oracle import refelem


@pytest.mark.parametrize("m", [1, 2, 3, 5, 8])
def test_gauss_rule_exact_for_degree_2m_minus_1(m):
    x, w = refelem.gauss(m)
    for k in range(2 * m):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-14
    # and not exact one degree higher (m >= 1): int x^{2m} != sum
    k = 2 * m
    assert abs(np.sum(w * x ** k) - 2.0 / (k + 1)) > 1e-6


@pytest.mark.parametrize("p", [0, 1, 2, 4, 7])
def test_lagrange_cardinal_and_monomial_reproduction(p):
    nodes, _ = refelem.gauss(p + 1)
    L = refelem.lagrange(nodes, nodes)
    assert np.allclose(L, np.eye(p + 1), atol=1e-14)
    xs = np.linspace(-1, 1, 11)
    Lx = refelem.lagrange(nodes, xs)
    Dx = refelem.lagrange_deriv(nodes, xs)
    for k in range(p + 1):
        assert np.allclose(nodes ** k @ Lx, xs ** k, atol=1e-12)
        dk = k * xs ** (k - 1) if k > 0 else 0 * xs
        assert np.allclose(nodes ** k @ Dx, dk, atol=1e-11)


@pytest.mark.parametrize("p,length", [(1, 1.0), (4, 0.25), (8, 3.0)])
def test_trace_basis_orthonormal(p, length):
    s, w = refelem.gauss(p + 2)
    psi = refelem.trace_basis(p, s, length)
    G = (psi * w * length / 2) @ psi.T
    assert np.allclose(G, np.eye(p + 1), atol=1e-13)


def test_legendre_closed_forms():
    s = np.linspace(-1, 1, 7)
    P = refelem.legendre(3, s)
    assert np.allclose(P[0], 1)
    assert np.allclose(P[1], s)
    assert np.allclose(P[2], 1.5 * s ** 2 - 0.5)
    assert np.allclose(P[3], 2.5 * s ** 3 - 1.5 * s)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_normal_derivative_and_nodal_gradient(p):
    """For v = x^p y^(p-1) + 2x - y on a 0.3 x 0.2 element centred at the
    origin: grad v . n on each edge and grad v at the nodes from its nodal
    values match the analytic derivatives (IPDG-H boundary terms, Sec. 2)."""
    hx, hy = 0.3, 0.2
    rq = refelem.RefQuad(p, hx, hy)
    v = lambda x, y: x ** p * y ** (p - 1) + 2 * x - y
    vx = lambda x, y: p * x ** (p - 1) * y ** (p - 1) + 2
    vy = lambda x, y: (p - 1) * x ** p * y ** max(p - 2, 0) - 1 if p > 1 else -1 + 0 * x
    p1 = p + 1
    a = np.arange(rq.nv) % p1
    b = np.arange(rq.nv) // p1
    X, Y = 0.5 * hx * rq.nodes[a], 0.5 * hy * rq.nodes[b]
    coef = v(X, Y)
    Gx, Gy = rq.nodal_gradient()
    assert np.abs(Gx @ coef - vx(X, Y)).max() < 1e-11
    assert np.abs(Gy @ coef - vy(X, Y)).max() < 1e-11
    s = rq.xq
    for edge, (x, y, n) in enumerate([(-hx / 2 + 0 * s, hy / 2 * s, (-1, 0)),
                                      (hx / 2 + 0 * s, hy / 2 * s, (1, 0)),
                                      (hx / 2 * s, -hy / 2 + 0 * s, (0, -1)),
                                      (hx / 2 * s, hy / 2 + 0 * s, (0, 1))]):
        dn = rq.edge_normal_derivative(edge)
        exact = n[0] * vx(x, y) + n[1] * vy(x, y)
        assert np.abs(coef @ dn - exact).max() < 1e-11, edge
