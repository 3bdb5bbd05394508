"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the multigrid method: it only draws random
coefficients and evaluates manufactured data at the points where the library's
interface expects them.

Input layouts (the library interface):
  log_kappa [E]                     per-element log-diffusivity, e = j*n + i
  f         [nrhs][(p+1)^2][E]      forcing at the tensor Gauss-Legendre nodes
                                    of each element, node (a, b) at b*(p+1)+a
  g_D       [nrhs][p+1][n_edges]    orthonormal-Legendre coefficients of the
                                    Dirichlet data on boundary edges (entries on
                                    interior edges are ignored)

Workloads (paper: arXiv:1811.09909):
  * ``poisson_sine``  : -lap u = f, u = sin(pi x) sin(pi y), kappa = 1, g_D = 0
    (16 x 16, p = 2, tau = 1 for the 3-level V(1,1)-CG configuration).
  * ``example1``      : Example I of Sec. 4.1, u = x y exp(x^2 y^3) with its
    Dirichlet data, kappa = 1.
  * ``lognormal``     : log kappa iid N(0, sigma^2) per element (seeded), f = 1,
    g_D = 0 -- the synthetic stand-in for the heterogeneous permeability of
    Example V (SPE10 layer 75, a dataset that is not used here).
  * ``example3``      : Example III's smooth kappa = 1 + 0.5 sin(2 pi x) cos(3 pi y)
    on the unit square (the paper's circle of triangles is not a quad mesh),
    sampled at element centres, with u = x y exp(x^2 y^3) and
    f = -div(kappa grad u) of the smooth kappa.
  * ``checkerboard``  : Example IV's two-block kappa in {1e6, 1} (element
    centres decide the block), f = 1, g_D = 0.
  * ``convdiff``      : -eps lap u + beta.grad u = f with constant eps (given
    per element as log eps) and beta, manufactured u = sin(pi x) sin(pi y)
    (so g_D = 0), tau_e = eps/h on every face plus the upwind max(beta.n, 0)
    the library adds.
"""
import math

import numpy as np
from numpy.polynomial import legendre as npleg


def n_edges(n):
    return 2 * n * (n + 1)


def gauss_nodes(p):
    x, _ = npleg.leggauss(p + 1)
    return x


def nodal(fun, n, p, x0=0.0, x1=1.0, y0=0.0, y1=1.0):
    """Evaluate fun(x, y) at the Gauss-Legendre nodes of every element.

    Returns [(p+1)^2][n*n] float64."""
    xi = gauss_nodes(p)
    p1 = p + 1
    hx = (x1 - x0) / n
    hy = (y1 - y0) / n
    e = np.arange(n * n)
    j, i = np.divmod(e, n)
    a = np.arange(p1 * p1) % p1
    b = np.arange(p1 * p1) // p1
    X = x0 + (i[None, :] + 0.5) * hx + 0.5 * hx * xi[a][:, None]
    Y = y0 + (j[None, :] + 0.5) * hy + 0.5 * hy * xi[b][:, None]
    return np.ascontiguousarray(fun(X, Y), dtype=np.float64)


def dirichlet(fun, n, p, x0=0.0, x1=1.0, y0=0.0, y1=1.0, nq=None):
    """Orthonormal-Legendre coefficients of fun on every boundary edge.

    Returns [p+1][n_edges] float64 (zero on interior edges)."""
    nq = nq if nq is not None else p + 8
    s, w = npleg.leggauss(nq)
    hx = (x1 - x0) / n
    hy = (y1 - y0) / n
    P = np.stack([npleg.legval(s, np.eye(p + 1)[k]) for k in range(p + 1)])
    out = np.zeros((p + 1, n_edges(n)))
    nvert = n * (n + 1)

    def coeffs(xs, ys, length):
        vals = fun(xs, ys)
        scale = np.sqrt((2.0 * np.arange(p + 1) + 1.0) / length)
        return (P * scale[:, None]) @ (w * vals) * (length / 2.0)

    for j in range(n):
        yc = y0 + (j + 0.5) * hy + 0.5 * hy * s
        for i in (0, n):
            xc = np.full_like(s, x0 + i * hx)
            out[:, j * (n + 1) + i] = coeffs(xc, yc, hy)
    for jj in (0, n):
        for i in range(n):
            xc = x0 + (i + 0.5) * hx + 0.5 * hx * s
            yc = np.full_like(s, y0 + jj * hy)
            out[:, nvert + jj * n + i] = coeffs(xc, yc, hx)
    return out


# --------------------------------------------------------------------------
# manufactured solutions
# --------------------------------------------------------------------------
def sine_u(x, y):
    return np.sin(np.pi * x) * np.sin(np.pi * y)


def sine_f(x, y):
    return 2.0 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(np.pi * y)


def sine_q(x, y):
    """q = -grad u for kappa = 1."""
    return (-np.pi * np.cos(np.pi * x) * np.sin(np.pi * y),
            -np.pi * np.sin(np.pi * x) * np.cos(np.pi * y))


def ex1_u(x, y):
    """Example I exact solution u = x y exp(x^2 y^3)."""
    return x * y * np.exp(x ** 2 * y ** 3)


def ex1_f(x, y):
    """-lap u for u = x y exp(x^2 y^3) (derivatives worked by hand)."""
    E = np.exp(x ** 2 * y ** 3)
    return -E * (6 * x * y ** 4 + 4 * x ** 3 * y ** 7 + 12 * x ** 3 * y ** 2 + 9 * x ** 5 * y ** 5)


def ex1_q(x, y):
    E = np.exp(x ** 2 * y ** 3)
    return (-y * E * (1 + 2 * x ** 2 * y ** 3), -x * E * (1 + 3 * x ** 2 * y ** 3))


# --------------------------------------------------------------------------
# configurations
# --------------------------------------------------------------------------
class Workload:
    """One synthetic problem: mesh size, order, coefficients and data."""

    def __init__(self, name, n, p, log_kappa, f, gD, tau_mode, tau_c,
                 x0=0.0, x1=1.0, y0=0.0, y1=1.0, seed=None, beta=None):
        self.name = name
        self.n, self.p = n, p
        self.log_kappa = np.ascontiguousarray(log_kappa, dtype=np.float64)
        self.f = np.ascontiguousarray(f, dtype=np.float64)
        self.gD = np.ascontiguousarray(gD, dtype=np.float64)
        self.tau_mode, self.tau_c = tau_mode, tau_c
        self.x0, self.x1, self.y0, self.y1 = x0, x1, y0, y1
        self.seed = seed
        self.beta = beta          # None: diffusion; (bx, by): convection-diffusion

    @property
    def E(self):
        return self.n * self.n

    @property
    def interior_trace_dofs(self):
        return 2 * self.n * (self.n - 1) * (self.p + 1)

    def tau(self):
        """tau per element as the library computes it (TAU_CONST, c/h_min or
        c kappa_e/h_min)."""
        h = min((self.x1 - self.x0) / self.n, (self.y1 - self.y0) / self.n)
        if self.tau_mode == "const":
            return self.tau_c
        if self.tau_mode == "kappa_over_h":
            return self.tau_c * np.exp(self.log_kappa) / h
        return self.tau_c / h


def poisson_sine(n=16, p=2, tau_mode="const", tau_c=1.0):
    f = nodal(sine_f, n, p)[None]
    gD = np.zeros((1, p + 1, n_edges(n)))
    return Workload(f"poisson_sine_{n}_p{p}", n, p, np.zeros(n * n), f, gD, tau_mode, tau_c)


def example1(n, p, tau_mode="over_h", tau_c=1.0):
    f = nodal(ex1_f, n, p)[None]
    gD = dirichlet(ex1_u, n, p)[None]
    return Workload(f"example1_{n}_p{p}", n, p, np.zeros(n * n), f, gD, tau_mode, tau_c)


def lognormal(n=256, p=4, sigma=1.0, seed=2, tau_mode="over_h", tau_c=1.0, nrhs=1):
    rng = np.random.default_rng(seed)
    logk = rng.normal(0.0, sigma, size=n * n)
    f = np.ones((nrhs, (p + 1) ** 2, n * n))
    gD = np.zeros((nrhs, p + 1, n_edges(n)))
    return Workload(f"lognormal_{n}_p{p}_s{seed}", n, p, logk, f, gD, tau_mode, tau_c, seed=seed)


def ex3_kappa(x, y):
    return 1.0 + 0.5 * np.sin(2 * np.pi * x) * np.cos(3 * np.pi * y)


def ex3_f(x, y):
    """-div(kappa grad u) = kappa (-lap u) + grad kappa . q with q = -grad u."""
    gx = np.pi * np.cos(2 * np.pi * x) * np.cos(3 * np.pi * y)
    gy = -1.5 * np.pi * np.sin(2 * np.pi * x) * np.sin(3 * np.pi * y)
    qx, qy = ex1_q(x, y)
    return ex3_kappa(x, y) * ex1_f(x, y) + gx * qx + gy * qy


def example3(n, p, tau_mode="over_h", tau_c=1.0):
    """Example III on the unit square: kappa sampled at element centres."""
    j, i = np.divmod(np.arange(n * n), n)
    logk = np.log(ex3_kappa((i + 0.5) / n, (j + 0.5) / n))
    f = nodal(ex3_f, n, p)[None]
    gD = dirichlet(ex1_u, n, p)[None]
    return Workload(f"example3_{n}_p{p}", n, p, logk, f, gD, tau_mode, tau_c)


def checkerboard(n, p, tau_mode="over_h", tau_c=1.0):
    """Example IV: kappa = 1e6 on (0,0.56)^2 and (0.56,1)^2, else 1.

    Element centres decide the block."""
    j, i = np.divmod(np.arange(n * n), n)
    xc = (i + 0.5) / n
    yc = (j + 0.5) / n
    hi = ((xc < 0.56) & (yc < 0.56)) | ((xc > 0.56) & (yc > 0.56))
    logk = np.where(hi, math.log(1e6), 0.0)
    f = np.ones((1, (p + 1) ** 2, n * n))
    gD = np.zeros((1, p + 1, n_edges(n)))
    return Workload(f"checkerboard_{n}_p{p}", n, p, logk, f, gD, tau_mode, tau_c)


def convdiff_f(eps, beta):
    """f = -eps lap u + beta.grad u for u = sin(pi x) sin(pi y)."""
    def f(x, y):
        return (2.0 * np.pi ** 2 * eps * np.sin(np.pi * x) * np.sin(np.pi * y)
                + beta[0] * np.pi * np.cos(np.pi * x) * np.sin(np.pi * y)
                + beta[1] * np.pi * np.sin(np.pi * x) * np.cos(np.pi * y))
    return f


def convdiff(n=512, p=6, eps=1e-3, beta=(1.0, 0.5), nrhs=1):
    """Convection-diffusion with a manufactured smooth solution: eps = 1e-3,
    beta = (1, 0.5) on 512 x 512 quads at p = 6 by default."""
    f = np.repeat(nodal(convdiff_f(eps, beta), n, p)[None], nrhs, axis=0)
    gD = np.zeros((nrhs, p + 1, n_edges(n)))
    return Workload(f"convdiff_{n}_p{p}", n, p, np.full(n * n, math.log(eps)), f, gD,
                    "over_h", eps, beta=tuple(float(b) for b in beta))


def random_vectors(n, nd, count, seed):
    """Seeded N(0,1) trace vectors [count][nd][n_edges] (for operator checks)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((count, nd, n_edges(n)))


def batched(nprob=64, nrhs=16, seed=4, sizes=(32, 64, 128, 256), orders=(2, 4, 8), sigma=0.5):
    """Independent diffusion problems: n uniform from `sizes`, p uniform from
    `orders`, log kappa iid N(0, sigma^2) per element, `nrhs` forcing
    right-hand sides with iid N(0, 1) nodal values, g_D = 0, tau = 1/h."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(nprob):
        n = int(rng.choice(sizes))
        p = int(rng.choice(orders))
        logk = rng.normal(0.0, sigma, size=n * n)
        f = rng.standard_normal((nrhs, (p + 1) ** 2, n * n))
        out.append(Workload(f"batch{k}_{n}_p{p}", n, p, logk, f,
                            np.zeros((nrhs, p + 1, n_edges(n))), "over_h", 1.0, seed=seed))
    return out


# --------------------------------------------------------------------------
# unstructured quadrilateral meshes
# --------------------------------------------------------------------------
def umesh(nx, ny, lx=1.0, ly=1.0, jitter=0.2, holes=(), seed=0):
    """Seeded unstructured all-quadrilateral mesh of [0, lx] x [0, ly].

    An nx x ny grid whose interior vertices are moved by up to
    ``jitter`` x the cell size in each direction; every cell is cut into two
    triangles along a randomly chosen diagonal; triangles whose centroid lies
    in one of the ``holes`` (disks (cx, cy, r)) are removed; every remaining
    triangle is split into three quadrilaterals through its edge midpoints and
    centroid.  The result is conforming, with vertices of valence 3 to 8.
    Returns verts [n_vert, 2] float64 and quads [E, 4] int32, each element
    counter-clockwise."""
    rng = np.random.default_rng(seed)
    hx, hy = lx / nx, ly / ny
    gx, gy = np.meshgrid(np.linspace(0.0, lx, nx + 1), np.linspace(0.0, ly, ny + 1))
    P = np.stack([gx.ravel(), gy.ravel()], axis=1)
    d = rng.uniform(-jitter, jitter, size=P.shape) * np.array([hx, hy])
    inner = ((P[:, 0] > 0) & (P[:, 0] < lx) & (P[:, 1] > 0) & (P[:, 1] < ly))
    P[inner] += d[inner]
    diag = rng.integers(0, 2, size=(ny, nx))
    tris = []
    for j in range(ny):
        for i in range(nx):
            v00 = j * (nx + 1) + i
            v10, v01, v11 = v00 + 1, v00 + nx + 1, v00 + nx + 2
            if diag[j, i]:
                tris += [(v00, v10, v11), (v00, v11, v01)]
            else:
                tris += [(v00, v10, v01), (v10, v11, v01)]
    keep = []
    for t in tris:
        c = P[list(t)].mean(axis=0)
        if all((c[0] - hx0) ** 2 + (c[1] - hy0) ** 2 >= r * r for hx0, hy0, r in holes):
            keep.append(t)
    verts = [tuple(p) for p in P]
    mid = {}

    def midpoint(a, b):
        k = (min(a, b), max(a, b))
        if k not in mid:
            mid[k] = len(verts)
            verts.append(tuple(0.5 * (P[a] + P[b])))
        return mid[k]

    quads = []
    for a, b, c in keep:
        mab, mbc, mca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
        g = len(verts)
        verts.append(tuple(P[[a, b, c]].mean(axis=0)))
        quads += [(a, mab, g, mca), (b, mbc, g, mab), (c, mca, g, mbc)]
    verts = np.array(verts, dtype=np.float64)
    quads = np.array(quads, dtype=np.int64)
    used = np.unique(quads)
    remap = -np.ones(len(verts), dtype=np.int64)
    remap[used] = np.arange(len(used))
    return verts[used], remap[quads].astype(np.int32)


EXAMPLE2_HOLES = tuple((0.25 + 0.5 * i, 0.25 + 0.5 * j, 0.1) for j in range(2) for i in range(4))
EXAMPLE2_SEEDS_7 = ((0.2, 0.3), (0.5, 0.75), (0.75, 0.25), (1.0, 0.6), (1.3, 0.3),
                    (1.5, 0.75), (1.8, 0.4))
EXAMPLE2_SEEDS_4 = ((0.3, 0.5), (0.8, 0.3), (1.25, 0.7), (1.7, 0.45))


def example2(n, p, seeds=7, seed=0):
    """Stand-in for Example II (Sec. 4.2): a 2 x 1 box with eight circular
    holes meshed by ``umesh`` (2n x n cells, about 12 n^2 quadrilaterals),
    kappa = 1, f = 1, zero Dirichlet data, 7 or 4 seed points spread over the
    box.  Returns (verts, quads, seeds, log_kappa [E], f [E][(p+1)^2])."""
    verts, quads = umesh(2 * n, n, 2.0, 1.0, 0.2, EXAMPLE2_HOLES, seed)
    sp = np.array(EXAMPLE2_SEEDS_7 if seeds == 7 else EXAMPLE2_SEEDS_4, dtype=np.float64)
    E = len(quads)
    return verts, quads, sp, np.zeros(E), np.ones((E, (p + 1) ** 2))


def seed_grid(nx, ny, lx=2.0, ly=1.0):
    """nx x ny seed points at the centres of a regular grid of the box, so
    that every level-1 macro-element holds about the same number of elements
    (the paper's criterion for placing seeds)."""
    xs = (np.arange(nx) + 0.5) * lx / nx
    ys = (np.arange(ny) + 0.5) * ly / ny
    return np.array([(x, y) for y in ys for x in xs], dtype=np.float64)
