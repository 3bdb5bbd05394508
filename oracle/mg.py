"""DtN-based geometric multigrid on global sparse matrices (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Restates Sec. 3 of arXiv:1811.09909 with every operator formed as a global
sparse matrix, in the order the paper defines them:

* Sec. 3.1.1 p-coarsening: level N carries P_p traces, level N-1 the same
  mesh with P_1 traces; J_N embeds P_1 in P_p (in the orthonormal Legendre
  basis: the first two modes), I_N = J_N, Q_{N-1} = J_N^*  (eqs. n_g1_Ik,
  n_g1_Qk), A_{N-1} = J_N^* A_N J_N (eq. ANm1).
* Sec. 3.1.2 h-coarsening by agglomerating 2 x 2 macro-elements: edges of
  level k split into E_{k,I} (inside a level k-1 macro-element) and E_{k,B}
  (eq. trace_partition); J_k injects the P_1 trace of each coarse macro-edge
  into its two halves (computed here by quadrature as the L2 projection, which
  is exact because P_1 restricted to a half is P_1);
  I_k = [-A_II^-1 A_IB J_k ; J_k]  (eq. n_1_Ik),
  Q_{k-1} = [-J_k^* A_BI A_II^-1 , J_k^*]  (eq. n_1_Qk),
  A_{k-1} = Q_{k-1} A_k I_k  (eq. coarse), formed as a sparse triple product.
  A_II^-1 is found by splitting A_II into the connected components of its
  sparsity graph and inverting each dense component.
* Sec. 3.3 smoothing steps m_{k-1} = beta m_k (beta = 2 in Sec. 4; optionally
  capped); Sec. 4.1 smoothers: block-Jacobi with one block per edge
  (undamped by default), damped point-Jacobi (omega = 2/3 in the paper),
  Chebyshev-accelerated point-Jacobi on [Lambda_max / 30, Lambda_max] with
  Lambda_max from a power iteration on D^-1 A, and LU-SGS (one forward and
  one backward point Gauss-Seidel sweep per step).  The Gauss-Seidel order is
  multicolour by edge: vertical edges with even column, vertical odd,
  horizontal with even row, horizontal odd (edges of one colour share no
  element), then edge number, then mode; the paper does not state its order.
* Sec. 3.4 local correction T_k = diag(A_II^-1, 0) (eq. localCorrection).
* Sec. 3.6 Algorithm 1 (V-cycle) with B_1 = A_1^-1 by a dense Cholesky
  factorisation (a dense LU with partial pivoting for the non-symmetric
  convection-diffusion operator), local correction in step 3 only ("pre", the paper's
  choice), in steps 3 and 5 ("both", symmetric, for CG) or nowhere ("none").

In the orthonormal trace bases used here the L2(E_k) adjoint J_k^* is the
transpose J_k^T, so operator and matrix forms coincide.

Dirichlet edges are removed from every level (homogeneous error equations);
all vectors live on the free (interior) trace dofs in edge-major order.

Pins (tests/test_oracle_mg.py): Galerkin identity vs a dense global Schur
complement (Proposition "DtN": A_{k-1} is the Schur complement after
eliminating all traces interior to level k-1 macro-elements), energy
preservation (Proposition "Energy preservation"), Q_{k-1} = I_k^T for
symmetric A, coarse operators annihilating traces of linear functions on
interior rows, V-cycle contraction, h-independent iteration counts against
the bands of the paper's Example I tables, divergence without local correction
at p = 1 (Example I, table without local correction).
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import scipy.sparse.csgraph as csgraph

from . import hdg as H
from . import refelem


def _free_dofs(n, nd, dirichlet=True):
    fe = np.nonzero(~H.boundary_edge_mask(n))[0] if dirichlet else np.arange(H.n_edges(n))
    return (fe[:, None] * nd + np.arange(nd)[None, :]).ravel()


def _position(n, nd, free):
    pos = -np.ones(H.n_edges(n) * nd, dtype=np.int64)
    pos[free] = np.arange(len(free))
    return pos


def _block_inverse(A):
    """Inverse of a sparse matrix that is block diagonal up to permutation:
    connected components of its graph, dense inverse of each component."""
    A = sp.csr_matrix(A)
    ncomp, labels = csgraph.connected_components(A, directed=False)
    order = np.argsort(labels, kind="stable")
    counts = np.bincount(labels, minlength=ncomp)
    rows, cols, vals = [], [], []
    # group components by size for a batched inverse
    starts = np.concatenate([[0], np.cumsum(counts)])
    by_size = {}
    for c in range(ncomp):
        by_size.setdefault(counts[c], []).append(c)
    Acsr = A.tocsr()
    for size, comps in by_size.items():
        idx = np.stack([order[starts[c]:starts[c] + size] for c in comps])   # [nc, size]
        blocks = np.zeros((len(comps), size, size))
        for a in range(size):
            for b in range(size):
                blocks[:, a, b] = np.asarray(Acsr[idx[:, a], idx[:, b]]).ravel()
        inv = np.linalg.inv(blocks)
        rows.append(np.repeat(idx, size, axis=1).ravel())
        cols.append(np.tile(idx, (1, size)).ravel())
        vals.append(inv.ravel())
    n = A.shape[0]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def child_injection():
    """J for one macro-edge: [child c][fine mode l][coarse mode k] (P1 -> P1),
    by quadrature of  int_child psi^child_l psi^macro_k  with |macro| = 2."""
    s, w = refelem.gauss(6)
    Jc = np.zeros((2, 2, 2))
    for c in range(2):
        t = (s - 1.0) / 2.0 if c == 0 else (s + 1.0) / 2.0
        psi_f = refelem.trace_basis(1, s, 1.0)     # child of length 1
        psi_c = refelem.trace_basis(1, t, 2.0)     # macro of length 2
        Jc[c] = (psi_f * w * 0.5) @ psi_c.T        # ds_phys = (1/2) ds
    return Jc


class Level:
    pass


SMOOTHERS = ("block_jacobi", "point_jacobi", "chebyshev", "lu_sgs")
POWER_ITERS = 30          # power iterations for Lambda_max (Chebyshev)


def power_start(n, nd, free):
    """Deterministic start vector of the power iteration on the free dofs:
    dof (edge e, mode k) of a mesh with E edges gets 1 + (h mod 1024) / 1024,
    h = (i * 2654435761) mod 2^32 with i = k E + e (the library's layout
    index).  Shared definition, so both sides start from the same vector."""
    ne = H.n_edges(n)
    e, k = np.divmod(free, nd)
    i = (k * ne + e).astype(np.uint64)
    h = (i * np.uint64(2654435761)) % np.uint64(1 << 32)
    return 1.0 + (h % np.uint64(1024)).astype(np.float64) / 1024.0


def lambda_max_power(A, dinv, x0, iters=POWER_ITERS):
    """Largest eigenvalue of D^-1 A by power iteration: x <- y / |y|,
    y = D^-1 A x, estimate |y| for the unit x of the last step."""
    x = x0 / np.linalg.norm(x0)
    lam = 0.0
    for _ in range(iters):
        y = dinv * (A @ x)
        lam = np.linalg.norm(y)
        x = y / lam
    return lam


def colour_order(n, nd, free):
    """Positions of the free dofs in LU-SGS order (colour, edge, mode)."""
    nvert = n * (n + 1)
    e, k = np.divmod(free, nd)
    vert = e < nvert
    col = np.where(vert, (e % (n + 1)) % 2, 2 + ((e - nvert) // n) % 2)
    return np.lexsort((k, e, col))


class Hierarchy:
    """Multigrid hierarchy built from the fine trace system of an HDGProblem.

    Parameters follow the library's options: coarsest_n (stop agglomerating
    at n <= coarsest_n), m_fine, m_growth (beta), m_max, local_corr in
    {"none", "pre", "both"}, omega (block-Jacobi damping, 1 = undamped).
    dirichlet=False keeps the boundary edges as unknowns on every level (the
    pure-Neumann operators, singular; used only to check the hierarchy)."""

    def __init__(self, problem, Ae=None, coarsest_n=2, m_fine=1, m_growth=2, m_max=None,
                 local_corr="pre", omega=1.0, dirichlet=True, smoother="block_jacobi"):
        if smoother not in SMOOTHERS:
            raise ValueError(f"unknown smoother {smoother}")
        self.smoother = smoother
        self.problem = problem
        self.dirichlet = dirichlet
        self.local_corr = local_corr
        self.omega = omega
        if Ae is None:
            Ae, _ = problem.condense()
        A_full = problem.assemble(Ae)
        n, p = problem.n, problem.p
        free = _free_dofs(n, p + 1, dirichlet)
        levels = []
        L = Level()
        L.n, L.nd, L.free = n, p + 1, free
        L.A = A_full[free][:, free].tocsr()
        levels.append(L)
        Jc = child_injection()
        self.Jc = Jc
        # p-coarsening
        if p > 1:
            Lc = Level()
            Lc.n, Lc.nd = n, 2
            Lc.free = _free_dofs(n, 2, dirichlet)
            fpos = _position(n, p + 1, L.free)
            fe = Lc.free // 2
            mode = Lc.free % 2
            rows = fpos[fe * (p + 1) + mode]
            J = sp.csr_matrix((np.ones(len(rows)), (rows, np.arange(len(rows)))),
                              shape=(len(L.free), len(Lc.free)))
            L.kind = "p"
            L.I = J
            L.Q = J.T.tocsr()
            L.T = None
            Lc.A = (L.Q @ L.A @ L.I).tocsr()
            levels.append(Lc)
            L = Lc
        # h-coarsening
        while L.n > coarsest_n:
            if L.n % 2:
                raise ValueError("mesh size must halve evenly down to coarsest_n")
            self._h_coarsen(L, levels)
            L = levels[-1]
        # smoothing schedule
        m = m_fine
        for lev in levels:
            lev.m = m
            m = m * m_growth
            if m_max is not None:
                m = min(m, m_max)
        for lev in levels:
            lev.Dinv = self._block_jacobi(lev) if dirichlet else None
            if dirichlet and lev.A.shape[0]:
                self._smoother_setup(lev)
        coarse = levels[-1]
        coarse.chol = coarse.lu = None
        if coarse.A.shape[0] and dirichlet:
            if problem.symmetric:
                coarse.chol = sla.cho_factor(coarse.A.toarray())
            else:
                coarse.lu = sla.lu_factor(coarse.A.toarray())
        self.levels = levels

    # ------------------------------------------------------------------
    def _h_coarsen(self, L, levels):
        n = L.n
        nc = n // 2
        nvf = n * (n + 1)
        edges = np.arange(H.n_edges(n))
        is_int = np.where(edges < nvf, (edges % (n + 1)) % 2 == 1, ((edges - nvf) // n) % 2 == 1)
        fe = L.free // 2
        Iset = np.nonzero(is_int[fe])[0]               # positions in free ordering
        Bset = np.nonzero(~is_int[fe])[0]
        Lc = Level()
        Lc.n, Lc.nd = nc, 2
        Lc.free = _free_dofs(nc, 2, self.dirichlet)
        cpos = _position(nc, 2, Lc.free)
        # J_k: fine B dofs <- coarse dofs (child injection of each macro-edge)
        rows, cols, vals = [], [], []
        nvc = nc * (nc + 1)
        Jc = self.Jc
        for bpos, fdof in zip(Bset, L.free[Bset]):
            e, l = divmod(fdof, 2)
            if e < nvf:
                j, i = divmod(e, n + 1)                 # vertical edge (i, j), i even
                ce = (j // 2) * (nc + 1) + i // 2
                c = j % 2
            else:
                j, i = divmod(e - nvf, n)               # horizontal edge (i, j), j even
                ce = nvc + (j // 2) * nc + i // 2
                c = i % 2
            for k in range(2):
                cp = cpos[ce * 2 + k]
                if cp >= 0:
                    rows.append(bpos)
                    cols.append(cp)
                    vals.append(Jc[c, l, k])
        nfree = len(L.free)
        J = sp.csr_matrix((vals, (rows, cols)), shape=(nfree, len(Lc.free)))  # rows on B
        PI = sp.csr_matrix((np.ones(len(Iset)), (np.arange(len(Iset)), Iset)), shape=(len(Iset), nfree))
        PB = sp.csr_matrix((np.ones(len(Bset)), (np.arange(len(Bset)), Bset)), shape=(len(Bset), nfree))
        A = L.A
        AII = PI @ A @ PI.T
        AIB = PI @ A @ PB.T
        ABI = PB @ A @ PI.T
        JB = PB @ J                                     # J_k on the B block
        AIIinv = _block_inverse(AII)
        # I_k = [ -A_II^-1 A_IB J ; J ]   (eq. n_1_Ik)
        Ik = PI.T @ (-(AIIinv @ (AIB @ JB))) + PB.T @ JB
        # Q_{k-1} = [ -J^T A_BI A_II^-1 , J^T ]   (eq. n_1_Qk)
        Qk = (-(JB.T @ ABI @ AIIinv)) @ PI + JB.T @ PB
        L.kind = "h"
        L.I = sp.csr_matrix(Ik)
        L.Q = sp.csr_matrix(Qk)
        L.Iset = Iset
        L.AIIinv = AIIinv
        L.T = PI.T @ AIIinv @ PI                        # diag(A_II^-1, 0)
        Lc.A = (L.Q @ A @ L.I).tocsr()                  # eq. coarse
        levels.append(Lc)

    def _smoother_setup(self, L):
        A = L.A.tocsr()
        L.dpt = 1.0 / A.diagonal()
        if self.smoother == "chebyshev":
            L.lmax = lambda_max_power(A, L.dpt, power_start(L.n, L.nd, L.free))
        if self.smoother == "lu_sgs":
            order = colour_order(L.n, L.nd, L.free)
            P = sp.csr_matrix((np.ones(len(order)), (np.arange(len(order)), order)),
                              shape=(len(order), len(order)))
            Ap = (P @ A @ P.T).tocsr()
            L.gs_P = P
            L.gs_lower = sp.tril(Ap, 0).tocsr()        # D + L in colour order
            L.gs_upper = sp.triu(Ap, 0).tocsr()        # D + U

    def smooth(self, L, r, e, steps):
        """`steps` smoothing iterations on A e = r from e."""
        A = L.A
        for _ in range(steps) if self.smoother != "chebyshev" else range(1):
            if self.smoother == "block_jacobi":
                e = e + self.omega * (L.Dinv @ (r - A @ e))
            elif self.smoother == "point_jacobi":
                e = e + self.omega * L.dpt * (r - A @ e)
            elif self.smoother == "lu_sgs":
                P = L.gs_P
                res = P @ (r - A @ e)
                e = e + P.T @ spla.spsolve_triangular(L.gs_lower, res, lower=True)
                res = P @ (r - A @ e)
                e = e + P.T @ spla.spsolve_triangular(L.gs_upper, res, lower=False)
        if self.smoother == "chebyshev":
            lmax = L.lmax
            lmin = lmax / 30.0
            theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
            sigma = theta / delta
            rho = 1.0 / sigma
            d = L.dpt * (r - A @ e) / theta
            e = e + d
            for _ in range(steps - 1):
                rho_new = 1.0 / (2.0 * sigma - rho)
                d = rho_new * rho * d + (2.0 * rho_new / delta) * L.dpt * (r - A @ e)
                e = e + d
                rho = rho_new
        return e

    @staticmethod
    def _block_jacobi(L):
        nd = L.nd
        A = L.A.tocoo()
        nb = A.shape[0] // nd
        blocks = np.zeros((nb, nd, nd))
        m = (A.row // nd) == (A.col // nd)
        blocks[A.row[m] // nd, A.row[m] % nd, A.col[m] % nd] = A.data[m]
        inv = np.linalg.inv(blocks) if nb else blocks
        r = np.repeat(np.arange(nb * nd).reshape(nb, nd), nd, axis=1).ravel()
        c = np.tile(np.arange(nb * nd).reshape(nb, nd), (1, nd)).ravel()
        return sp.csr_matrix((inv.ravel(), (r, c)), shape=A.shape)

    # ------------------------------------------------------------------
    def vcycle(self, r, k=0):
        """B_k r by Algorithm 1 (k = 0 is the finest level here)."""
        L = self.levels[k]
        if k == len(self.levels) - 1:
            if L.chol is not None:
                return sla.cho_solve(L.chol, r)
            return sla.lu_solve(L.lu, r) if L.lu is not None else np.zeros_like(r)
        A = L.A
        e = self.smooth(L, r, np.zeros_like(r), L.m)             # step 2
        if L.T is not None and self.local_corr in ("pre", "both"):
            e = e + L.T @ (r - A @ e)                            # step 3
        rc = L.Q @ (r - A @ e)                                   # step 4
        e = e + L.I @ self.vcycle(rc, k + 1)
        if L.T is not None and self.local_corr == "both":
            e = e + L.T @ (r - A @ e)                            # step 5
        return self.smooth(L, r, e, L.m)                         # step 6

    # ------------------------------------------------------------------
    # outer iterations (Sec. 3.6 and Sec. 4); b, x on the fine free dofs
    def solve_fixed_point(self, b, tol=1e-9, max_it=200):
        A = self.levels[0].A
        x = np.zeros_like(b)
        nb = np.linalg.norm(b)
        hist = []
        for it in range(1, max_it + 1):
            x = x + self.vcycle(b - A @ x)
            res = np.linalg.norm(b - A @ x) / nb
            hist.append(res)
            if not np.isfinite(res) or res > 1e8:
                return x, it, hist, False
            if res <= tol:
                return x, it, hist, True
        return x, max_it, hist, False

    def solve_pcg(self, b, tol=1e-10, max_it=200):
        A = self.levels[0].A
        x = np.zeros_like(b)
        r = b.copy()
        nb = np.linalg.norm(b)
        z = self.vcycle(r)
        pdir = z.copy()
        rz = r @ z
        hist = []
        for it in range(1, max_it + 1):
            Ap = A @ pdir
            alpha = rz / (pdir @ Ap)
            x = x + alpha * pdir
            r = r - alpha * Ap
            res = np.linalg.norm(r) / nb
            hist.append(res)
            if res <= tol:
                return x, it, hist, True
            z = self.vcycle(r)
            rz_new = r @ z
            pdir = z + (rz_new / rz) * pdir
            rz = rz_new
        return x, max_it, hist, False

    def solve_gmres(self, b, tol=1e-10, max_it=200, restart=30, left=False):
        """Restarted GMRES with the V-cycle as preconditioner.

        right (default): the residual it monitors is the true one;
        left=True: the paper's left preconditioning, monitoring ||B r||/||B b||."""
        A = self.levels[0].A
        x = np.zeros_like(b)
        nb = np.linalg.norm(self.vcycle(b)) if left else np.linalg.norm(b)
        total = 0
        hist = []
        while total < max_it:
            r = b - A @ x
            if left:
                r = self.vcycle(r)
            beta = np.linalg.norm(r)
            if beta / nb <= tol:
                return x, total, hist, True
            V = [r / beta]
            Z = []
            Hm = np.zeros((restart + 1, restart))
            g = np.zeros(restart + 1)
            g[0] = beta
            cs, sn = [], []
            j = 0
            for j in range(restart):
                if left:
                    w = self.vcycle(A @ V[j])
                    Z.append(V[j])
                else:
                    zj = self.vcycle(V[j])
                    Z.append(zj)
                    w = A @ zj
                for i in range(j + 1):
                    Hm[i, j] = w @ V[i]
                    w = w - Hm[i, j] * V[i]
                Hm[j + 1, j] = np.linalg.norm(w)
                V.append(w / Hm[j + 1, j] if Hm[j + 1, j] > 0 else w)
                for i in range(j):
                    t = cs[i] * Hm[i, j] + sn[i] * Hm[i + 1, j]
                    Hm[i + 1, j] = -sn[i] * Hm[i, j] + cs[i] * Hm[i + 1, j]
                    Hm[i, j] = t
                den = np.hypot(Hm[j, j], Hm[j + 1, j])
                cs.append(Hm[j, j] / den)
                sn.append(Hm[j + 1, j] / den)
                Hm[j, j] = den
                Hm[j + 1, j] = 0.0
                g[j + 1] = -sn[j] * g[j]
                g[j] = cs[j] * g[j]
                total += 1
                hist.append(abs(g[j + 1]) / nb)
                if abs(g[j + 1]) / nb <= tol or total >= max_it:
                    break
            y = sla.solve_triangular(Hm[:j + 1, :j + 1], g[:j + 1])
            for i in range(j + 1):
                x = x + y[i] * Z[i]
            res = (np.linalg.norm(self.vcycle(b - A @ x)) if left else np.linalg.norm(b - A @ x)) / nb
            if res <= tol:
                return x, total, hist, True
        return x, total, hist, False

    # helpers to move between the library layout and the free-dof vector
    def to_free(self, x_api, k=0):
        L = self.levels[k]
        return H.api_to_edge_major(x_api, L.n, L.nd)[L.free]

    def from_free(self, x, k=0):
        L = self.levels[k]
        full = np.zeros(H.n_edges(L.n) * L.nd)
        full[L.free] = x
        return H.edge_major_to_api(full, L.n, L.nd)
