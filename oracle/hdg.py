"""HDG discretisation, static condensation, direct solve and recovery (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Follows Sec. 2 of arXiv:1811.09909 with K = kappa*I per element:

  (HDG_local1)  (kappa^-1 q, v)_K - (u, div v)_K + <lambda, v.n>_dK = 0
  (HDG_local2)  -(q, grad w)_K + <qhat.n, w>_dK = (f, w)_K
  (HDG_flux)    qhat.n = q.n + tau (u - lambda)
  (conservation) sum_K <qhat.n, mu>_e = 0 on every interior edge e,

with lambda = g_D on boundary edges, "applied directly (strongly) via the
trace unknowns" (Example I, Sec. 4.1; reading: g_D is given as its L2
projection onto P_p per boundary edge).  Every bilinear form is integrated by
the over-integrating rule of ``refelem.RefQuad`` exactly in the form printed in
the paper (HDG_local2 is NOT integrated by parts here).

Static condensation (Sec. 2, last paragraph; Sec. 3, eq. trace_linear_system):
for each element the full local block L (3 n_v x 3 n_v, unknowns
z = [q_x, q_y, u]) is solved by a general LU with partial pivoting
(numpy.linalg.solve), giving

  z = L^-1 (F - R lambda),   A_e = C L^-1 R + tau E_lambda,   g_e = C L^-1 F,

where C lambda-tests the conservation flux and E_lambda is the trace mass
matrix (identity in the orthonormal trace basis).  The global trace system is
sum_e A_e lambda_e = sum_e g_e on interior edges.

Mesh and numbering (the library's documented layout, shared convention only):
uniform n x n rectangles on [x0,x1] x [y0,y1]; element e = j*n + i; vertical
edge at x_i between rows j: index j*(n+1) + i; horizontal edge at y_j:
n*(n+1) + j*n + i; element-local edges 0=left, 1=right, 2=bottom, 3=top.
Trace vectors handed in and out use the mode-major layout [mode][edge]; the
oracle works internally edge-major (dof = edge*(p+1) + mode).

Convection-diffusion (not in the paper; the library's stated extension):
-div(eps grad u) + div(beta u) = f with constant beta and eps = kappa per
element.  The flux variable stays q = -eps grad u; HDG_local2 becomes
  -(q + beta u, grad w)_K + <hhat.n, w>_dK = (f, w)_K,
  hhat.n = q.n + (beta.n) lambda + tau_f (u - lambda),
and the conservation condition sums <hhat.n, mu> over both sides of every
interior edge.  tau_f = tau_e + max(beta.n_f, 0) on face f (upwinding: on
outflow faces the total flux uses the interior u).  The local block is no
longer symmetric; the same general LU condenses it into
  A_e = C L^-1 R - T,  T = sum_f (beta.n_f - tau_f) El_f.
With beta = 0 this is the diffusion element (T = -tau El).

Hybridized interior penalty schemes (Sec. 2, eqs. IPDG_flux, SIPG_H,
IPG_H): the primal local problem in u alone,
  (kappa grad u, grad w)_K - s_f <u - lambda, kappa grad w.n>_dK
      - <kappa grad u.n, w>_dK + <tau (u - lambda), w>_dK = (f, w)_K,
with the flux uhat.n = -kappa grad u.n + tau (u - lambda) in the same
conservation condition; s_f = 1 (SIPG-H), -1 (NIPG-H), 0 (IIPG-H).  The
local block L (n_v x n_v) is condensed by the same general LU; the recovered
flux is q = -kappa grad u_h at the volume nodes (reading: the primal schemes
have no separate flux unknown).

Pins (tests/test_oracle_hdg.py): polynomial patch test (exact to roundoff),
O(h^{p+1}) rates for u and q, A_e 1 = 0, A_e symmetric PSD, homogeneity
A_e(c kappa, c tau) = c A_e, SPD global trace operator, condensed solve equal
to a dense uncondensed solve, closed-form 1x1 p=0 element.
Convection-diffusion (tests/test_oracle_convdiff.py): the general path with
beta = 0 equals the diffusion path; linear and quadratic patch tests with
convection (exact to roundoff); the closed form A_e 1 = <beta.n, mu>;
positive-definite symmetric part of the global trace operator (the upwind
tau); O(h^{p+1}) rates for u; condensed solve equal to the dense uncondensed
solve.
IPDG-H (tests/test_oracle_ipdg.py): Q_p patch tests for the three schemes
(exact to roundoff), SIPG-H symmetric and positive semi-definite with
A_e 1 = 0, the NIPG-H energy identity (the s_f terms cancel), condensed equal
to uncondensed solves, O(h^{p+1}) / O(h^p) rates, and the paper's NIPG-H
iteration tables for Example I (tests/golden/paper_example1_iterations.txt).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import refelem


# --------------------------------------------------------------------------
# mesh topology
# --------------------------------------------------------------------------
def n_edges(n):
    return 2 * n * (n + 1)


def element_edges(n):
    """[n*n, 4] global edge indices (left, right, bottom, top) of each element."""
    j, i = np.divmod(np.arange(n * n), n)
    nv = n * (n + 1)
    left = j * (n + 1) + i
    right = j * (n + 1) + i + 1
    bottom = nv + j * n + i
    top = nv + (j + 1) * n + i
    return np.stack([left, right, bottom, top], axis=1)


def boundary_edge_mask(n):
    """True for edges on the domain boundary (Dirichlet edges)."""
    e = np.arange(n_edges(n))
    nv = n * (n + 1)
    mask = np.zeros(len(e), dtype=bool)
    vi = e[:nv] % (n + 1)
    mask[:nv] = (vi == 0) | (vi == n)
    hj = (e[nv:] - nv) // n
    mask[nv:] = (hj == 0) | (hj == n)
    return mask


def api_to_edge_major(x, n, nd):
    """[nd][n_edges] (library layout) -> [n_edges*nd] edge-major vector."""
    return np.ascontiguousarray(np.asarray(x).reshape(nd, n_edges(n)).T).ravel()


def edge_major_to_api(x, n, nd):
    return np.ascontiguousarray(np.asarray(x).reshape(n_edges(n), nd).T)


# --------------------------------------------------------------------------
# element operators
# --------------------------------------------------------------------------
class ElementForms:
    """Reference bilinear forms of one element (size hx x hy), split by how
    they depend on kappa^-1 and tau so that L = L0 + kappa^-1 LM + tau Lt."""

    def __init__(self, p, hx, hy, nq=None, quad=None):
        """quad: an element with the RefQuad table interface (volume_tables,
        edge_tables) in place of the hx x hy rectangle, e.g. a mapped
        quadrilateral; the primal (IPDG-H) pieces are then not formed."""
        self.p = p
        rq = refelem.RefQuad(p, hx, hy, nq) if quad is None else quad
        self.rq = rq
        nv = rq.nv
        nt = 4 * (p + 1)
        self.nv, self.nt = nv, nt
        phi, dphidx, dphidy, wJ = rq.volume_tables()
        Mv = (phi * wJ) @ phi.T                     # (phi_b, phi_a)
        Dx = (dphidx * wJ) @ phi.T                  # Dx[a, b] = (phi_b, d_x phi_a)
        Dy = (dphidy * wJ) @ phi.T
        Ex = np.zeros((nv, nv))                     # <phi_b n_x, phi_a>
        Ey = np.zeros((nv, nv))
        Eb = np.zeros((nv, nv))                     # <phi_b, phi_a>_dK
        Cx = np.zeros((nv, nt))                     # <psi_k, phi_a n_x>
        Cy = np.zeros((nv, nt))
        Fb = np.zeros((nv, nt))                     # <psi_k, phi_a>
        El = np.zeros((nt, nt))                     # <psi_l, psi_k>
        # per-face pieces for face-dependent tau and the convective flux
        self.Eb_f = np.zeros((4, nv, nv))
        self.Fb_f = np.zeros((4, nv, nt))
        self.El_f = np.zeros((4, nt, nt))
        self.normals = np.zeros((4, 2))
        for edge in range(4):
            ph, psi, wds, (nx, ny) = rq.edge_tables(edge)
            sl = slice(edge * (p + 1), (edge + 1) * (p + 1))
            mass_vv = (ph * wds) @ ph.T
            mass_vt = (ph * wds) @ psi.T
            Ex += nx * mass_vv
            Ey += ny * mass_vv
            Eb += mass_vv
            Cx[:, sl] += nx * mass_vt
            Cy[:, sl] += ny * mass_vt
            Fb[:, sl] += mass_vt
            El[sl, sl] += (psi * wds) @ psi.T
            self.Eb_f[edge] = mass_vv
            self.Fb_f[edge][:, sl] = mass_vt
            self.El_f[edge][sl, sl] = (psi * wds) @ psi.T
            self.normals[edge] = (nx, ny)
        self.Dx, self.Dy = Dx, Dy
        self.Cx, self.Cy = Cx, Cy
        # primal (IPDG-H) pieces: stiffness (grad phi_b, grad phi_a), the
        # boundary terms N[a, b] = <phi_b, grad phi_a.n> and
        # Hn[a, k] = <psi_k, grad phi_a.n>
        self.Kst = (dphidx * wJ) @ dphidx.T + (dphidy * wJ) @ dphidy.T
        if quad is None:
            self.Nn = np.zeros((nv, nv))
            self.Hn = np.zeros((nv, nt))
            for edge in range(4):
                ph, psi, wds, _ = rq.edge_tables(edge)
                dn = rq.edge_normal_derivative(edge)
                sl = slice(edge * (p + 1), (edge + 1) * (p + 1))
                self.Nn += (dn * wds) @ ph.T
                self.Hn[:, sl] += (dn * wds) @ psi.T
            self.Gx, self.Gy = rq.nodal_gradient()
        Z = np.zeros((nv, nv))
        # rows: [HDG_local1 x-test, HDG_local1 y-test, HDG_local2]
        self.LM = np.block([[Mv, Z, Z], [Z, Mv, Z], [Z, Z, Z]])
        self.L0 = np.block([[Z, Z, -Dx], [Z, Z, -Dy],
                            [-Dx + Ex, -Dy + Ey, Z]])
        self.Lt = np.block([[Z, Z, Z], [Z, Z, Z], [Z, Z, Eb]])
        # lambda columns: R = R0 + tau Rt
        self.R0 = np.vstack([Cx, Cy, np.zeros((nv, nt))])
        self.Rt = np.vstack([np.zeros((nv, nt)), np.zeros((nv, nt)), -Fb])
        # conservation rows: C = C0 + tau Ct, lambda term -tau El
        self.C0 = np.hstack([Cx.T, Cy.T, np.zeros((nt, nv))])
        self.Ct = np.hstack([np.zeros((nt, nv)), np.zeros((nt, nv)), Fb.T])
        self.El = El
        self.Mv = Mv

    def local(self, kappa, tau):
        L = self.L0 + self.LM / kappa + tau * self.Lt
        R = self.R0 + tau * self.Rt
        C = self.C0 + tau * self.Ct
        return L, R, C

    def local_cd(self, kappa, tau_f, beta):
        """Convection-diffusion local block with per-face tau_f [4]:
        returns L, R, C, T (conservation rows C z + T lambda)."""
        nv, nt = self.nv, self.nt
        Z = np.zeros((nv, nv))
        bn = self.normals @ np.asarray(beta, dtype=np.float64)        # beta.n_f
        Euu = sum(tau_f[f] * self.Eb_f[f] for f in range(4))
        conv = -(beta[0] * self.Dx + beta[1] * self.Dy)                # -(beta u, grad w)
        L = self.L0 + self.LM / kappa + np.block([[Z, Z, Z], [Z, Z, Z], [Z, Z, Euu + conv]])
        Rl = sum((bn[f] - tau_f[f]) * self.Fb_f[f] for f in range(4))  # <(beta.n - tau) lambda, w>
        R = self.R0 + np.vstack([np.zeros((2 * nv, nt)), Rl])
        Cu = sum(tau_f[f] * self.Fb_f[f] for f in range(4)).T         # <tau u, mu>
        C = np.hstack([self.Cx.T, self.Cy.T, Cu])
        T = sum((bn[f] - tau_f[f]) * self.El_f[f] for f in range(4))
        return L, R, C, T

    def local_ipdg(self, kappa, tau, sf):
        """IPDG-H local block of eq. IPG_H (u only): L u + R lambda = M f and
        conservation rows C u + T lambda."""
        L = kappa * (self.Kst - sf * self.Nn - self.Nn.T) + tau * self.Eb_sum()
        R = sf * kappa * self.Hn - tau * self.Fb_sum()
        C = (-kappa * self.Hn + tau * self.Fb_sum()).T
        T = -tau * self.El
        return L, R, C, T

    def Eb_sum(self):
        return self.Eb_f.sum(axis=0)

    def Fb_sum(self):
        return self.Fb_f.sum(axis=0)

    def load(self, fnodal):
        """F = [0, 0, (f_h, phi_a)] for the Q_p interpolant of nodal f."""
        nv = self.nv
        F = np.zeros(3 * nv)
        F[2 * nv:] = self.Mv @ fnodal
        return F


class HDGProblem:
    """HDG trace system on a uniform n x n rectangle mesh (oracle).

    kappa: per-element diffusivity [n*n] (K = kappa I); tau: scalar or [n*n].
    beta: None (diffusion) or a constant convection velocity (bx, by); then
    tau is the base value and face f of element e uses
    tau_e + max(beta.n_f, 0).
    scheme: "hdg" (Sec. 2, eqs. HDG_local1/2) or one of the hybridized
    interior penalty schemes "sipg", "nipg", "iipg" (eq. IPG_H with
    s_f = 1, -1, 0; diffusion only).
    """

    SCHEMES = {"sipg": 1.0, "nipg": -1.0, "iipg": 0.0}

    def __init__(self, n, p, kappa, tau, x0=0.0, x1=1.0, y0=0.0, y1=1.0, nq=None, beta=None,
                 scheme="hdg"):
        self.n, self.p = n, p
        self.E = n * n
        self.hx = (x1 - x0) / n
        self.hy = (y1 - y0) / n
        self.x0, self.y0 = x0, y0
        self.kappa = np.broadcast_to(np.asarray(kappa, dtype=np.float64), (self.E,)).copy()
        self.tau = np.broadcast_to(np.asarray(tau, dtype=np.float64), (self.E,)).copy()
        self.forms = ElementForms(p, self.hx, self.hy, nq)
        self.nv, self.nt = self.forms.nv, self.forms.nt
        self.nd = p + 1
        self.ne = n_edges(n)
        self.edges = element_edges(n)
        self.bmask = boundary_edge_mask(n)
        self._Ae = None
        self._ge_f = None
        self.beta = None if beta is None else np.asarray(beta, dtype=np.float64)
        if scheme != "hdg" and scheme not in self.SCHEMES:
            raise ValueError(f"unknown scheme {scheme}")
        if scheme != "hdg" and self.beta is not None:
            raise ValueError("the interior penalty schemes are diffusion only")
        self.scheme = scheme
        self.ipdg = scheme != "hdg"
        self.sf = self.SCHEMES.get(scheme)
        self.symmetric = self.beta is None and scheme in ("hdg", "sipg")
        if self.beta is not None:
            bn = self.forms.normals @ self.beta
            self.tau_f = self.tau[:, None] + np.maximum(bn, 0.0)[None, :]

    def local(self, e):
        """(L, R, C, T) of element e: conservation rows read C z + T lambda."""
        fr = self.forms
        if self.ipdg:
            return fr.local_ipdg(self.kappa[e], self.tau[e], self.sf)
        if self.beta is None:
            L, R, C = fr.local(self.kappa[e], self.tau[e])
            return L, R, C, -self.tau[e] * fr.El
        return fr.local_cd(self.kappa[e], self.tau_f[e], self.beta)

    def _condense_general(self, f):
        E, nv, nt = self.E, self.nv, self.nt
        Ae = np.empty((E, nt, nt))
        ge = np.zeros((E, nt)) if f is not None else None
        for e in range(E):
            L, R, C, T = self.local(e)
            rhs = R if f is None else np.column_stack([R, self.load(f, e)])
            X = np.linalg.solve(L, rhs)                  # LU, partial pivoting
            Ae[e] = C @ X[:, :nt] - T
            if f is not None:
                ge[e] = C @ X[:, nt]
        return Ae, ge

    def load(self, f, e):
        """Right-hand side of element e's local block for nodal forcing f."""
        if self.ipdg:
            return self.forms.Mv @ f[:, e]
        return self.forms.load(f[:, e])

    def _flux_ipdg(self, u_e, e):
        """q = -kappa grad u_h at the volume nodes (primal schemes)."""
        fr = self.forms
        return -self.kappa[e] * np.stack([fr.Gx @ u_e, fr.Gy @ u_e])

    # -- per-element condensation (LU with partial pivoting) -------------
    def element_dofs(self):
        """[E, n_t] edge-major global dof numbers of each element's traces."""
        nd = self.nd
        return (self.edges[:, :, None] * nd + np.arange(nd)[None, None, :]).reshape(self.E, -1)

    def condense(self, f=None, chunk=2048):
        """Return A_e [E, n_t, n_t] and g_e [E, n_t] (g_e only if f given).

        f: nodal forcing [n_v][E] (library layout)."""
        if self.beta is not None or self.ipdg:
            return self._condense_general(f)
        E, nv, nt = self.E, self.nv, self.nt
        Ae = np.empty((E, nt, nt))
        ge = np.zeros((E, nt)) if f is not None else None
        fr = self.forms
        for s in range(0, E, chunk):
            idx = np.arange(s, min(E, s + chunk))
            k = self.kappa[idx][:, None, None]
            t = self.tau[idx][:, None, None]
            L = fr.L0[None] + fr.LM[None] / k + t * fr.Lt[None]
            R = fr.R0[None] + t * fr.Rt[None]
            C = fr.C0[None] + t * fr.Ct[None]
            if f is not None:
                F = np.zeros((len(idx), 3 * nv, 1))
                F[:, 2 * nv:, 0] = (fr.Mv @ f[:, idx]).T
                rhs = np.concatenate([R, F], axis=2)
            else:
                rhs = R
            X = np.linalg.solve(L, rhs)                 # LU, partial pivoting
            Ae[idx] = C @ X[:, :, :nt] + t * fr.El[None]
            if f is not None:
                ge[idx] = (C @ X[:, :, nt:])[:, :, 0]
        return Ae, ge

    def element_operator(self, e, f=None):
        """A_e (and g_e for nodal forcing f [n_v][E]) of one element by the
        same general LU of the local block (for sampled checks at sizes where
        condensing every element is too slow)."""
        L, R, C, T = self.local(e)
        rhs = R if f is None else np.column_stack([R, self.load(f, e)])
        X = np.linalg.solve(L, rhs)
        Ae = C @ X[:, :self.nt] - T
        return (Ae, C @ X[:, self.nt]) if f is not None else Ae

    def recover_element(self, lam_api, f, e):
        """(u_e, q_e) of one element from the full trace vector (library layout)."""
        nd, nv = self.nd, self.nv
        ne = self.ne
        lam_e = np.concatenate([np.asarray(lam_api)[:, ed] for ed in self.edges[e]])
        L, R, _, _ = self.local(e)
        z = np.linalg.solve(L, self.load(f, e) - R @ lam_e)
        if self.ipdg:
            return z, self._flux_ipdg(z, e)
        return z[2 * nv:], np.stack([z[:nv], z[nv:2 * nv]])

    # -- global trace system ----------------------------------------------
    def assemble(self, Ae):
        """Sparse global trace matrix over all edges (edge-major dofs)."""
        dofs = self.element_dofs()
        nt = self.nt
        rows = np.repeat(dofs, nt, axis=1).ravel()
        cols = np.tile(dofs, (1, nt)).ravel()
        N = self.ne * self.nd
        return sp.csr_matrix((Ae.reshape(self.E, -1).ravel(), (rows, cols)), shape=(N, N))

    def assemble_rhs(self, ge):
        g = np.zeros(self.ne * self.nd)
        np.add.at(g, self.element_dofs().ravel(), ge.ravel())
        return g

    def free_dofs(self):
        """Edge-major dofs not on the domain boundary."""
        free_edges = np.nonzero(~self.bmask)[0]
        return (free_edges[:, None] * self.nd + np.arange(self.nd)[None, :]).ravel()

    def dirichlet_dofs(self):
        b_edges = np.nonzero(self.bmask)[0]
        return (b_edges[:, None] * self.nd + np.arange(self.nd)[None, :]).ravel()

    def system(self, f, gD=None):
        """(A_ff, b_f, A_full, g_full, lam_D): the interior trace system
        A_ff lam_f = g_f - A_fD lam_D."""
        Ae, ge = self.condense(f)
        A = self.assemble(Ae)
        g = self.assemble_rhs(ge)
        lamD = np.zeros(self.ne * self.nd)
        if gD is not None:
            full = api_to_edge_major(gD, self.n, self.nd)
            dd = self.dirichlet_dofs()
            lamD[dd] = full[dd]
        fd = self.free_dofs()
        b = g - A @ lamD
        return A[fd][:, fd].tocsc(), b[fd], A, g, lamD

    def solve_direct(self, f, gD=None, ordering="COLAMD"):
        """Sparse direct solve (SuperLU) of the trace system; returns the full
        trace vector in the library layout [nd][n_edges].  ordering: SuperLU's
        column ordering (permc_spec); "MMD_AT_PLUS_A" (minimum degree on
        A^T + A) fills far less on these 2-D trace systems at large n."""
        Aff, bf, A, g, lamD = self.system(f, gD)
        lam = lamD.copy()
        if ordering == "COLAMD":
            lam[self.free_dofs()] = spla.spsolve(Aff, bf)
        else:
            lam[self.free_dofs()] = spla.splu(Aff.tocsc(), permc_spec=ordering).solve(bf)
        return edge_major_to_api(lam, self.n, self.nd)

    # -- recovery ---------------------------------------------------------
    def recover(self, lam_api, f):
        """Local recovery z_e = L_e^-1 (F_e - R_e lambda_e) (Sec. 2).

        Returns u [n_v][E] and q [2][n_v][E] in the library layout."""
        lam = api_to_edge_major(lam_api, self.n, self.nd)
        dofs = self.element_dofs()
        fr = self.forms
        nv = self.nv
        u = np.empty((nv, self.E))
        q = np.empty((2, nv, self.E))
        if self.ipdg:
            for e in range(self.E):
                L, R, _, _ = self.local(e)
                u[:, e] = np.linalg.solve(L, self.load(f, e) - R @ lam[dofs[e]])
                q[:, :, e] = self._flux_ipdg(u[:, e], e)
            return u, q
        if self.beta is not None:
            for e in range(self.E):
                L, R, _, _ = self.local(e)
                z = np.linalg.solve(L, fr.load(f[:, e]) - R @ lam[dofs[e]])
                q[0][:, e], q[1][:, e], u[:, e] = z[:nv], z[nv:2 * nv], z[2 * nv:]
            return u, q
        for s in range(0, self.E, 2048):
            idx = np.arange(s, min(self.E, s + 2048))
            k = self.kappa[idx][:, None, None]
            t = self.tau[idx][:, None, None]
            L = fr.L0[None] + fr.LM[None] / k + t * fr.Lt[None]
            R = fr.R0[None] + t * fr.Rt[None]
            F = np.zeros((len(idx), 3 * nv))
            F[:, 2 * nv:] = (fr.Mv @ f[:, idx]).T
            rhs = F - (R @ lam[dofs[idx]][:, :, None])[:, :, 0]
            z = np.linalg.solve(L, rhs[:, :, None])[:, :, 0]
            q[0][:, idx] = z[:, :nv].T
            q[1][:, idx] = z[:, nv:2 * nv].T
            u[:, idx] = z[:, 2 * nv:].T
        return u, q

    # -- brute force --------------------------------------------------------
    def solve_uncondensed(self, f, gD=None):
        """Dense solve of the full (q, u, lambda) system without condensation.

        Unknowns: z_e for all elements, then free trace dofs.  Rows: the local
        equations of every element, then the conservation equations of every
        interior edge.  Only for tiny meshes."""
        E, nv, nt = self.E, self.nv, self.nt
        nzl = nv if self.ipdg else 3 * nv          # local unknowns per element
        nz = nzl * E
        fd = self.free_dofs()
        pos = -np.ones(self.ne * self.nd, dtype=np.int64)
        pos[fd] = np.arange(len(fd))
        N = nz + len(fd)
        M = np.zeros((N, N))
        rhs = np.zeros(N)
        lamD = np.zeros(self.ne * self.nd)
        if gD is not None:
            full = api_to_edge_major(gD, self.n, self.nd)
            dd = self.dirichlet_dofs()
            lamD[dd] = full[dd]
        dofs = self.element_dofs()
        for e in range(E):
            L, R, C, T = self.local(e)
            zr = slice(nzl * e, nzl * (e + 1))
            M[zr, zr] = L
            rhs[zr] = self.load(f, e)
            for c in range(nt):
                d = dofs[e, c]
                if pos[d] >= 0:
                    M[zr, nz + pos[d]] += R[:, c]
                else:
                    rhs[zr] -= R[:, c] * lamD[d]
            for r in range(nt):
                d = dofs[e, r]
                if pos[d] < 0:
                    continue
                row = nz + pos[d]
                M[row, zr] += C[r]
                for c in range(nt):
                    dc = dofs[e, c]
                    val = T[r, c]
                    if pos[dc] >= 0:
                        M[row, nz + pos[dc]] += val
                    else:
                        rhs[row] -= val * lamD[dc]
        sol = np.linalg.solve(M, rhs)
        lam = lamD.copy()
        lam[fd] = sol[nz:]
        z = sol[:nz].reshape(E, nzl)
        if self.ipdg:
            u = z.T.copy()
            q = np.stack([self._flux_ipdg(u[:, e], e) for e in range(E)], axis=2)
            return edge_major_to_api(lam, self.n, self.nd), u, q
        u = z[:, 2 * nv:].T.copy()
        q = np.stack([z[:, :nv].T, z[:, nv:2 * nv].T])
        return edge_major_to_api(lam, self.n, self.nd), u, q

    # -- geometry helpers for tests -----------------------------------------
    def node_coords(self):
        """Physical coordinates of the volume nodes, [n_v][E] each."""
        xi = self.forms.rq.nodes
        p1 = self.p + 1
        j, i = np.divmod(np.arange(self.E), self.n)
        a = np.arange(self.nv) % p1
        b = np.arange(self.nv) // p1
        X = self.x0 + (i[None, :] + 0.5) * self.hx + 0.5 * self.hx * xi[a][:, None]
        Y = self.y0 + (j[None, :] + 0.5) * self.hy + 0.5 * self.hy * xi[b][:, None]
        return X, Y

    def l2_error(self, vals, exact, nq=None):
        """||v_h - exact||_{L2(Omega)} for nodal field vals [n_v][E]."""
        p = self.p
        nq = nq if nq is not None else p + 4
        xq, wq = refelem.gauss(nq)
        lq = refelem.lagrange(self.forms.rq.nodes, xq)      # [p+1, nq]
        # interpolation matrix nodal -> tensor quadrature points
        Iq = np.einsum('aq,br->rqba', lq, lq).reshape(nq * nq, self.nv)
        j, i = np.divmod(np.arange(self.E), self.n)
        XQ = self.x0 + (i[None, :] + 0.5) * self.hx + 0.5 * self.hx * np.tile(xq, nq)[:, None]
        YQ = self.y0 + (j[None, :] + 0.5) * self.hy + 0.5 * self.hy * np.repeat(xq, nq)[:, None]
        vh = Iq @ vals
        w = np.outer(wq, wq).ravel()[:, None] * (self.hx * self.hy / 4.0)
        return float(np.sqrt(np.sum(w * (vh - exact(XQ, YQ)) ** 2)))
