"""Adjoint gradient of a misfit functional (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Functional: J(m, f) = 1/2 sum_e (u_e - u_obs,e)^T M (u_e - u_obs,e), with m_e the
per-element log-diffusivity (kappa_e = exp(m_e)), u the HDG volume solution
at the Gauss nodes and M the Gauss-point volume mass matrix (the misfit norm
of the L2 reading, evaluated by quadrature on the nodal values).

The derivative is taken on the FULL uncondensed discrete system of
oracle/hdg.py -- unknowns (z_e = [q_x, q_y, u]_e for every element, interior
traces lambda):
    r_e = L_e z_e + R_e lambda_e - F_e = 0,
    c   = sum_e (C_e z_e - tau El lambda_e) = 0   (interior trace rows),
with L_e = L0 + kappa_e^-1 LM + tau Lt, F_e = [0, 0, M f_e].  The adjoint
system (d r / d x)^T psi = -dJ/dx is assembled as one global sparse matrix
and solved with SuperLU; then
    dJ/dm_e = psi_e^T (dL_e/dm_e) z_e = -kappa_e^-1 psi_e^T LM z_e,
    dJ/df_e = -psi_{u,e}^T M.
This is independent of the CUDA path's condensed (u, lambda) derivation.

Pin: central finite differences of the oracle's own forward map
(tests/test_oracle_adjoint.py).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import hdg as H


def misfit(problem, u, u_obs):
    """J = 1/2 sum_e d_e^T M d_e with d = u - u_obs (nodal, [nv][E]) and M the
    volume mass matrix of the element (integrated by the oracle's rule)."""
    d = u - u_obs
    return 0.5 * float(np.einsum('ae,ab,be->', d, problem.forms.Mv, d))


def forward(problem, f, gD=None):
    lam = problem.solve_direct(f, gD)
    u, q = problem.recover(lam, f)
    return lam, u, q


def _full_system(problem, gD):
    """Global sparse Jacobian of (r, c) with respect to (z, lambda_free)."""
    pr = problem
    E, nv, nt = pr.E, pr.nv, pr.nt
    fr = pr.forms
    nz = 3 * nv * E
    fd = pr.free_dofs()
    pos = -np.ones(pr.ne * pr.nd, dtype=np.int64)
    pos[fd] = np.arange(len(fd))
    dofs = pr.element_dofs()
    rows, cols, vals = [], [], []
    for e in range(E):
        L, R, C = fr.local(pr.kappa[e], pr.tau[e])
        z0 = 3 * nv * e
        ii, jj = np.meshgrid(np.arange(3 * nv), np.arange(3 * nv), indexing='ij')
        rows.append((z0 + ii).ravel()); cols.append((z0 + jj).ravel()); vals.append(L.ravel())
        for c in range(nt):
            p = pos[dofs[e, c]]
            if p >= 0:
                rows.append(z0 + np.arange(3 * nv)); cols.append(np.full(3 * nv, nz + p)); vals.append(R[:, c])
        for r in range(nt):
            p = pos[dofs[e, r]]
            if p < 0:
                continue
            rows.append(np.full(3 * nv, nz + p)); cols.append(z0 + np.arange(3 * nv)); vals.append(C[r])
            for c in range(nt):
                pc = pos[dofs[e, c]]
                if pc >= 0 and fr.El[r, c] != 0.0:
                    rows.append(np.array([nz + p])); cols.append(np.array([nz + pc]))
                    vals.append(np.array([-pr.tau[e] * fr.El[r, c]]))
    N = nz + len(fd)
    return sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N, N)), nz


def gradient(problem, f, u_obs, gD=None):
    """(J, dJ/dm [E], dJ/df [nv][E]) by the adjoint of the uncondensed system."""
    pr = problem
    E, nv = pr.E, pr.nv
    lam, u, _ = forward(pr, f, gD)
    J = misfit(pr, u, u_obs)
    # state z_e from the forward solution
    lam_em = H.api_to_edge_major(lam, pr.n, pr.nd)
    dofs = pr.element_dofs()
    fr = pr.forms
    Z = np.zeros((E, 3 * nv))
    for e in range(E):
        L, R, _ = fr.local(pr.kappa[e], pr.tau[e])
        Z[e] = np.linalg.solve(L, fr.load(f[:, e]) - R @ lam_em[dofs[e]])
    K, nz = _full_system(pr, gD)
    # dJ/dx: only the u-blocks of z carry the misfit
    rhs = np.zeros(K.shape[0])
    d = u - u_obs
    for e in range(E):
        rhs[3 * nv * e + 2 * nv: 3 * nv * (e + 1)] = -(fr.Mv @ d[:, e])
    psi = spla.spsolve(K.T.tocsc(), rhs)
    dJdm = np.zeros(E)
    dJdf = np.zeros((nv, E))
    for e in range(E):
        pe = psi[3 * nv * e: 3 * nv * (e + 1)]
        dJdm[e] = -(pe @ (fr.LM @ Z[e])) / pr.kappa[e]
        dJdf[:, e] = -(fr.Mv.T @ pe[2 * nv:])
    return J, dJdm, dJdf


def misfit_of(n, p, logk, tau, f, u_obs, gD=None):
    """Forward map m -> J used for finite differences."""
    pr = H.HDGProblem(n, p, np.exp(logk), tau)
    _, u, _ = forward(pr, f, gD)
    return misfit(pr, u, u_obs)
