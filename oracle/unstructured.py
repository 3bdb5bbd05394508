"""Unstructured quadrilateral meshes (oracle): mapped HDG elements, seed-point
agglomeration and the DtN multigrid hierarchy of Sec. 3 on it.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Mesh.  Vertices xy [n_vert, 2] and elements quads [E, 4] listed
counter-clockwise.  Element e is the image of [-1, 1]^2 under the bilinear
map taking the corners (-1,-1), (1,-1), (1,1), (-1,1) to its vertices 0..3;
local edge j runs from vertex j to vertex j+1 (mod 4).  The global edges are
the distinct vertex pairs (lo, hi), numbered in lexicographic order; the trace
basis of an edge is the orthonormal Legendre basis of refelem.trace_basis on
the physical edge, with s = -1 at vertex lo and s = 1 at vertex hi.

Element operators.  The HDG forms of Sec. 2 (eqs. HDG_local1/2, HDG_flux;
the same blocks as hdg.ElementForms) integrated over the mapped element with
an nq-point tensor Gauss rule (default p + 3).  On a bilinear map det J is
bilinear and det J times a physical derivative is the cofactor matrix (linear
entries) applied to the reference gradient, so every form is a polynomial of
degree <= 2p + 1 per direction and any rule with nq >= p + 1 is exact.  The
local block is condensed by a general LU exactly as in hdg.HDGProblem.

Agglomeration (Sec. 3.1.2, seed points; the readings are listed in the
design notes of the repository):
  P_0      element e joins the seed nearest its vertex average (squared
           Euclidean distance, ties to the lower seed index); seeds that
           attract no element are dropped.
  P_{r+1}  every macro-element of P_r with m > 1 elements is cut in four by
           two rounds of bisection: its element centroids are sorted along
           the axis of larger spread (x when equal), ties by element index,
           and the first floor(m/2) form the first half.  Parts are numbered
           in order of their parent macro-element, then first half's parts
           before the second half's; empty parts are dropped.
  A cut partition is kept while it has at most E/2 macro-elements; the
  mesh itself is P_H.
Macro-edges.  The units of the finest partition are the mesh edges.  On
P_r (r < H) every unit of P_{r+1} whose two sides (macro-elements, -1 for the
domain boundary) have different parents in P_r is grouped by that pair of
parents; inside a group two units are linked at a vertex where exactly two
unit ends of the group meet.  Every connected set of linked units is one
macro-edge of P_r (a path or a cycle of units).  Units with equal parents are
interior to their parent.  Macro-edges are numbered by their lowest unit.
Parameterisation (the remark in Sec. 3.1): arc length along the macro-edge.
A path starts at the free end with the lower vertex index (equal ends: at the
end unit with the lower index); a cycle starts at its lowest junction vertex
and leaves it along the lower of the two units there; a macro-edge of one
unit keeps that unit's parameterisation.  The coarse space on a macro-edge of
length L is P_1 in arc length s with the orthonormal basis 1/sqrt(L),
sqrt(3/L)(2 s/L - 1) (Sec. 3.1.1: P_1 below the finest level).

Multigrid levels (finest first): the mesh with P_p traces, the mesh with P_1
traces (p > 1), then P_{H-1}, ..., P_0.  Every level keeps the macro-edges
that are not on the domain boundary (homogeneous Dirichlet data for the
error equations).  J between two h-levels is the L2 projection of the coarse
macro-edge basis onto the finer one, computed here by Gauss quadrature on
every mesh edge; the operators I_k, Q_{k-1}, T_k and A_{k-1} are those of
oracle.mg (eqs. n_1_Ik, n_1_Qk, localCorrection, coarse), and the V-cycle and
the outer iterations are oracle.mg.Hierarchy's.

Pins (tests/test_oracle_unstructured.py): an axis-aligned square element
equals hdg.ElementForms' element; linear solutions reproduced to round-off
on a jittered mesh; O(h^{p+1}) convergence of u under uniform refinement;
over-integration invariance; A_e 1 = 0; nestedness of the macro-edge spaces
(the finer basis reproduces every coarse basis function); the DtN identity
(A_{k-1} equals the Schur complement of the fine operator onto the coarse
space); partitions and macro-edges by brute force on a hand-built mesh; V-cycle
contraction and PCG convergence.
"""
from collections import defaultdict

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import hdg as H
from . import mg as MG
from . import refelem


# --------------------------------------------------------------------------
# mesh topology
# --------------------------------------------------------------------------
def mesh_edges(quads):
    """(edge_vertices [n_e, 2] (lo, hi), elem_edges [E, 4], edge_elems [n_e, 2])
    with edges in lexicographic (lo, hi) order; edge_elems lists the one or two
    elements of each edge in ascending order, -1 for none."""
    quads = np.asarray(quads, dtype=np.int64)
    E = len(quads)
    a = quads
    b = np.roll(quads, -1, axis=1)
    lo = np.minimum(a, b)
    hi = np.maximum(a, b)
    keys = sorted(set(zip(lo.ravel().tolist(), hi.ravel().tolist())))
    index = {k: i for i, k in enumerate(keys)}
    elem_edges = np.array([[index[(int(lo[e, j]), int(hi[e, j]))] for j in range(4)]
                           for e in range(E)], dtype=np.int64).reshape(E, 4)
    edge_elems = -np.ones((len(keys), 2), dtype=np.int64)
    for e in range(E):
        for j in range(4):
            g = elem_edges[e, j]
            if edge_elems[g, 0] < 0:
                edge_elems[g, 0] = e
            elif edge_elems[g, 1] < 0:
                edge_elems[g, 1] = e
            else:
                raise ValueError("non-conforming mesh: an edge with three elements")
    return np.array(keys, dtype=np.int64).reshape(-1, 2), elem_edges, edge_elems


def centroids(verts, quads):
    """Vertex average of every element, summed in vertex order 0..3."""
    v = np.asarray(verts, dtype=np.float64)[np.asarray(quads)]
    return (((v[:, 0] + v[:, 1]) + v[:, 2]) + v[:, 3]) * 0.25


# --------------------------------------------------------------------------
# mapped element
# --------------------------------------------------------------------------
_CORNERS = np.array([[-1.0, -1.0], [1.0, -1.0], [1.0, 1.0], [-1.0, 1.0]])


class MappedQuad:
    """Volume and edge tables of one bilinearly mapped quadrilateral with the
    RefQuad interface (volume node index j*(p+1) + i, i along xi)."""

    def __init__(self, p, xy, flips, nq=None):
        self.p = p
        self.nq = nq if nq is not None else p + 3
        self.xy = np.asarray(xy, dtype=np.float64)
        self.flips = list(flips)
        self.nodes, _ = refelem.gauss(p + 1)
        self.xq, self.wq = refelem.gauss(self.nq)
        self.nv = (p + 1) ** 2

    def _map(self, xi, eta):
        """x, y and the Jacobian entries at reference points."""
        N = 0.25 * np.stack([(1 - xi) * (1 - eta), (1 + xi) * (1 - eta),
                             (1 + xi) * (1 + eta), (1 - xi) * (1 + eta)])
        Nxi = 0.25 * np.stack([-(1 - eta), (1 - eta), (1 + eta), -(1 + eta)])
        Neta = 0.25 * np.stack([-(1 - xi), -(1 + xi), (1 + xi), (1 - xi)])
        X, Y = self.xy[:, 0], self.xy[:, 1]
        return (X @ N, Y @ N, X @ Nxi, X @ Neta, Y @ Nxi, Y @ Neta)

    def _basis(self, xi, eta):
        p1 = self.p + 1
        lx = refelem.lagrange(self.nodes, xi)
        ly = refelem.lagrange(self.nodes, eta)
        dlx = refelem.lagrange_deriv(self.nodes, xi)
        dly = refelem.lagrange_deriv(self.nodes, eta)
        phi = np.zeros((self.nv, len(xi)))
        dxi = np.zeros_like(phi)
        deta = np.zeros_like(phi)
        for j in range(p1):
            for i in range(p1):
                a = j * p1 + i
                phi[a] = lx[i] * ly[j]
                dxi[a] = dlx[i] * ly[j]
                deta[a] = lx[i] * dly[j]
        return phi, dxi, deta

    def volume_tables(self):
        xi = np.tile(self.xq, self.nq)
        eta = np.repeat(self.xq, self.nq)
        w = np.outer(self.wq, self.wq).ravel()
        _, _, xx, xe, yx, ye = self._map(xi, eta)
        det = xx * ye - xe * yx
        if np.any(det <= 0):
            raise ValueError("element not counter-clockwise or degenerate")
        phi, dxi, deta = self._basis(xi, eta)
        # grad = J^-T grad_ref,  J = [[x_xi, x_eta], [y_xi, y_eta]]
        dx = (ye * dxi - yx * deta) / det
        dy = (-xe * dxi + xx * deta) / det
        return phi, dx, dy, w * det

    def edge_tables(self, edge):
        """(phi on the edge [n_v, nq], psi [p+1, nq] in the global edge
        orientation, w_ds [nq], outward unit normal) of local edge 0..3."""
        s = self.xq
        c0 = _CORNERS[edge]
        c1 = _CORNERS[(edge + 1) % 4]
        xi = 0.5 * (1 - s) * c0[0] + 0.5 * (1 + s) * c1[0]
        eta = 0.5 * (1 - s) * c0[1] + 0.5 * (1 + s) * c1[1]
        phi, _, _ = self._basis(xi, eta)
        d = self.xy[(edge + 1) % 4] - self.xy[edge]
        length = float(np.hypot(d[0], d[1]))
        normal = (d[1] / length, -d[0] / length)
        sg = -s if self.flips[edge] else s
        psi = refelem.trace_basis(self.p, sg, length)
        return phi, psi, self.wq * (length / 2.0), normal

    def points(self, xi, eta):
        x, y, _, _, _, _ = self._map(np.asarray(xi, float), np.asarray(eta, float))
        return x, y


class UHDGProblem:
    """HDG trace system on an unstructured quadrilateral mesh (diffusion,
    K = kappa I per element, scalar or per-element tau).

    Forcing and recovered fields are nodal, element-major: f[e, a] at the
    (p+1)^2 Gauss points of element e (node a = j*(p+1) + i).  Trace vectors
    are edge-major: dof = edge*(p+1) + mode over all edges."""

    def __init__(self, verts, quads, p, kappa, tau, nq=None):
        self.verts = np.asarray(verts, dtype=np.float64)
        self.quads = np.asarray(quads, dtype=np.int64)
        self.p = p
        self.E = len(self.quads)
        self.nd = p + 1
        self.edge_vertices, self.edges, self.edge_elems = mesh_edges(self.quads)
        self.ne = len(self.edge_vertices)
        self.bmask = self.edge_elems[:, 1] < 0
        self.kappa = np.broadcast_to(np.asarray(kappa, dtype=np.float64), (self.E,)).copy()
        self.tau = np.broadcast_to(np.asarray(tau, dtype=np.float64), (self.E,)).copy()
        self.nq = nq
        self.nv = (p + 1) ** 2
        self.nt = 4 * (p + 1)
        self.symmetric = True
        self._forms = {}

    def quad(self, e):
        q = self.quads[e]
        flips = [q[j] > q[(j + 1) % 4] for j in range(4)]
        return MappedQuad(self.p, self.verts[q], flips, self.nq)

    def forms(self, e):
        if e not in self._forms:
            self._forms[e] = H.ElementForms(self.p, 1.0, 1.0, quad=self.quad(e))
        return self._forms[e]

    def element_operator(self, e, f=None):
        """A_e [n_t, n_t] (and g_e for nodal forcing f [E, n_v]): general LU of
        the local block, A_e = C L^-1 R + tau El."""
        fr = self.forms(e)
        L, R, C = fr.local(self.kappa[e], self.tau[e])
        rhs = R if f is None else np.column_stack([R, fr.load(f[e])])
        X = np.linalg.solve(L, rhs)
        Ae = C @ X[:, :self.nt] + self.tau[e] * fr.El
        return (Ae, C @ X[:, self.nt]) if f is not None else Ae

    def condense(self, f=None):
        Ae = np.empty((self.E, self.nt, self.nt))
        ge = np.zeros((self.E, self.nt)) if f is not None else None
        for e in range(self.E):
            if f is None:
                Ae[e] = self.element_operator(e)
            else:
                Ae[e], ge[e] = self.element_operator(e, f)
        return Ae, ge

    def element_dofs(self):
        nd = self.nd
        return (self.edges[:, :, None] * nd + np.arange(nd)[None, None, :]).reshape(self.E, -1)

    def assemble(self, Ae):
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
        fe = np.nonzero(~self.bmask)[0]
        return (fe[:, None] * self.nd + np.arange(self.nd)[None, :]).ravel()

    def project_dirichlet(self, g):
        """Trace vector (all edges, edge-major) holding the L2 projection of
        g(x, y) onto P_p of every boundary edge (zero elsewhere)."""
        lam = np.zeros(self.ne * self.nd)
        s, w = refelem.gauss(self.p + 3)
        for ed in np.nonzero(self.bmask)[0]:
            lo, hi = self.edge_vertices[ed]
            a, b = self.verts[lo], self.verts[hi]
            length = float(np.hypot(*(b - a)))
            x = 0.5 * (1 - s) * a[0] + 0.5 * (1 + s) * b[0]
            y = 0.5 * (1 - s) * a[1] + 0.5 * (1 + s) * b[1]
            psi = refelem.trace_basis(self.p, s, length)
            lam[ed * self.nd:(ed + 1) * self.nd] = (psi * w * (length / 2)) @ g(x, y)
        return lam

    def solve_direct(self, f, g=None):
        """(lambda over all edges, edge-major) by a sparse direct solve; g: the
        Dirichlet function (None = homogeneous)."""
        Ae, ge = self.condense(f)
        A = self.assemble(Ae)
        b = self.assemble_rhs(ge)
        lam = self.project_dirichlet(g) if g is not None else np.zeros(self.ne * self.nd)
        fd = self.free_dofs()
        rhs = (b - A @ lam)[fd]
        lam[fd] = spla.spsolve(A[fd][:, fd].tocsc(), rhs)
        return lam

    def recover(self, lam, f):
        """(u [E, n_v], q [E, 2, n_v]) at the volume nodes."""
        u = np.zeros((self.E, self.nv))
        q = np.zeros((self.E, 2, self.nv))
        nv = self.nv
        for e in range(self.E):
            fr = self.forms(e)
            L, R, _ = fr.local(self.kappa[e], self.tau[e])
            lam_e = lam[self.element_dofs()[e]]
            z = np.linalg.solve(L, fr.load(f[e]) - R @ lam_e)
            u[e] = z[2 * nv:]
            q[e, 0] = z[:nv]
            q[e, 1] = z[nv:2 * nv]
        return u, q

    def node_coords(self):
        """Physical coordinates [E, n_v, 2] of every element's volume nodes."""
        p1 = self.p + 1
        nodes, _ = refelem.gauss(p1)
        xi = np.tile(nodes, p1)
        eta = np.repeat(nodes, p1)
        out = np.zeros((self.E, self.nv, 2))
        for e in range(self.E):
            x, y = self.quad(e).points(xi, eta)
            out[e, :, 0], out[e, :, 1] = x, y
        return out

    def l2_error(self, u, exact):
        """|| u_h - exact ||_L2 with u_h the nodal Q_p field u [E, n_v]."""
        err = 0.0
        for e in range(self.E):
            qd = self.quad(e)
            phi, _, _, wJ = qd.volume_tables()
            xi = np.tile(qd.xq, qd.nq)
            eta = np.repeat(qd.xq, qd.nq)
            x, y = qd.points(xi, eta)
            d = u[e] @ phi - exact(x, y)
            err += float(np.sum(wJ * d * d))
        return np.sqrt(err)


# --------------------------------------------------------------------------
# seed-point agglomeration
# --------------------------------------------------------------------------
def seed_partition(verts, quads, seeds):
    """P_0: element -> macro-element (nearest seed, compacted in seed order)."""
    c = centroids(verts, quads)
    seeds = np.asarray(seeds, dtype=np.float64)
    E = len(c)
    best = np.zeros(E, dtype=np.int64)
    for e in range(E):
        bd = None
        for s in range(len(seeds)):
            dx = c[e, 0] - seeds[s, 0]
            dy = c[e, 1] - seeds[s, 1]
            d = dx * dx + dy * dy
            if bd is None or d < bd:
                bd, best[e] = d, s
    used = np.unique(best)
    remap = -np.ones(len(seeds), dtype=np.int64)
    remap[used] = np.arange(len(used))
    return remap[best]


def _bisect(elems, c):
    """Split a sorted element list in two halves along the axis of larger
    centroid spread (x on ties); ties in the coordinate by element index."""
    xs = c[elems, 0]
    ys = c[elems, 1]
    axis = 0 if (xs.max() - xs.min()) >= (ys.max() - ys.min()) else 1
    key = c[elems, axis]
    order = sorted(range(len(elems)), key=lambda t: (key[t], elems[t]))
    half = len(elems) // 2
    first = sorted(elems[t] for t in order[:half])
    second = sorted(elems[t] for t in order[half:])
    return first, second


def split_partition(part, c):
    """P_{r+1} from P_r: every macro-element with more than one element cut in
    four by two rounds of bisection."""
    nmac = int(part.max()) + 1
    members = [[] for _ in range(nmac)]
    for e in range(len(part)):
        members[part[e]].append(e)
    out = -np.ones(len(part), dtype=np.int64)
    nxt = 0
    for m in range(nmac):
        el = members[m]
        if len(el) == 1:
            pieces = [el]
        else:
            a, b = _bisect(np.array(el), c)
            pieces = []
            for half in (a, b):
                if len(half) <= 1:
                    pieces.append(half)
                else:
                    pieces.extend(_bisect(np.array(half), c))
        for pc in pieces:
            if len(pc):
                out[pc] = nxt
                nxt += 1
    return out


def partitions(verts, quads, seeds):
    """[P_0, P_1, ..., P_{H-1}]: element -> macro-element maps, coarsest
    first; a cut partition is kept while it has at most E/2 macro-elements
    (two or more elements per macro-element on average)."""
    c = centroids(verts, quads)
    part = seed_partition(verts, quads, seeds)
    out = [part]
    E = len(part)
    while True:
        part = split_partition(part, c)
        if 2 * (int(part.max()) + 1) > E:
            return out
        out.append(part)


# --------------------------------------------------------------------------
# macro-edges
# --------------------------------------------------------------------------
class Chain:
    """A macro-edge: ordered units (finer macro-edges) with directions, the
    mesh edges it covers (ordered, with +1 for lo -> hi), its two sides."""

    def __init__(self, units, dirs, start, end, sides, edges, edirs, length, closed):
        self.units, self.dirs = units, dirs
        self.start, self.end = start, end
        self.sides = sides
        self.edges, self.edirs = edges, edirs
        self.length = length
        self.closed = closed


def mesh_units(verts, edge_vertices, edge_elems):
    out = []
    for m, (lo, hi) in enumerate(edge_vertices):
        d = verts[hi] - verts[lo]
        a, b = edge_elems[m]
        out.append(Chain([m], [1], int(lo), int(hi), (int(a), int(b)), [m], [1],
                         float(np.hypot(d[0], d[1])), False))
    return out


def link_units(units, parent):
    """Macro-edges of the coarser partition from the units of the finer one.

    parent: finer macro-element -> coarser macro-element.  Returns
    (chains sorted by lowest unit, interior [(unit, coarse macro)])."""
    groups = defaultdict(list)
    interior = []
    for ui, u in enumerate(units):
        a, b = u.sides
        pa = int(parent[a])
        pb = int(parent[b]) if b >= 0 else -1
        if pa == pb:
            interior.append((ui, pa))
            continue
        key = (min(pa, pb), max(pa, pb)) if pb >= 0 else (pa, -1)
        groups[key].append(ui)
    chains = []
    for key, ulist in groups.items():
        at = defaultdict(list)
        for ui in ulist:
            at[units[ui].start].append(ui)
            at[units[ui].end].append(ui)
        links = defaultdict(list)            # unit -> [(vertex, other unit)]
        for v, us in at.items():
            if len(us) == 2 and us[0] != us[1]:
                links[us[0]].append((v, us[1]))
                links[us[1]].append((v, us[0]))
        seen = set()
        for u0 in sorted(ulist):
            if u0 in seen:
                continue
            comp, stack = [], [u0]
            seen.add(u0)
            while stack:
                x = stack.pop()
                comp.append(x)
                for _, y in links[x]:
                    if y not in seen:
                        seen.add(y)
                        stack.append(y)
            chains.append(_order_chain(sorted(comp), units, links, key))
    chains.sort(key=lambda ch: min(ch.units))
    return chains, interior


def _order_chain(comp, units, links, sides):
    if len(comp) == 1:
        u = units[comp[0]]
        return Chain([comp[0]], [1], u.start, u.end, sides, list(u.edges), list(u.edirs),
                     u.length, u.closed or u.start == u.end)
    ends = [x for x in comp if len(links[x]) == 1]
    if ends:                                  # path
        def free_vertex(x):
            v = links[x][0][0]
            return units[x].end if units[x].start == v else units[x].start
        fa, fb = free_vertex(ends[0]), free_vertex(ends[1])
        if fa != fb:
            first, v = (ends[0], fa) if fa < fb else (ends[1], fb)
        else:
            first = min(ends)
            v = fa
        closed = False
    else:                                     # cycle
        v = min(w for x in comp for w, _ in links[x])
        first = min(y for x in comp for w, y in links[x] if w == v)
        closed = True
    order, dirs = [], []
    x, cur, prev = first, v, None
    start = v
    while True:
        u = units[x]
        d = 1 if u.start == cur else -1
        order.append(x)
        dirs.append(d)
        cur = u.end if d == 1 else u.start
        nxt = [y for w, y in links[x] if w == cur and y != prev]
        if closed and len(order) == len(comp):
            break
        if not nxt:
            break
        prev, x = x, nxt[0]
        if x == first:
            break
    edges, edirs = [], []
    for x, d in zip(order, dirs):
        u = units[x]
        if d == 1:
            edges += u.edges
            edirs += u.edirs
        else:
            edges += u.edges[::-1]
            edirs += [-t for t in u.edirs[::-1]]
    length = sum(units[x].length for x in order)
    return Chain(order, dirs, start, cur, sides, edges, edirs, length, closed)


def hierarchy_chains(verts, quads, seeds):
    """(partitions [P_0..P_{H-1}], levels) where levels[t] for t = 0..H
    describes partition P_{H-t} (t = 0: the mesh itself) as
    {"units": chains, "interior": [(finer unit, macro)] (t >= 1)}."""
    verts = np.asarray(verts, dtype=np.float64)
    edge_vertices, _, edge_elems = mesh_edges(quads)
    parts = partitions(verts, quads, seeds)
    Hn = len(parts)
    levels = [{"units": mesh_units(verts, edge_vertices, edge_elems), "interior": []}]
    E = len(quads)
    finer = np.arange(E)                          # element -> finer macro (identity at the mesh)
    for r in range(Hn - 1, -1, -1):
        coarse = parts[r]
        parent = np.zeros(int(finer.max()) + 1, dtype=np.int64)
        parent[finer] = coarse
        chains, interior = link_units(levels[-1]["units"], parent)
        levels.append({"units": chains, "interior": interior})
        finer = coarse
    return parts, levels


# --------------------------------------------------------------------------
# the multigrid hierarchy
# --------------------------------------------------------------------------
def chain_basis(chains, verts, edge_vertices, n_mesh_edges, keep):
    """Phi [2 n_mesh_edges, 2 len(keep)]: the P_1 arc-length basis of each kept
    macro-edge in the P_1 Legendre coefficients of the mesh edges, by Gauss
    quadrature on every mesh edge (L2 projection; exact, the restriction is
    linear)."""
    s, w = refelem.gauss(4)
    rows, cols, vals = [], [], []
    for col, ci in enumerate(keep):
        ch = chains[ci]
        L = ch.length
        off = 0.0
        for m, d in zip(ch.edges, ch.edirs):
            lo, hi = edge_vertices[m]
            ell = float(np.hypot(*(verts[hi] - verts[lo])))
            # arc length along the macro-edge at the quadrature points
            arc = off + ell * ((1 + s) / 2 if d == 1 else (1 - s) / 2)
            t = arc / L
            coarse = np.stack([np.full_like(t, 1 / np.sqrt(L)), np.sqrt(3 / L) * (2 * t - 1)])
            fine = refelem.trace_basis(1, s, ell)
            blk = (fine * w * (ell / 2)) @ coarse.T             # [fine mode, coarse mode]
            for l in range(2):
                for k in range(2):
                    rows.append(2 * m + l)
                    cols.append(2 * col + k)
                    vals.append(blk[l, k])
            off += ell
    return sp.csr_matrix((vals, (rows, cols)), shape=(2 * n_mesh_edges, 2 * len(keep)))


class ULevel(MG.Level):
    pass


class UHierarchy(MG.Hierarchy):
    """oracle.mg.Hierarchy on an unstructured mesh (block-Jacobi smoother)."""

    def __init__(self, problem, seeds, Ae=None, m_fine=1, m_growth=2, m_max=None,
                 local_corr="both", omega=1.0):
        self.smoother = "block_jacobi"
        self.problem = problem
        self.dirichlet = True
        self.local_corr = local_corr
        self.omega = omega
        pr = problem
        p = pr.p
        if Ae is None:
            Ae, _ = pr.condense()
        self.parts, self.chain_levels = hierarchy_chains(pr.verts, pr.quads, seeds)
        A_full = pr.assemble(Ae)
        free = pr.free_dofs()
        levels = []
        L = ULevel()
        L.nd, L.free = p + 1, free
        L.A = A_full[free][:, free].tocsr()
        levels.append(L)
        interior_edges = np.nonzero(~pr.bmask)[0]
        if p > 1:
            Lc = ULevel()
            Lc.nd = 2
            Lc.free = (interior_edges[:, None] * 2 + np.arange(2)[None, :]).ravel()
            cols = np.arange(len(Lc.free))
            rows = (np.arange(len(interior_edges))[:, None] * (p + 1)
                    + np.arange(2)[None, :]).ravel()
            J = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(len(free), len(cols)))
            L.kind, L.I, L.Q, L.T = "p", J, J.T.tocsr(), None
            Lc.A = (L.Q @ L.A @ L.I).tocsr()
            levels.append(Lc)
            L = Lc
        # finest P_1 basis: the interior mesh edges themselves
        ne = pr.ne
        keep = list(interior_edges)
        Phi = sp.csr_matrix((np.ones(2 * len(keep)),
                             ((np.array(keep)[:, None] * 2 + np.arange(2)).ravel(),
                              np.arange(2 * len(keep)))), shape=(2 * ne, 2 * len(keep)))
        L.Phi = Phi
        L.keep = keep
        self.nested_residual = 0.0
        for t in range(1, len(self.chain_levels)):
            lev = self.chain_levels[t]
            units_fine = self.chain_levels[t - 1]["units"]
            chains = lev["units"]
            keepc = [i for i, ch in enumerate(chains) if ch.sides[1] >= 0]
            Phic = chain_basis(chains, pr.verts, pr.edge_vertices, ne, keepc)
            Jfull = (L.Phi.T @ Phic).tocsr()
            self.nested_residual = max(self.nested_residual,
                                       abs(L.Phi @ Jfull - Phic).max() if Phic.nnz else 0.0)
            # fine positions: L.keep lists the fine units carrying dofs, in order
            int_units = {u for u, _ in lev["interior"]}
            pos_I = [i for i, u in enumerate(L.keep) if u in int_units]
            pos_B = [i for i, u in enumerate(L.keep) if u not in int_units]
            Iset = np.array([2 * i + k for i in pos_I for k in range(2)], dtype=np.int64)
            Bset = np.array([2 * i + k for i in pos_B for k in range(2)], dtype=np.int64)
            Lc = ULevel()
            Lc.nd = 2
            Lc.keep = keepc
            Lc.Phi = Phic
            self._coarsen(L, Lc, Iset, Bset, Jfull)
            levels.append(Lc)
            L = Lc
        m = m_fine
        for lev in levels:
            lev.m = m
            m = m * m_growth
            if m_max is not None:
                m = min(m, m_max)
        for lev in levels:
            lev.Dinv = self._block_jacobi(lev)
        coarse = levels[-1]
        coarse.lu = None
        coarse.chol = sla.cho_factor(coarse.A.toarray()) if coarse.A.shape[0] else None
        self.levels = levels

    @staticmethod
    def _coarsen(L, Lc, Iset, Bset, J):
        """I_k, Q_{k-1}, T_k and A_{k-1} = Q_{k-1} A_k I_k (eqs. n_1_Ik,
        n_1_Qk, localCorrection, coarse); J: all fine dofs -> coarse dofs."""
        nfree = L.A.shape[0]
        PI = sp.csr_matrix((np.ones(len(Iset)), (np.arange(len(Iset)), Iset)),
                           shape=(len(Iset), nfree))
        PB = sp.csr_matrix((np.ones(len(Bset)), (np.arange(len(Bset)), Bset)),
                           shape=(len(Bset), nfree))
        A = L.A
        AII = PI @ A @ PI.T
        AIB = PI @ A @ PB.T
        ABI = PB @ A @ PI.T
        JB = PB @ J
        AIIinv = MG._block_inverse(AII) if len(Iset) else sp.csr_matrix((0, 0))
        L.kind = "h"
        L.I = sp.csr_matrix(PI.T @ (-(AIIinv @ (AIB @ JB))) + PB.T @ JB)
        L.Q = sp.csr_matrix((-(JB.T @ ABI @ AIIinv)) @ PI + JB.T @ PB)
        L.Iset = Iset
        L.AIIinv = AIIinv
        L.T = PI.T @ AIIinv @ PI
        Lc.A = (L.Q @ A @ L.I).tocsr()
