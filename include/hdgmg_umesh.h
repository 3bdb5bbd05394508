/*
 * hdgmg_umesh.h -- C ABI of the unstructured-mesh path of libhdgmg: the HDG
 * trace system on a conforming mesh of convex quadrilaterals and the DtN
 * multigrid of Sec. 3 of arXiv:1811.09909 on macro-elements built from seed
 * points (Sec. 3.1.2, the agglomeration used for Example II).
 *
 * Problem: -div(kappa grad u) = f, u = 0 on the whole boundary (the outer
 * boundary and the boundaries of holes), K = kappa_e I per element, HDG with
 * a constant tau (Sec. 2, eqs. HDG_local1/2, HDG_flux, conservation).
 *
 * Conventions
 * -----------
 *  mesh       vertices [n_vert][2] FP64; elements [n_elem][4] int32 vertex
 *             indices listed counter-clockwise.  Element e is the image of
 *             [-1,1]^2 under the bilinear map taking (-1,-1), (1,-1), (1,1),
 *             (-1,1) to its vertices 0..3; local edge j runs from vertex j to
 *             vertex j+1 (mod 4).
 *  edges      the distinct vertex pairs (lo, hi), lo < hi, numbered in
 *             lexicographic order (hdgmg_umesh_plan_edges returns them).  An
 *             edge with one element is a boundary (Dirichlet) edge.
 *  traces     [n_edges][p+1] (edge-major), mode k of the orthonormal basis
 *             psi_k = sqrt((2k+1)/|e|) P_k(s), s = -1 at vertex lo, +1 at hi.
 *  volume     [n_elem][(p+1)^2], node (i, j) -> j*(p+1) + i at the
 *             Gauss-Legendre points (i along the reference xi axis);
 *             flux q = -kappa grad u: [n_elem][2][(p+1)^2], x first.
 *  level vectors (hdgmg_umesh_apply / _vcycle): the macro-edges of the level
 *             that are not on the boundary, in the level's order, times the
 *             level's modes per macro-edge (p+1 on the finest level, 2 below),
 *             macro-edge-major.  On the finest level these are the interior
 *             mesh edges in edge order.
 *
 * Multigrid levels (finest first): the mesh with P_p traces; the mesh with
 * P_1 traces (p > 1; Sec. 3.1.1); then the partitions P_{H-1}, ..., P_0 (the
 * coarsest, from the seeds).
 *  P_0      element e joins the seed nearest its vertex average
 *           ((((x0+x1)+x2)+x3)/4, squared Euclidean distance, ties to the lower
 *           seed); seeds that attract no element are dropped, the rest
 *           renumbered in seed order.
 *  P_{r+1}  each macro-element of P_r with m > 1 elements is cut in four by
 *           two rounds of bisection: element centroids sorted along the axis of
 *           larger spread (x when equal; ties in the coordinate by element
 *           index), the first floor(m/2) forming the first half.  Parts are
 *           numbered in order of their parent, the first half's parts first.
 *           A cut partition is kept while it has at most n_elem/2
 *           macro-elements.
 *  macro-edges of P_r: units of the next finer partition (mesh edges below
 *           P_{H-1}) whose two sides have different parents, grouped by that
 *           pair (boundary = -1) and linked at vertices where exactly two unit
 *           ends of the group meet; each linked set is a macro-edge (a path or
 *           a cycle), numbered by its lowest unit.  Its coarse space is P_1 in
 *           arc length (basis 1/sqrt(L), sqrt(3/L)(2s/L - 1)); a path starts at
 *           the free end with the lower vertex index (equal ends: at the end
 *           unit with the lower index), a cycle at its lowest junction vertex
 *           along the lower of its two units there, a one-unit macro-edge keeps
 *           the unit's parameterisation.
 * J between levels is exact (nested spaces: the coarse P_1 arc-length
 * function restricted to a unit is P_1 in the unit's arc length).
 *
 * Memory, streams and errors as in hdgmg.h.
 */
#ifndef HDGMG_UMESH_H
#define HDGMG_UMESH_H

#include <stdint.h>
#include "hdgmg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t n_vert;
  const double* xy;       /* host [n_vert][2]                                 */
  int32_t n_elem;
  const int32_t* quads;   /* host [n_elem][4], counter-clockwise, convex      */
  int32_t p;              /* 1..8                                             */
  double tau;             /* HDG stabilisation, > 0                           */
  int32_t n_seeds;
  const double* seeds;    /* host [n_seeds][2]                                */
} hdgmg_umesh_problem;

/* ---- host-only plan: the hierarchy's topology and geometry -------------- */

typedef struct hdgmg_umesh_plan hdgmg_umesh_plan;

/* Build the plan on the host (no device use): edges, partitions,
 * macro-edges and their parameterisation, the per-level index lists and the
 * closed-form J blocks.  EINVAL for an empty or non-conforming mesh, a
 * vertex index out of range, an element that is not convex and
 * counter-clockwise, p outside 1..8, tau <= 0 or no seed.  The arrays are
 * copied; the caller keeps ownership of the problem. */
hdgmg_status hdgmg_umesh_plan_create(hdgmg_umesh_plan** plan,
                                     const hdgmg_umesh_problem* problem);
void hdgmg_umesh_plan_destroy(hdgmg_umesh_plan* plan);

/* out[0] = n_edges, out[1] = number of partitions H (P_0..P_{H-1}),
 * out[2] = number of multigrid levels, out[3] = interior trace unknowns. */
hdgmg_status hdgmg_umesh_plan_sizes(const hdgmg_umesh_plan* plan, int64_t* out);

/* edge_vertices host [n_edges][2] (lo, hi) out. */
hdgmg_status hdgmg_umesh_plan_edges(const hdgmg_umesh_plan* plan,
                                    int32_t* edge_vertices);

/* elem_to_macro host [n_elem] out: the macro-element of every element in
 * partition P_r, 0 <= r < H. */
hdgmg_status hdgmg_umesh_plan_partition(const hdgmg_umesh_plan* plan,
                                        int32_t r, int32_t* elem_to_macro);

/* Macro-edges of the partition t steps above the mesh (t = 0: the mesh
 * edges, t = H: P_0).  counts host [2] out: number of macro-edges, total
 * number of (mesh edge, direction) items.  If info is not NULL it receives
 * [n][6]: side0, side1 (macro-elements, side1 = -1 on the boundary; the
 * pair as it was grouped), start vertex, end vertex, closed (0/1), offset of
 * the macro-edge's first item; items (if not NULL) [n_items][2]: mesh edge
 * and direction (+1: lo -> hi) in arc-length order. */
hdgmg_status hdgmg_umesh_plan_macro_edges(const hdgmg_umesh_plan* plan, int32_t t,
                                          int64_t* counts, int32_t* info,
                                          int32_t* items);

/* ---- solver context ------------------------------------------------------ */

typedef struct hdgmg_umesh hdgmg_umesh;

/* The options hdgmg_umesh_create uses when given NULL: hdgmg_default_opts
 * with omega = 0.8, m_fine = 2, m_max = 4.  On meshes with irregular
 * elements the undamped edge block-Jacobi smoother is not convergent on its
 * own (more smoothing steps make the V-cycle worse), so it is damped and
 * applied twice on the finest level, doubling per level up to 4. */
void hdgmg_umesh_default_opts(hdgmg_opts* opts);

/* Create a context on the current device: builds the plan, uploads it and
 * allocates every buffer.  Options used: m_fine, m_growth, m_max,
 * local_corr, omega, krylov (NONE or CG; GMRES: EINVAL), max_it, rtol,
 * precision (opts NULL: hdgmg_umesh_default_opts).  precision FP64: the
 * whole path in FP64; FP32: the V-cycle on FP32 copies of every level
 * operator, block-Jacobi inverse, transfer block and the coarsest inverse,
 * inside the FP64 outer iteration (FP64 operator, residual, dot products);
 * FP32_IR and BF16: EINVAL.  smoother must be BLOCK_JACOBI (EINVAL
 * otherwise).
 * EINVAL also when a macro-element's local system exceeds 160 unknowns, a
 * macro-element has more than 64 macro-edges, or the coarsest level exceeds
 * 1024 unknowns.  stream: a cudaStream_t (NULL =
 * legacy default stream). */
hdgmg_status hdgmg_umesh_create(hdgmg_umesh** ctx,
                                const hdgmg_umesh_problem* problem,
                                const hdgmg_opts* opts, void* stream);

/* Set-up: log_kappa device [n_elem] FP64.  Element condensation with the
 * element geometry (A_e = kappa K_e + tau I - W_e^T S_e^-1 W_e, S_e =
 * kappa G_e + tau E_e Cholesky-factored per element and kept for the
 * right-hand side and the recovery), p-coarsening, the Schur complements of
 * every macro-element (eqs. n_1_Ik, coarse), block-Jacobi inverses and the
 * dense factorisation of the coarsest level.  EBREAKDOWN on a non-positive
 * pivot. */
hdgmg_status hdgmg_umesh_setup(hdgmg_umesh* ctx, const double* log_kappa);

/* Solve: f device [n_elem][(p+1)^2]; lambda device [n_edges][p+1] out
 * (boundary entries 0); u device [n_elem][(p+1)^2] out or NULL; q device
 * [n_elem][2][(p+1)^2] out or NULL; info host out or NULL.  ENOCONV still
 * writes the last iterate. */
hdgmg_status hdgmg_umesh_solve(hdgmg_umesh* ctx, const double* f, double* lambda,
                               double* u, double* q, hdgmg_info* info);

/* Level sizes: out[0] = unknowns, out[1] = (macro-)elements, out[2] =
 * modes per macro-edge, out[3] = padded element size nd_max. */
hdgmg_status hdgmg_umesh_level_sizes(const hdgmg_umesh* ctx, int32_t level,
                                     int64_t* out);

/* Element operators of a level after set-up: A device [n_el][nd_max][nd_max]
 * FP64 out (symmetric, zero padding; EINVAL before the first set-up), dofs
 * host [n_el][nd_max] out: the level-vector index of every row (-1: padding
 * or a boundary edge).  Either pointer may be NULL. */
hdgmg_status hdgmg_umesh_element_matrices(const hdgmg_umesh* ctx, int32_t level,
                                          double* A, int32_t* dofs);

/* y = A_level x (device level vectors). */
hdgmg_status hdgmg_umesh_apply(hdgmg_umesh* ctx, int32_t level, const double* x,
                               double* y);

/* z = B r: one V-cycle of Algorithm 1 on the finest level (device, FP64 in
 * and out; the cycle itself in the context's precision). */
hdgmg_status hdgmg_umesh_vcycle(hdgmg_umesh* ctx, const double* r, double* z);

void hdgmg_umesh_destroy(hdgmg_umesh* ctx);

#ifdef __cplusplus
}
#endif

#endif /* HDGMG_UMESH_H */
