"""CPU FP64 oracle for the HDG trace system and its DtN-based geometric multigrid.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the C-ABI library under
``paper_1811_09909_gb300/`` and its Python binding) may import, call or link
anything in this package; only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

It is a plain, slow, deliberately different restatement of the method of
Wildey, Muralikrishnan and Bui-Thanh, "Unified geometric multigrid algorithm for
hybridized high-order finite element methods" (arXiv:1811.09909):

* ``refelem``  -- quadrature, Lagrange (volume) and orthonormal Legendre (trace)
  bases, written from their textbook definitions.
* ``hdg``      -- the HDG local equations of Sec. 2 (eqs. HDG_local1, HDG_local2,
  HDG_flux, conservation) assembled literally by over-integrated quadrature,
  static condensation by a general LU with partial pivoting of the full
  (q_x, q_y, u) block, global assembly of the trace system of Sec. 3
  (eq. trace_linear_system), sparse direct solve, local recovery, and a
  brute-force uncondensed solve; the hybridized interior penalty schemes
  SIPG-H, NIPG-H and IIPG-H of eq. IPG_H through the same condensation.
* ``mg``       -- the multigrid of Sec. 3: p-coarsening (Sec. 3.1.1),
  h-agglomeration with the interior/boundary split (Sec. 3.1.2,
  eq. trace_partition), prolongation and restriction (eqs. n_1_Ik, n_g1_Ik,
  n_1_Qk, n_g1_Qk), Galerkin coarse operators (eqs. coarse, Akm1, ANm1),
  edge block-Jacobi smoothing (Sec. 4.1), local correction (eq.
  localCorrection) and the V-cycle of Algorithm 1, all on global sparse
  matrices; outer fixed-point iteration, PCG and right-preconditioned GMRES.
* ``unstructured`` -- the same HDG element on bilinearly mapped quadrilaterals
  of an unstructured mesh, the seed-point agglomeration of Sec. 3.1.2 with
  recursive cuts into four, macro-edges parameterised by arc length (the
  remark in Sec. 3.1), J as an L2 projection by quadrature, and the hierarchy
  and V-cycle of ``mg`` on those levels.

Naming follows the usual HDG convention rather than the paper's: u is the
scalar, q = -kappa grad u the flux, lambda the trace of u.

Floating point: IEEE FP64 with round-to-nearest throughout.

Parity status of each function is stated in its docstring; functions without
an independent pin say "parity unpinned".
"""
