// Work items of the P1 levels (two trace modes per edge, Sec. 3.1.2): the
// block-Jacobi sweep and the residual (Sec. 4.1), the local correction (eq.
// localCorrection), restriction (eq. n_1_Qk) and prolongation (eq. n_1_Ik),
// and their fused forms.  Shared by the launched kernels and the persistent
// V-cycle.  The storage (NS: full row-major; else packed symmetric) and the
// local edge of each element are compile-time, so every operator entry's
// offset is a constant times the element count; level sizes are divided by
// multiply-shift (FastDiv); indices are 32-bit.  The accumulation order of
// every sum is that of the element-centric definitions (row by row, column
// 0 to 7), so the results do not depend on which kernel runs an item.
// Requires c_Jc and c_Jcf (the child injection) in the including translation unit.
#pragma once

#include "k_common.cuh"

namespace hdgmg {

// child injection J_c[c][fine mode][coarse mode] in the cycle's precision
template <typename T>
static __device__ __forceinline__ T jc(int c, int kf, int kc);
template <>
__device__ __forceinline__ float jc<float>(int c, int kf, int kc) {
  return c_Jcf[c][kf][kc];
}
template <>
__device__ __forceinline__ double jc<double>(int c, int kf, int kc) {
  return c_Jc[c][kf][kc];
}

static __device__ __forceinline__ int fdiv(int x, const FastDiv& f) {
  return (int)((__umulhi((unsigned)x, f.m) + (unsigned)x) >> f.s);
}

// Dirichlet edge test from the edge's grid position
static __device__ __forceinline__ bool p1_bnd(const P1Geom& g, int E) {
  if (E < g.nvert) {
    const int j = fdiv(E, g.dn1), i = E - j * (g.n + 1);
    return i == 0 || i == g.n;
  }
  const int u = E - g.nvert, j = fdiv(u, g.dn);
  return j == 0 || j == g.n;
}

// rows 2 LE and 2 LE + 1 of element (ei, ej) times x
template <typename T, bool NS, int LE>
__device__ __forceinline__ void p1_rows(const P1Geom& g, const T* __restrict__ A, const T* x, int ei,
                                        int ej, T& s0, T& s1) {
  const int K = ej * g.n + ei;
  const int e0 = ej * (g.n + 1) + ei, e2 = g.nvert + ej * g.n + ei;
  const int ed[4] = {e0, e0 + 1, e2, e2 + g.n};
  const T* AK = A + K;
  T a = T(0), b = T(0);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const T xc = x[(c & 1) * g.nedge + ed[c >> 1]];
    const T a0 = AK[(NS ? (2 * LE) * 8 + c : pk_any(2 * LE, c)) * g.nE];
    const T a1 = AK[(NS ? (2 * LE + 1) * 8 + c : pk_any(2 * LE + 1, c)) * g.nE];
    a += a0 * xc;
    b += a1 * xc;
  }
  s0 = a;
  s1 = b;
}

// (A x)_E on edge E from its two elements; false (nothing computed) on a
// Dirichlet edge
template <typename T, bool NS>
__device__ __forceinline__ bool p1_acc(const P1Geom& g, const T* __restrict__ A, const T* x, int E,
                                       T& acc0, T& acc1) {
  T s00, s01, s10, s11;
  if (E < g.nvert) {                      // vertical: left element (its right edge), right one
    const int j = fdiv(E, g.dn1), i = E - j * (g.n + 1);
    if (i == 0 || i == g.n) return false;
    p1_rows<T, NS, 1>(g, A, x, i - 1, j, s00, s01);
    p1_rows<T, NS, 0>(g, A, x, i, j, s10, s11);
  } else {                                // horizontal: element below (its top edge), above
    const int u = E - g.nvert, j = fdiv(u, g.dn), i = u - j * g.n;
    if (j == 0 || j == g.n) return false;
    p1_rows<T, NS, 3>(g, A, x, i, j - 1, s00, s01);
    p1_rows<T, NS, 2>(g, A, x, i, j, s10, s11);
  }
  acc0 = s00 + s10;
  acc1 = s01 + s11;
  return true;
}

// D_E^-1 d (packed [d00, d10, d11] or full [d00, d01, d10, d11])
template <typename T, bool NS>
__device__ __forceinline__ void p1_dinv(const P1Geom& g, const T* __restrict__ Dinv, int E, T d0,
                                        T d1, T& u0, T& u1) {
  const T a00 = Dinv[E], a01 = Dinv[g.nedge + E], a10 = Dinv[2 * g.nedge + E];
  if (NS) {
    u0 = a00 * d0 + a01 * d1;
    u1 = a10 * d0 + Dinv[3 * g.nedge + E] * d1;
  } else {
    u0 = a00 * d0 + a01 * d1;
    u1 = a01 * d0 + a10 * d1;
  }
}

// SWEEP: out_E = x_E + omega D_E^-1 (r_E - (A x)_E); else out_E = (A x)_E;
// Dirichlet edges get 0.  x != out.
template <typename T, bool NS, bool SWEEP>
__device__ __forceinline__ void p1_edge(const P1Geom& g, const T* __restrict__ A,
                                        const T* __restrict__ Dinv, const T* r, const T* x, T* out,
                                        T omega, int E) {
  T acc0, acc1;
  if (!p1_acc<T, NS>(g, A, x, E, acc0, acc1)) {
    out[E] = T(0);
    out[g.nedge + E] = T(0);
    return;
  }
  if (SWEEP) {
    T u0, u1;
    p1_dinv<T, NS>(g, Dinv, E, r[E] - acc0, r[g.nedge + E] - acc1, u0, u1);
    out[E] = x[E] + omega * u0;
    out[g.nedge + E] = x[g.nedge + E] + omega * u1;
  } else {
    out[E] = acc0;
    out[g.nedge + E] = acc1;
  }
}

// first block-Jacobi sweep from e = 0: e_E = omega D_E^-1 r_E (interior edges)
template <typename T, bool NS>
__device__ __forceinline__ void p1_first(const P1Geom& g, const T* __restrict__ Dinv, const T* r,
                                         T* e, T omega, int E) {
  if (p1_bnd(g, E)) return;
  const T d[2] = {r[E], r[g.nedge + E]};
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    T s = T(0);
#pragma unroll
    for (int b = 0; b < 2; ++b) s += Dinv[(NS ? a * 2 + b : pk_any(a, b)) * g.nedge + E] * d[b];
    e[a * g.nedge + E] = omega * s;
  }
}

// the p-restriction J_N^T (r0 - y0) of the level above into r1 (modes 0, 1),
// y0 reset on all nd0 modes, and the first sweep e1 = omega D1^-1 r1
template <typename T, bool NS>
__device__ __forceinline__ void p1_first_restrict_p(const P1Geom& g, int nd0,
                                                    const T* __restrict__ Dinv1, const T* r0, T* y0,
                                                    T* r1, T* e1, T omega, int E) {
  const int ne = g.nedge;
  const T d0 = r0[E] - y0[E], d1 = r0[ne + E] - y0[ne + E];
  for (int k = 0; k < nd0; ++k) y0[k * ne + E] = T(0);
  r1[E] = d0;
  r1[ne + E] = d1;
  if (p1_bnd(g, E)) return;
  T u0, u1;
  p1_dinv<T, NS>(g, Dinv1, E, d0, d1, u0, u1);
  e1[E] = omega * u0;
  e1[ne + E] = omega * u1;
}

// --------------------------------------------- macro-element geometry
// Macro-element C = (I, J) of the coarse level covers fine elements
// (2I..2I+1, 2J..2J+1).  Interior edges ie: 0 v(2I+1, 2J), 1 v(2I+1, 2J+1),
// 2 h(2I, 2J+1), 3 h(2I+1, 2J+1); perimeter child edges (me, c): 0 left
// v(2I, 2J+c), 1 right v(2I+2, 2J+c), 2 bottom h(2I+c, 2J), 3 top
// h(2I+c, 2J+2).  Coarse edges of C: 0 left, 1 right, 2 bottom, 3 top.
struct MacroEdges {
  int ie[4], pe[8], ce[4];
};
static __device__ __forceinline__ void macro_edges(const P1Geom& g, int I, int J, MacroEdges& m) {
  const int n = g.n;
  const int v0 = 2 * J * (n + 1) + 2 * I;            // v(2I, 2J)
  const int h0 = g.nvert + 2 * J * n + 2 * I;         // h(2I, 2J)
  m.ie[0] = v0 + 1;
  m.ie[1] = v0 + 1 + (n + 1);
  m.ie[2] = h0 + n;
  m.ie[3] = h0 + n + 1;
  m.pe[0] = v0;                 // (me 0, c 0)
  m.pe[1] = v0 + (n + 1);       // (me 0, c 1)
  m.pe[2] = v0 + 2;
  m.pe[3] = v0 + 2 + (n + 1);
  m.pe[4] = h0;
  m.pe[5] = h0 + 1;
  m.pe[6] = h0 + 2 * n;
  m.pe[7] = h0 + 2 * n + 1;
  const int nc = g.nc;
  m.ce[0] = J * (nc + 1) + I;
  m.ce[1] = m.ce[0] + 1;
  m.ce[2] = g.nvc + J * nc + I;
  m.ce[3] = m.ce[2] + nc;
}

// local correction e_I = A_II^-1 r_I + Y e_B, one item per (C, interior dof
// a): t = a nC + C
template <typename T, bool NS>
__device__ __forceinline__ void p1_lc(const P1Geom& g, const T* __restrict__ AIIinv,
                                      const T* __restrict__ Y, const T* r, T* e, int t) {
  const int a = fdiv(t, g.dnC), C = t - a * g.nC;
  const int J = fdiv(C, g.dnc), I = C - J * g.nc;
  MacroEdges m;
  macro_edges(g, I, J, m);
  const int ne = g.nedge, nC = g.nC;
  const T* Ai = AIIinv + C;
  const T* Yc = Y + (a * 16) * nC + C;
  T s = T(0);
#pragma unroll
  for (int ie = 0; ie < 4; ++ie)
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int kk = ie * 2 + k;
      s += Ai[(NS ? a * 8 + kk : pk_any(a, kk)) * nC] * r[k * ne + m.ie[ie]];
    }
#pragma unroll
  for (int b = 0; b < 8; ++b)
#pragma unroll
    for (int k = 0; k < 2; ++k) s += Yc[(b * 2 + k) * nC] * e[k * ne + m.pe[b]];
  e[(a & 1) * ne + m.ie[a >> 1]] = s;
}

// coarse edge E: its two fine child edges, and its macro-elements with the
// coarse-edge slot mes in each (vertical: left C (its right edge), right C;
// horizontal: C below (top edge), C above); false for a Dirichlet coarse edge
struct CoarseEdge {
  int ch[2], C[2];
  bool vertical;
};
static __device__ __forceinline__ bool coarse_edge(const P1Geom& g, int E, CoarseEdge& q) {
  const int n = g.n, nc = g.nc;
  if (E < g.nvc) {
    const int J = fdiv(E, g.dnc1), I = E - J * (nc + 1);
    if (I == 0 || I == nc) return false;
    q.vertical = true;
    q.ch[0] = 2 * J * (n + 1) + 2 * I;
    q.ch[1] = q.ch[0] + (n + 1);
    q.C[0] = J * nc + I - 1;
    q.C[1] = J * nc + I;
  } else {
    const int u = E - g.nvc, J = fdiv(u, g.dnc), I = u - J * nc;
    if (J == 0 || J == nc) return false;
    q.vertical = false;
    q.ch[0] = g.nvert + 2 * J * n + 2 * I;
    q.ch[1] = q.ch[0] + 1;
    q.C[0] = (J - 1) * nc + I;
    q.C[1] = J * nc + I;
  }
  return true;
}

// r_c = J^T s_B + Rt^T s_I with s = r - y, one item per (coarse edge E,
// coarse mode kc): t = kc nedc + E
template <typename T>
__device__ __forceinline__ void p1_restrict(const P1Geom& g, const T* __restrict__ Rt, const T* r,
                                            const T* y, T* rc, int t) {
  const int kc = t >= g.nedc ? 1 : 0, E = t - kc * g.nedc;
  CoarseEdge q;
  if (!coarse_edge(g, E, q)) {
    rc[t] = T(0);
    return;
  }
  const int ne = g.nedge, nC = g.nC;
  T acc = T(0);
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const T s0 = r[q.ch[c]] - y[q.ch[c]];
    const T s1 = r[ne + q.ch[c]] - y[ne + q.ch[c]];
    acc += jc<T>(c, 0, kc) * s0 + jc<T>(c, 1, kc) * s1;
  }
  // coarse-edge slot of E in each macro-element: vertical 1 / 0, horizontal 3 / 2
  const int mes0 = q.vertical ? 1 : 3;
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const int C = q.C[side];
    const int J = fdiv(C, g.dnc), I = C - J * g.nc;
    MacroEdges m;
    macro_edges(g, I, J, m);
    const T* Rc = Rt + ((mes0 - side) * 2 + kc) * nC + C;
#pragma unroll
    for (int ie = 0; ie < 4; ++ie)
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const T s = r[k * ne + m.ie[ie]] - y[k * ne + m.ie[ie]];
        acc += Rc[((ie * 2 + k) * 8) * nC] * s;
      }
  }
  rc[t] = acc;
}

// the coarser level's first sweep at coarse edge E after r_c is formed
template <typename T, bool NS>
__device__ __forceinline__ void p1_coarse_first(const P1Geom& g, const T* __restrict__ Dinvc,
                                                const T* rc, T* ec, T omega, int E) {
  const int nedc = g.nedc;
  const T d[2] = {rc[E], rc[nedc + E]};
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    T s = T(0);
#pragma unroll
    for (int b = 0; b < 2; ++b) s += Dinvc[(NS ? a * 2 + b : pk_any(a, b)) * nedc + E] * d[b];
    ec[a * nedc + E] = omega * s;
  }
}

// restriction into both modes of coarse edge E, then (ec != null) the
// coarser level's first sweep at E
template <typename T, bool NS>
__device__ __forceinline__ void p1_restrict_first(const P1Geom& g, const T* __restrict__ Rt,
                                                  const T* r, const T* y, T* rc,
                                                  const T* __restrict__ Dinvc, T* ec, T omega,
                                                  int E) {
  p1_restrict<T>(g, Rt, r, y, rc, E);
  p1_restrict<T>(g, Rt, r, y, rc, g.nedc + E);
  CoarseEdge q;
  if (ec && coarse_edge(g, E, q)) p1_coarse_first<T, NS>(g, Dinvc, rc, ec, omega, E);
}

// After a local correction the residual vanishes on the interior edges of
// every macro-element (e_I solves the interior equations of the
// macro-element), so Q_{k-1} s = J^T s_B: one item per coarse edge E forms
// the residual r - A e on its two child edges and J^T of it into both
// modes, then (ec != null) the coarser level's first sweep at E.  Omitting
// Rt^T s_I drops rounding-level terms only.
template <typename T, bool NS>
__device__ __forceinline__ void p1_resid_restrict(const P1Geom& g, const T* __restrict__ A,
                                                  const T* r, const T* e, T* rc,
                                                  const T* __restrict__ Dinvc, T* ec, T omega,
                                                  int E) {
  const int nedc = g.nedc, ne = g.nedge;
  CoarseEdge q;
  if (!coarse_edge(g, E, q)) {
    rc[E] = T(0);
    rc[nedc + E] = T(0);
    return;
  }
  T acc[2] = {T(0), T(0)};
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    T y0, y1;
    p1_acc<T, NS>(g, A, e, q.ch[c], y0, y1);   // child edges of an interior coarse edge are interior
    const T s0 = r[q.ch[c]] - y0;
    const T s1 = r[ne + q.ch[c]] - y1;
#pragma unroll
    for (int kc = 0; kc < 2; ++kc) acc[kc] += jc<T>(c, 0, kc) * s0 + jc<T>(c, 1, kc) * s1;
  }
  rc[E] = acc[0];
  rc[nedc + E] = acc[1];
  if (ec) p1_coarse_first<T, NS>(g, Dinvc, rc, ec, omega, E);
}

// The same with one item per (coarse edge E, child c), t = 2 E + c: each lane
// of an adjacent pair forms its child's residual and J^T contribution, the
// pair adds them by a shuffle (the c = 0 lane, in the order of
// p1_resid_restrict) and the c = 0 lane writes r_c and the first sweep.  Both
// lanes of a pair are always active together.
template <typename T, bool NS>
__device__ __forceinline__ void p1_resid_restrict2(const P1Geom& g, const T* __restrict__ A,
                                                   const T* r, const T* e, T* rc,
                                                   const T* __restrict__ Dinvc, T* ec, T omega,
                                                   int t) {
  const int nedc = g.nedc, ne = g.nedge;
  const int E = t >> 1, c = t & 1;
  CoarseEdge q;
  const bool interior = coarse_edge(g, E, q);
  T t0 = T(0), t1 = T(0);
  if (interior) {
    T y0, y1;
    p1_acc<T, NS>(g, A, e, q.ch[c], y0, y1);
    const T s0 = r[q.ch[c]] - y0;
    const T s1 = r[ne + q.ch[c]] - y1;
    t0 = jc<T>(c, 0, 0) * s0 + jc<T>(c, 1, 0) * s1;
    t1 = jc<T>(c, 0, 1) * s0 + jc<T>(c, 1, 1) * s1;
  }
  const unsigned mask = __activemask();
  const T o0 = __shfl_xor_sync(mask, t0, 1), o1 = __shfl_xor_sync(mask, t1, 1);
  if (c) return;
  if (!interior) {
    rc[E] = T(0);
    rc[nedc + E] = T(0);
    return;
  }
  rc[E] = (T(0) + t0) + o0;
  rc[nedc + E] = (T(0) + t1) + o1;
  if (ec) p1_coarse_first<T, NS>(g, Dinvc, rc, ec, omega, E);
}

// e_I += Pi e_c(C): one item per (C, interior dof a), t = a nC + C; e_B += J
// e_c: one item per (coarse edge E, half c), t = 8 nC + c nedc + E.  Every
// fine edge is touched exactly once, where y is reset.
template <typename T>
__device__ __forceinline__ void p1_prolong(const P1Geom& g, const T* __restrict__ Pi, const T* ec,
                                           T* e, T* y, int t) {
  const int nC = g.nC, nedc = g.nedc, ne = g.nedge;
  if (t < 8 * nC) {
    const int a = fdiv(t, g.dnC), C = t - a * nC;
    const int J = fdiv(C, g.dnc), I = C - J * g.nc;
    MacroEdges m;
    macro_edges(g, I, J, m);
    const T* Pc = Pi + (a * 8) * nC + C;
    T s = T(0);
#pragma unroll
    for (int me = 0; me < 4; ++me) {
      s += Pc[(me * 2) * nC] * ec[m.ce[me]];
      s += Pc[(me * 2 + 1) * nC] * ec[nedc + m.ce[me]];
    }
    const int ix = (a & 1) * ne + m.ie[a >> 1];
    e[ix] += s;
    y[ix] = T(0);
    return;
  }
  const int u = t - 8 * nC;
  if (u >= 2 * nedc) return;
  const int c = u >= nedc ? 1 : 0, E = u - c * nedc;
  int ch;
  const int n = g.n, nc = g.nc;
  if (E < g.nvc) {
    const int J = fdiv(E, g.dnc1), I = E - J * (nc + 1);
    ch = (2 * J + c) * (n + 1) + 2 * I;
  } else {
    const int v = E - g.nvc, J = fdiv(v, g.dnc), I = v - J * nc;
    ch = g.nvert + 2 * J * n + 2 * I + c;
  }
  const T x0 = ec[E], x1 = ec[nedc + E];
#pragma unroll
  for (int kf = 0; kf < 2; ++kf) {
    const int ix = kf * ne + ch;
    e[ix] += jc<T>(c, kf, 0) * x0 + jc<T>(c, kf, 1) * x1;
    y[ix] = T(0);
  }
}

// Prolongation followed by the second local correction (step 5), from x into
// out (x != out): perimeter child edges out = x + J e_c; interior edges of C
// e_I = A_II^-1 r_I + Y (x_B + J e_c).  Step 5 replaces the prolonged
// interior values Pi e_c, so they are not formed.  Items as p1_prolong.
template <typename T, bool NS>
__device__ __forceinline__ void p1_prolong_lc(const P1Geom& g, const T* __restrict__ AIIinv,
                                              const T* __restrict__ Y, const T* r, const T* ec,
                                              const T* x, T* out, int t) {
  const int nC = g.nC, nedc = g.nedc, ne = g.nedge;
  if (t < 8 * nC) {
    const int a = fdiv(t, g.dnC), C = t - a * nC;
    const int J = fdiv(C, g.dnc), I = C - J * g.nc;
    MacroEdges m;
    macro_edges(g, I, J, m);
    const T* Ai = AIIinv + C;
    const T* Yc = Y + (a * 16) * nC + C;
    T s = T(0);
#pragma unroll
    for (int ie = 0; ie < 4; ++ie)
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int kk = ie * 2 + k;
        s += Ai[(NS ? a * 8 + kk : pk_any(a, kk)) * nC] * r[k * ne + m.ie[ie]];
      }
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int me = b >> 1, c = b & 1;
      const T x0 = ec[m.ce[me]], x1 = ec[nedc + m.ce[me]];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const T eb = x[k * ne + m.pe[b]] + (jc<T>(c, k, 0) * x0 + jc<T>(c, k, 1) * x1);
        s += Yc[(b * 2 + k) * nC] * eb;
      }
    }
    out[(a & 1) * ne + m.ie[a >> 1]] = s;
    return;
  }
  const int u = t - 8 * nC;
  if (u >= 2 * nedc) return;
  const int c = u >= nedc ? 1 : 0, E = u - c * nedc;
  int ch;
  const int n = g.n, nc = g.nc;
  if (E < g.nvc) {
    const int J = fdiv(E, g.dnc1), I = E - J * (nc + 1);
    ch = (2 * J + c) * (n + 1) + 2 * I;
  } else {
    const int v = E - g.nvc, J = fdiv(v, g.dnc), I = v - J * nc;
    ch = g.nvert + 2 * J * n + 2 * I + c;
  }
  const T x0 = ec[E], x1 = ec[nedc + E];
#pragma unroll
  for (int kf = 0; kf < 2; ++kf) {
    const int ix = kf * ne + ch;
    out[ix] = x[ix] + (jc<T>(c, kf, 0) * x0 + jc<T>(c, kf, 1) * x1);
  }
}

}  // namespace hdgmg
