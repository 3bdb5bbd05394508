// Host-side plan of the unstructured-mesh multigrid (Sec. 3.1.2 seed-point
// agglomeration): mesh edges, partitions, macro-edges with their arc-length
// parameterisation, per-level index lists and the closed-form J blocks.
#pragma once
#include <string>
#include <vector>

#include "hdgmg_umesh.h"

namespace hdgmg {

// A macro-edge: ordered units of the next finer level with their directions,
// the mesh edges it covers in arc-length order (+1: lo -> hi) and its sides.
struct UChain {
  std::vector<int> units, dirs, edges, edirs;
  int start = -1, end = -1, s0 = -1, s1 = -1;
  double length = 0.0;
  bool closed = false;
};

// One multigrid level: (macro-)elements with their macro-edge slots.
struct UPlanLevel {
  int nd = 0;              // modes per macro-edge
  int n_el = 0;            // elements / macro-elements
  int n_units = 0;         // macro-edges, boundary ones included
  int n_blk = 0;           // macro-edges carrying unknowns
  int nu = 0;              // slots per element (padded)
  int t = 0;               // partition level (0: the mesh)
  std::vector<int> unit_blk;      // macro-edge -> unknown block or -1
  std::vector<int> el_slot;       // [n_el][nu] unknown block or -1
  std::vector<int> blk_t0, blk_t1;  // per block: el*nu + slot on its two sides
};

// h-coarsening data from level f to level f+1, per coarse macro-element E:
// local blocks (interior of E first, then the units of E's macro-edges in
// E's slot order and arc-length order), children with slot maps, J_E.
struct UPlanH {
  int n_E = 0;
  int nloc_max = 0, nI_max = 0, nB_max = 0, nc_max = 0;
  std::vector<int> loc_ptr, loc_blk, nI, own;
  std::vector<int> ch_ptr, ch_el, ch_map;   // ch_map [children][nu_f]
  std::vector<long long> J_off, AI_off, Y_off;
  std::vector<double> J;                     // per E row-major [2 nB][2 nc]
};

struct UPlan {
  int p = 0, E = 0, nvert = 0, ne = 0;
  double tau = 0.0;
  std::vector<double> xy;
  std::vector<int> quads, ev, elem_edges, ee;
  std::vector<std::vector<int>> parts;       // P_0 .. P_{H-1}
  std::vector<std::vector<UChain>> chains;   // t = 0 (mesh edges) .. H (P_0)
  std::vector<UPlanLevel> levels;            // multigrid levels, finest first
  std::vector<UPlanH> hc;                    // hc[i]: level first_h+i -> +1
  int first_h = 0;
  long long trace_dofs = 0;
};

// Builds the plan; returns false with a message for invalid input.
bool build_uplan(const hdgmg_umesh_problem& pr, UPlan& plan, std::string& err);

}  // namespace hdgmg
