// Host plan of the unstructured-mesh multigrid: seed-point agglomeration
// (Sec. 3.1.2), macro-edges and their parameterisation (the remark in Sec.
// 3.1), the index lists of every level and the J blocks between levels.
// Built with floating-point contraction off: every integer decision (nearest
// seed, bisection order) comes from the same fp64 operations on any host.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <utility>

#include "internal.h"
#include "umesh_plan.h"

namespace hdgmg {
namespace {

void centroid(const UPlan& P, int e, double& cx, double& cy) {
  const int* q = &P.quads[4 * e];
  cx = (((P.xy[2 * q[0]] + P.xy[2 * q[1]]) + P.xy[2 * q[2]]) + P.xy[2 * q[3]]) * 0.25;
  cy = (((P.xy[2 * q[0] + 1] + P.xy[2 * q[1] + 1]) + P.xy[2 * q[2] + 1]) + P.xy[2 * q[3] + 1]) * 0.25;
}

bool mesh_edges(UPlan& P, std::string& err) {
  std::vector<std::pair<long long, int>> keys;   // (lo * nvert + hi, element*4 + j)
  keys.reserve(4 * (size_t)P.E);
  for (int e = 0; e < P.E; ++e)
    for (int j = 0; j < 4; ++j) {
      const int a = P.quads[4 * e + j], b = P.quads[4 * e + (j + 1) % 4];
      const int lo = std::min(a, b), hi = std::max(a, b);
      keys.push_back({(long long)lo * P.nvert + hi, 4 * e + j});
    }
  std::sort(keys.begin(), keys.end());
  P.elem_edges.assign(4 * (size_t)P.E, -1);
  P.ev.clear();
  P.ee.clear();
  long long prev = -1;
  for (const auto& k : keys) {
    if (k.first != prev) {
      P.ev.push_back((int)(k.first / P.nvert));
      P.ev.push_back((int)(k.first % P.nvert));
      P.ee.push_back(-1);
      P.ee.push_back(-1);
      prev = k.first;
    }
    const int g = (int)P.ev.size() / 2 - 1;
    P.elem_edges[k.second] = g;
  }
  P.ne = (int)P.ev.size() / 2;
  for (int e = 0; e < P.E; ++e)          // ascending elements per edge
    for (int j = 0; j < 4; ++j) {
      const int g = P.elem_edges[4 * e + j];
      if (P.ee[2 * g] < 0) P.ee[2 * g] = e;
      else if (P.ee[2 * g + 1] < 0 && P.ee[2 * g] != e) P.ee[2 * g + 1] = e;
      else { err = "non-conforming mesh: an edge shared by more than two element sides"; return false; }
    }
  return true;
}

std::vector<int> seed_partition(const UPlan& P, const std::vector<double>& seeds) {
  const int ns = (int)seeds.size() / 2;
  std::vector<int> best(P.E, 0);
  for (int e = 0; e < P.E; ++e) {
    double cx, cy;
    centroid(P, e, cx, cy);
    double bd = 0.0;
    for (int s = 0; s < ns; ++s) {
      const double dx = cx - seeds[2 * s], dy = cy - seeds[2 * s + 1];
      const double d = dx * dx + dy * dy;
      if (s == 0 || d < bd) { bd = d; best[e] = s; }
    }
  }
  std::vector<int> remap(ns, -1);
  for (int e = 0; e < P.E; ++e) remap[best[e]] = 1;
  int k = 0;
  for (int s = 0; s < ns; ++s)
    if (remap[s] > 0) remap[s] = k++;
  for (int e = 0; e < P.E; ++e) best[e] = remap[best[e]];
  return best;
}

void bisect(const std::vector<int>& el, const std::vector<double>& c,
            std::vector<int>& first, std::vector<int>& second) {
  double xmin = c[2 * el[0]], xmax = xmin, ymin = c[2 * el[0] + 1], ymax = ymin;
  for (int e : el) {
    xmin = std::min(xmin, c[2 * e]); xmax = std::max(xmax, c[2 * e]);
    ymin = std::min(ymin, c[2 * e + 1]); ymax = std::max(ymax, c[2 * e + 1]);
  }
  const int axis = (xmax - xmin) >= (ymax - ymin) ? 0 : 1;
  std::vector<int> order(el);
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    const double ka = c[2 * a + axis], kb = c[2 * b + axis];
    return ka < kb || (ka == kb && a < b);
  });
  const size_t half = el.size() / 2;
  first.assign(order.begin(), order.begin() + half);
  second.assign(order.begin() + half, order.end());
  std::sort(first.begin(), first.end());
  std::sort(second.begin(), second.end());
}

std::vector<int> split_partition(const std::vector<int>& part, const std::vector<double>& c) {
  const int nmac = *std::max_element(part.begin(), part.end()) + 1;
  std::vector<std::vector<int>> members(nmac);
  for (int e = 0; e < (int)part.size(); ++e) members[part[e]].push_back(e);
  std::vector<int> out(part.size(), -1);
  int nxt = 0;
  for (int m = 0; m < nmac; ++m) {
    std::vector<std::vector<int>> pieces;
    if (members[m].size() == 1) {
      pieces.push_back(members[m]);
    } else {
      std::vector<int> a, b;
      bisect(members[m], c, a, b);
      for (const auto* half : {&a, &b}) {
        if (half->size() <= 1) {
          pieces.push_back(*half);
        } else {
          std::vector<int> x, y;
          bisect(*half, c, x, y);
          pieces.push_back(x);
          pieces.push_back(y);
        }
      }
    }
    for (const auto& pc : pieces) {
      if (pc.empty()) continue;
      for (int e : pc) out[e] = nxt;
      ++nxt;
    }
  }
  return out;
}

// Links the units of the finer level into the macro-edges of the coarser
// partition (parent: finer macro-element -> coarser one).  interior receives
// (unit, coarse macro) of the units inside one coarse macro-element.
// Groups are formed by sorting (pair of coarse sides, unit); inside a group
// the unit ends are sorted by vertex, and two units are linked at a vertex
// where exactly two unit ends of the group meet.  Every decision depends only
// on the indices, so the order of the work does not change the result.
void link_units(const std::vector<UChain>& units, const std::vector<int>& parent,
                std::vector<UChain>& chains, std::vector<std::pair<int, int>>& interior) {
  struct KU { int a, b, u; };
  std::vector<KU> sk;
  sk.reserve(units.size());
  interior.clear();
  for (int ui = 0; ui < (int)units.size(); ++ui) {
    const UChain& u = units[ui];
    const int pa = parent[u.s0];
    const int pb = u.s1 >= 0 ? parent[u.s1] : -1;
    if (pa == pb) { interior.push_back({ui, pa}); continue; }
    if (pb >= 0) sk.push_back({std::min(pa, pb), std::max(pa, pb), ui});
    else sk.push_back({pa, -1, ui});
  }
  std::sort(sk.begin(), sk.end(), [](const KU& x, const KU& y) {
    return x.a < y.a || (x.a == y.a && (x.b < y.b || (x.b == y.b && x.u < y.u)));
  });
  chains.clear();
  std::vector<std::pair<int, int>> inc;          // (vertex, local unit) per unit end
  std::vector<int> nlink, comp, stack;
  std::vector<std::pair<int, int>> lk;           // [local][2]: (vertex, other local unit)
  std::vector<char> seen;
  for (size_t g0 = 0; g0 < sk.size();) {
    size_t g1 = g0;
    while (g1 < sk.size() && sk[g1].a == sk[g0].a && sk[g1].b == sk[g0].b) ++g1;
    const int n = (int)(g1 - g0);
    auto U = [&](int li) -> const UChain& { return units[sk[g0 + li].u]; };
    auto uid = [&](int li) { return sk[g0 + li].u; };
    inc.clear();
    for (int li = 0; li < n; ++li) {
      inc.push_back({U(li).start, li});
      inc.push_back({U(li).end, li});
    }
    std::sort(inc.begin(), inc.end());
    nlink.assign(n, 0);
    lk.assign(2 * (size_t)n, {-1, -1});
    for (size_t k0 = 0; k0 < inc.size();) {
      size_t k1 = k0;
      while (k1 < inc.size() && inc[k1].first == inc[k0].first) ++k1;
      if (k1 - k0 == 2 && inc[k0].second != inc[k0 + 1].second) {
        const int x = inc[k0].second, y = inc[k0 + 1].second, v = inc[k0].first;
        lk[2 * x + nlink[x]++] = {v, y};
        lk[2 * y + nlink[y]++] = {v, x};
      }
      k0 = k1;
    }
    seen.assign(n, 0);
    for (int l0 = 0; l0 < n; ++l0) {              // ascending unit index
      if (seen[l0]) continue;
      comp.clear();
      stack.assign(1, l0);
      seen[l0] = 1;
      while (!stack.empty()) {
        const int x = stack.back();
        stack.pop_back();
        comp.push_back(x);
        for (int q = 0; q < nlink[x]; ++q) {
          const int y = lk[2 * x + q].second;
          if (!seen[y]) { seen[y] = 1; stack.push_back(y); }
        }
      }
      std::sort(comp.begin(), comp.end());        // local order = unit order
      UChain ch;
      ch.s0 = sk[g0].a;
      ch.s1 = sk[g0].b;
      if (comp.size() == 1) {
        const UChain& u = U(comp[0]);
        ch.units = {uid(comp[0])};
        ch.dirs = {1};
        ch.start = u.start;
        ch.end = u.end;
        ch.edges = u.edges;
        ch.edirs = u.edirs;
        ch.length = u.length;
        ch.closed = u.closed || u.start == u.end;
        chains.push_back(std::move(ch));
        continue;
      }
      std::vector<int> ends;
      for (int x : comp)
        if (nlink[x] == 1) ends.push_back(x);
      int first, v;
      bool closed;
      if (!ends.empty()) {
        auto free_vertex = [&](int x) {
          const int w = lk[2 * x].first;
          return U(x).start == w ? U(x).end : U(x).start;
        };
        const int fa = free_vertex(ends[0]), fb = free_vertex(ends[1]);
        if (fa != fb) {
          if (fa < fb) { first = ends[0]; v = fa; } else { first = ends[1]; v = fb; }
        } else {
          first = std::min(ends[0], ends[1]);
          v = fa;
        }
        closed = false;
      } else {
        v = -1;
        for (int x : comp)
          for (int q = 0; q < nlink[x]; ++q)
            if (v < 0 || lk[2 * x + q].first < v) v = lk[2 * x + q].first;
        first = -1;
        for (int x : comp)
          for (int q = 0; q < nlink[x]; ++q)
            if (lk[2 * x + q].first == v && (first < 0 || lk[2 * x + q].second < first)) first = lk[2 * x + q].second;
        closed = true;
      }
      int x = first, cur = v, prev = -1;
      ch.start = v;
      std::vector<int> order;
      while (true) {
        const UChain& u = U(x);
        const int d = u.start == cur ? 1 : -1;
        order.push_back(x);
        ch.dirs.push_back(d);
        cur = d == 1 ? u.end : u.start;
        int nxt = -1;
        for (int q = 0; q < nlink[x]; ++q)
          if (lk[2 * x + q].first == cur && lk[2 * x + q].second != prev) { nxt = lk[2 * x + q].second; break; }
        if (closed && order.size() == comp.size()) break;
        if (nxt < 0) break;
        prev = x;
        x = nxt;
        if (x == first) break;
      }
      ch.end = cur;
      ch.closed = closed;
      double length = 0.0;
      for (size_t i = 0; i < order.size(); ++i) {
        const UChain& u = U(order[i]);
        ch.units.push_back(uid(order[i]));
        if (ch.dirs[i] == 1) {
          ch.edges.insert(ch.edges.end(), u.edges.begin(), u.edges.end());
          ch.edirs.insert(ch.edirs.end(), u.edirs.begin(), u.edirs.end());
        } else {
          for (size_t k = u.edges.size(); k-- > 0;) {
            ch.edges.push_back(u.edges[k]);
            ch.edirs.push_back(-u.edirs[k]);
          }
        }
        length += u.length;
      }
      ch.length = length;
      chains.push_back(std::move(ch));
    }
    g0 = g1;
  }
  std::sort(chains.begin(), chains.end(), [](const UChain& a, const UChain& b) {
    return *std::min_element(a.units.begin(), a.units.end()) <
           *std::min_element(b.units.begin(), b.units.end());
  });
}

// J block [fine mode l][coarse mode k] of a unit of length l at arc offset
// s0 (direction d) in a macro-edge of length L: the coarse basis
// 1/sqrt(L), sqrt(3/L)(2s/L - 1) restricted to the unit is a + b tau (tau in
// [0, 1] along the unit), whose coefficients in the unit's orthonormal P_1
// basis are sqrt(l)(a + b/2) and sqrt(3 l) b / 6.
void j_block(double L, double l, double s0, int d, double out[2][2]) {
  const double c3 = std::sqrt(3.0 / L);
  const double a0 = 1.0 / std::sqrt(L), b0 = 0.0;
  double a1, b1;
  if (d == 1) { a1 = c3 * (2.0 * s0 / L - 1.0); b1 = c3 * 2.0 * l / L; }
  else { a1 = c3 * (2.0 * (s0 + l) / L - 1.0); b1 = -c3 * 2.0 * l / L; }
  out[0][0] = std::sqrt(l) * (a0 + b0 / 2.0);
  out[1][0] = std::sqrt(3.0 * l) * b0 / 6.0;
  out[0][1] = std::sqrt(l) * (a1 + b1 / 2.0);
  out[1][1] = std::sqrt(3.0 * l) * b1 / 6.0;
}

void mesh_level(const UPlan& P, int nd, UPlanLevel& L) {
  L.nd = nd;
  L.t = 0;
  L.n_el = P.E;
  L.n_units = P.ne;
  L.nu = 4;
  L.unit_blk.assign(P.ne, -1);
  int k = 0;
  for (int m = 0; m < P.ne; ++m)
    if (P.ee[2 * m + 1] >= 0) L.unit_blk[m] = k++;
  L.n_blk = k;
  L.el_slot.assign(4 * (size_t)P.E, -1);
  L.blk_t0.assign(k, -1);
  L.blk_t1.assign(k, -1);
  for (int e = 0; e < P.E; ++e)
    for (int j = 0; j < 4; ++j) {
      const int m = P.elem_edges[4 * e + j];
      const int b = L.unit_blk[m];
      L.el_slot[4 * e + j] = b;
      if (b < 0) continue;
      if (P.ee[2 * m] == e) L.blk_t0[b] = 4 * e + j;
      else L.blk_t1[b] = 4 * e + j;
    }
}

void chain_level(int n_el, const std::vector<UChain>& ch, int t, UPlanLevel& L) {
  L.nd = 2;
  L.t = t;
  L.n_el = n_el;
  L.n_units = (int)ch.size();
  L.unit_blk.assign(ch.size(), -1);
  std::vector<std::vector<int>> slots(n_el);
  int k = 0;
  for (int c = 0; c < (int)ch.size(); ++c) {
    if (ch[c].s1 < 0) continue;
    L.unit_blk[c] = k++;
    slots[ch[c].s0].push_back(c);
    slots[ch[c].s1].push_back(c);
  }
  L.n_blk = k;
  L.nu = 1;
  for (const auto& s : slots) L.nu = std::max(L.nu, (int)s.size());
  L.el_slot.assign((size_t)n_el * L.nu, -1);
  L.blk_t0.assign(k, -1);
  L.blk_t1.assign(k, -1);
  for (int E = 0; E < n_el; ++E)
    for (int s = 0; s < (int)slots[E].size(); ++s) {
      const int c = slots[E][s];
      const int b = L.unit_blk[c];
      L.el_slot[(size_t)E * L.nu + s] = b;
      if (ch[c].s0 == E) L.blk_t0[b] = E * L.nu + s;
      else L.blk_t1[b] = E * L.nu + s;
    }
}

}  // namespace

hdgmg_status fail_plan(hdgmg_status st, const std::string& msg) {
  set_last_error(msg);
  return st;
}

bool build_uplan(const hdgmg_umesh_problem& pr, UPlan& P, std::string& err) {
  if (pr.n_vert <= 0 || pr.n_elem <= 0 || !pr.xy || !pr.quads) { err = "empty mesh"; return false; }
  if (pr.p < 1 || pr.p > 8) { err = "p must be in 1..8"; return false; }
  if (!(pr.tau > 0.0)) { err = "tau must be positive"; return false; }
  if (pr.n_seeds <= 0 || !pr.seeds) { err = "at least one seed point is required"; return false; }
  P.p = pr.p;
  P.E = pr.n_elem;
  P.nvert = pr.n_vert;
  P.tau = pr.tau;
  P.xy.assign(pr.xy, pr.xy + 2 * (size_t)pr.n_vert);
  P.quads.assign(pr.quads, pr.quads + 4 * (size_t)pr.n_elem);
  for (int v : P.quads)
    if (v < 0 || v >= P.nvert) { err = "vertex index out of range"; return false; }
  for (int e = 0; e < P.E; ++e)        // convex and counter-clockwise: every corner turns left
    for (int j = 0; j < 4; ++j) {
      const int a = P.quads[4 * e + (j + 3) % 4], b = P.quads[4 * e + j], c = P.quads[4 * e + (j + 1) % 4];
      const double cr = (P.xy[2 * b] - P.xy[2 * a]) * (P.xy[2 * c + 1] - P.xy[2 * b + 1]) -
                        (P.xy[2 * b + 1] - P.xy[2 * a + 1]) * (P.xy[2 * c] - P.xy[2 * b]);
      if (!(cr > 0.0)) { err = "element " + std::to_string(e) + " is not convex and counter-clockwise"; return false; }
    }
  if (!mesh_edges(P, err)) return false;
  std::vector<double> seeds(pr.seeds, pr.seeds + 2 * (size_t)pr.n_seeds);
  std::vector<double> c(2 * (size_t)P.E);
  for (int e = 0; e < P.E; ++e) centroid(P, e, c[2 * e], c[2 * e + 1]);
  // partitions (Sec. 3.1.2): seeds, then recursive cuts in four
  P.parts.clear();
  std::vector<int> part = seed_partition(P, seeds);
  P.parts.push_back(part);
  while (true) {
    part = split_partition(part, c);
    const int nmac = *std::max_element(part.begin(), part.end()) + 1;
    if (2LL * nmac > P.E) break;
    P.parts.push_back(part);
  }
  const int H = (int)P.parts.size();
  // macro-edges, from the mesh edges up
  P.chains.assign(H + 1, {});
  std::vector<std::vector<std::pair<int, int>>> interior(H + 1);
  auto& mesh = P.chains[0];
  mesh.resize(P.ne);
  for (int m = 0; m < P.ne; ++m) {
    UChain& u = mesh[m];
    const int lo = P.ev[2 * m], hi = P.ev[2 * m + 1];
    u.units = {m};
    u.dirs = {1};
    u.edges = {m};
    u.edirs = {1};
    u.start = lo;
    u.end = hi;
    u.s0 = P.ee[2 * m];
    u.s1 = P.ee[2 * m + 1];
    u.length = std::hypot(P.xy[2 * hi] - P.xy[2 * lo], P.xy[2 * hi + 1] - P.xy[2 * lo + 1]);
  }
  std::vector<int> finer(P.E);
  std::iota(finer.begin(), finer.end(), 0);
  for (int t = 1; t <= H; ++t) {
    const std::vector<int>& coarse = P.parts[H - t];
    std::vector<int> parent(*std::max_element(finer.begin(), finer.end()) + 1, 0);
    for (int e = 0; e < P.E; ++e) parent[finer[e]] = coarse[e];
    link_units(P.chains[t - 1], parent, P.chains[t], interior[t]);
    finer = coarse;
  }
  // multigrid levels
  P.levels.clear();
  P.levels.emplace_back();
  mesh_level(P, P.p + 1, P.levels.back());
  P.trace_dofs = (long long)P.levels[0].n_blk * (P.p + 1);
  if (P.p > 1) {
    P.levels.emplace_back();
    mesh_level(P, 2, P.levels.back());
  }
  P.first_h = (int)P.levels.size() - 1;
  P.hc.clear();
  for (int t = 1; t <= H; ++t) {
    const std::vector<int>& coarse = P.parts[H - t];
    const int n_el = *std::max_element(coarse.begin(), coarse.end()) + 1;
    P.levels.emplace_back();
    chain_level(n_el, P.chains[t], t, P.levels.back());
    const UPlanLevel& Lf = P.levels[P.levels.size() - 2];
    const UPlanLevel& Lc = P.levels.back();
    const std::vector<UChain>& units_f = P.chains[t - 1];
    const std::vector<UChain>& chains_c = P.chains[t];
    // finer element -> coarse macro
    std::vector<int> parent(Lf.n_el, 0);
    {
      const std::vector<int>* fine_part = t >= 2 ? &P.parts[H - t + 1] : nullptr;
      for (int e = 0; e < P.E; ++e) parent[fine_part ? (*fine_part)[e] : e] = coarse[e];
    }
    std::vector<int> blk_chain(Lc.n_blk, -1);
    for (int c2 = 0; c2 < (int)chains_c.size(); ++c2)
      if (Lc.unit_blk[c2] >= 0) blk_chain[Lc.unit_blk[c2]] = c2;
    UPlanH h;
    h.n_E = n_el;
    std::vector<std::vector<int>> kids(n_el), inner(n_el);
    for (int f = 0; f < Lf.n_el; ++f) kids[parent[f]].push_back(f);
    for (const auto& iu : interior[t]) inner[iu.second].push_back(iu.first);
    std::vector<int> local(Lf.n_blk, -1);   // fine block -> local index in the current E
    h.loc_ptr.push_back(0);
    h.ch_ptr.push_back(0);
    h.J_off.push_back(0);
    h.AI_off.push_back(0);
    h.Y_off.push_back(0);
    for (int E = 0; E < n_el; ++E) {
      const int base = (int)h.loc_blk.size();
      for (int u : inner[E]) {
        const int b = Lf.unit_blk[u];
        if (b < 0) continue;
        local[b] = (int)h.loc_blk.size() - base;
        h.loc_blk.push_back(b);
        h.own.push_back(1);
      }
      const int nI = (int)h.loc_blk.size() - base;
      // B blocks: the units of E's macro-edges, slot order then arc order
      std::vector<std::pair<int, int>> bref;   // (coarse slot, position in chain)
      int nc = 0;                      // slots are filled from 0 without gaps
      while (nc < Lc.nu && Lc.el_slot[(size_t)E * Lc.nu + nc] >= 0) ++nc;
      for (int s = 0; s < nc; ++s) {
        const UChain& ch = chains_c[blk_chain[Lc.el_slot[(size_t)E * Lc.nu + s]]];
        for (size_t i = 0; i < ch.units.size(); ++i) {
          const int b = Lf.unit_blk[ch.units[i]];
          if (b < 0) continue;
          local[b] = (int)h.loc_blk.size() - base;
          h.loc_blk.push_back(b);
          h.own.push_back(ch.s0 == E ? 1 : 0);
          bref.push_back({s, (int)i});
        }
      }
      const int nB = (int)h.loc_blk.size() - base - nI;
      h.nI.push_back(nI);
      h.loc_ptr.push_back((int)h.loc_blk.size());
      h.nloc_max = std::max(h.nloc_max, nI + nB);
      h.nI_max = std::max(h.nI_max, nI);
      h.nB_max = std::max(h.nB_max, nB);
      h.nc_max = std::max(h.nc_max, nc);
      // J_E [2 nB][2 nc]
      const size_t j0 = h.J.size();
      h.J.resize(j0 + (size_t)4 * nB * nc, 0.0);
      for (int r = 0; r < nB; ++r) {
        const int s = bref[r].first, pos = bref[r].second;
        const UChain& ch = chains_c[blk_chain[Lc.el_slot[(size_t)E * Lc.nu + s]]];
        double s0 = 0.0;                 // arc offset of the unit (summed in chain order)
        for (int i = 0; i < pos; ++i) s0 += units_f[ch.units[i]].length;
        double blk[2][2];
        j_block(ch.length, units_f[ch.units[pos]].length, s0, ch.dirs[pos], blk);
        for (int l = 0; l < 2; ++l)
          for (int k = 0; k < 2; ++k)
            h.J[j0 + (size_t)(2 * r + l) * (2 * nc) + 2 * s + k] = blk[l][k];
      }
      h.J_off.push_back((long long)h.J.size());
      h.AI_off.push_back(h.AI_off.back() + 4LL * nI * nI);
      h.Y_off.push_back(h.Y_off.back() + 4LL * nI * nB);
      // children and their slot maps
      for (int f : kids[E]) {
        h.ch_el.push_back(f);
        for (int s = 0; s < Lf.nu; ++s) {
          const int b = Lf.el_slot[(size_t)f * Lf.nu + s];
          h.ch_map.push_back(b < 0 ? -1 : local[b]);
        }
      }
      h.ch_ptr.push_back((int)h.ch_el.size());
      for (size_t q = base; q < h.loc_blk.size(); ++q) local[h.loc_blk[q]] = -1;
    }
    P.hc.push_back(std::move(h));
  }
  return true;
}

}  // namespace hdgmg

// ---- C ABI: host-only plan ------------------------------------------------
struct hdgmg_umesh_plan {
  hdgmg::UPlan plan;
};

extern "C" {

hdgmg_status hdgmg_umesh_plan_create(hdgmg_umesh_plan** out, const hdgmg_umesh_problem* pr) {
  if (!out || !pr) return hdgmg::fail_plan(HDGMG_EINVAL, "null argument");
  *out = nullptr;
  auto* p = new (std::nothrow) hdgmg_umesh_plan;
  if (!p) return hdgmg::fail_plan(HDGMG_ENOMEM, "host allocation failed");
  std::string err;
  if (!hdgmg::build_uplan(*pr, p->plan, err)) {
    delete p;
    return hdgmg::fail_plan(HDGMG_EINVAL, err.c_str());
  }
  *out = p;
  return HDGMG_OK;
}

void hdgmg_umesh_plan_destroy(hdgmg_umesh_plan* p) { delete p; }

hdgmg_status hdgmg_umesh_plan_sizes(const hdgmg_umesh_plan* p, int64_t* out) {
  if (!p || !out) return hdgmg::fail_plan(HDGMG_EINVAL, "null argument");
  out[0] = p->plan.ne;
  out[1] = (int64_t)p->plan.parts.size();
  out[2] = (int64_t)p->plan.levels.size();
  out[3] = p->plan.trace_dofs;
  return HDGMG_OK;
}

hdgmg_status hdgmg_umesh_plan_edges(const hdgmg_umesh_plan* p, int32_t* ev) {
  if (!p || !ev) return hdgmg::fail_plan(HDGMG_EINVAL, "null argument");
  std::memcpy(ev, p->plan.ev.data(), p->plan.ev.size() * sizeof(int32_t));
  return HDGMG_OK;
}

hdgmg_status hdgmg_umesh_plan_partition(const hdgmg_umesh_plan* p, int32_t r, int32_t* out) {
  if (!p || !out) return hdgmg::fail_plan(HDGMG_EINVAL, "null argument");
  if (r < 0 || r >= (int32_t)p->plan.parts.size()) return hdgmg::fail_plan(HDGMG_EINVAL, "partition index out of range");
  std::memcpy(out, p->plan.parts[r].data(), p->plan.parts[r].size() * sizeof(int32_t));
  return HDGMG_OK;
}

hdgmg_status hdgmg_umesh_plan_macro_edges(const hdgmg_umesh_plan* p, int32_t t, int64_t* counts,
                                          int32_t* info, int32_t* items) {
  if (!p || !counts) return hdgmg::fail_plan(HDGMG_EINVAL, "null argument");
  if (t < 0 || t >= (int32_t)p->plan.chains.size()) return hdgmg::fail_plan(HDGMG_EINVAL, "level out of range");
  const auto& ch = p->plan.chains[t];
  int64_t n_items = 0;
  for (size_t c = 0; c < ch.size(); ++c) {
    if (info) {
      int32_t* r = info + 6 * c;
      r[0] = ch[c].s0; r[1] = ch[c].s1; r[2] = ch[c].start; r[3] = ch[c].end;
      r[4] = ch[c].closed ? 1 : 0; r[5] = (int32_t)n_items;
    }
    if (items)
      for (size_t i = 0; i < ch[c].edges.size(); ++i) {
        items[2 * (n_items + i)] = ch[c].edges[i];
        items[2 * (n_items + i) + 1] = ch[c].edirs[i];
      }
    n_items += (int64_t)ch[c].edges.size();
  }
  counts[0] = (int64_t)ch.size();
  counts[1] = n_items;
  return HDGMG_OK;
}

}  // extern "C"
