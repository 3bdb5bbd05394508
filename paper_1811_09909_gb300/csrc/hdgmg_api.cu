// C ABI of the hdgmg library: context, set-up, V-cycle, outer Krylov
// iteration, recovery (arXiv:1811.09909, Sec. 2-3; see include/hdgmg.h).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "internal.h"

using namespace hdgmg;

#include <atomic>
#include <mutex>

namespace hdgmg {
static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace hdgmg

namespace {
thread_local std::string g_last_error;

hdgmg_status fail(hdgmg_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}
}  // namespace

namespace hdgmg {
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace hdgmg

namespace {

#define CUDA_TRY(call)                                                                    \
  do {                                                                                    \
    cudaError_t err__ = (call);                                                           \
    if (err__ != cudaSuccess)                                                             \
      return fail(err__ == cudaErrorMemoryAllocation ? HDGMG_ENOMEM : HDGMG_ECUDA,        \
                  std::string(#call) + ": " + cudaGetErrorString(err__));                 \
  } while (0)

#define STATUS_TRY(call)                  \
  do {                                    \
    hdgmg_status st__ = (call);           \
    if (st__ != HDGMG_OK) return st__;    \
  } while (0)
}  // namespace

constexpr int kMaxRhsBlock = 16;

struct hdgmg_ctx {
  hdgmg_problem prob{};
  hdgmg_opts opts{};
  bool ns = false;             // non-symmetric operators (full storage): convection-diffusion,
                               // NIPG-H, IIPG-H
  double ktau = 0.0;           // the element-independent tau the element kernels add (a
                               // kappa-proportional tau is folded into the tables)
  cudaStream_t stream = nullptr;
  double hx = 0, hy = 0, hmin = 0;
  int p = 0, n = 0, nv = 0, nt = 0;
  RefElement ref;
  RefDevice refd{};
  CdTables cd{};               // convection-diffusion tables (ns only)
  std::vector<double> cdS0, cdW0, cdV0, cdad;   // host copies of the cd tables
  PencilDevice pb{};           // non-symmetric pencil basis (ns), rebuilt when eps0 moves
  EigBasisNS pb_host;          // its host copy (accuracy checks)
  bool pb_valid = false;
  bool cd_basis = false;       // ns: this set-up condenses through pb (else local LU)
  std::vector<void*> allocs;
  std::vector<Level> levels;
  double* logk = nullptr;
  double* kap = nullptr;       // exp(log kappa) per element
  bool basis = false;          // symmetric S condensed through the shared eigenbasis
  bool l2_window = false;      // an L2 persistence window was set on cap_stream
  double* Lfac = nullptr;      // factors of S when not: LU (full, ns) or Cholesky (packed)
  int* err = nullptr;
  int* err_h = nullptr;
  // coarsest level
  int* freeidx = nullptr;
  int* fedge = nullptr;
  int nf = 0;
  double* dense = nullptr;     // coarsest operator, then its Cholesky factor
  double* clinv = nullptr;     // L^-1
  double* cinv = nullptr;      // A_1^-1
  // outer Krylov vectors (finest level, FP64)
  double *x = nullptr, *r = nullptr, *z = nullptr, *pv = nullptr, *Ap = nullptr, *b = nullptr;
  double *lam = nullptr, *partial = nullptr, *scal = nullptr, *scal_h = nullptr;
  unsigned* counter = nullptr;   // last-block counter of the fused reductions
  // flexible GMRES (allocated on first use): V [(m+1)][len], Z [m][len]
  double *gmV = nullptr, *gmZ = nullptr, *gmH = nullptr, *gmcs = nullptr, *gmsn = nullptr;
  double *gmg = nullptr, *gmh = nullptr, *gmpart = nullptr, *gmtol = nullptr, *gmh_host = nullptr;
  int* gmj = nullptr;
  int* gmtot = nullptr;
  cudaGraph_t gm_graph = nullptr;
  cudaGraphExec_t gm_exec = nullptr;
  long long gm_body_launches = 0;
  // adjoint buffers (allocated on first use)
  double *adj_f = nullptr, *adj_lam = nullptr, *adj_u = nullptr;
  double *fwd_lam = nullptr, *fwd_u = nullptr, *mis_d = nullptr, *mis_g = nullptr;
  // host-call staging
  double *st_f = nullptr, *st_g = nullptr, *st_l = nullptr, *st_u = nullptr, *st_q = nullptr;
  bool setup_done = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, evk0 = nullptr, evk1 = nullptr;
  double t_setup_ms = 0.0, t_condense_ms = 0.0;
  int condense_threads = 0;    // autotuned launch shape of the condensation kernel (TPE * 16 + EPB)
  // PCG loop as one CUDA graph with a device-evaluated while condition
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t cg_graph = nullptr;
  cudaGraphExec_t cg_exec = nullptr;
  int* it_dev = nullptr;
  int* it_h = nullptr;
  double* init_h = nullptr;
  long long cg_body_launches = 0;
  long long launches_setup = 0, launches_solve = 0, capture_launches = 0;
  // P1 tail of the hierarchy run by the fused single-block V-cycle kernel
  int tail_start = -1;
  // mixed form: inner FP32 PCG (vectors xs, ps, Aps; r and z are level 0's)
  float *xs = nullptr, *ps = nullptr, *Aps = nullptr;
  double* scal32 = nullptr;
  cudaGraph_t cg32_graph = nullptr;
  cudaGraphExec_t cg32_exec = nullptr;
  long long cg32_body_launches = 0;
  int refinements = 0;
  TailParams<float> tp32;
  TailParams<double> tp64;
  // P1 tail run by one thread-block cluster (preferred when available)
  int ctail_start = -1;
  CTailParams<float> cp32;
  CTailParams<double> cp64;
  // persistent P1 cycle: the levels from pc_start down run as one cooperative
  // launch of pc_blocks blocks; pc_bar[0] is its grid barrier's arrival count
  // (pc_bar[1] that of the blocked form, which launches pc_blocks_b blocks:
  // each count stays a multiple of its own grid size between launches),
  // err[2] its expired-wait flag
  int pc_start = -1;
  int pc_blocks = 0;
  unsigned long long* pc_bar = nullptr;
  PCycleParams<float> pc32;
  PCycleParams<double> pc64;
  // step trace of the persistent cycle (hdgmg_trace_vcycle): device buffer of
  // pc_trace_cap (time, tag) pairs, armed for one call only
  unsigned long long* pc_trace = nullptr;
  int pc_trace_cap = 0;
  bool pc_trace_armed = false;
  // fused PCG body: the finest level's last post-smoothing step also forms the
  // PCG's r.z (rz_fuse set while the body is recorded; rz_done: it was)
  bool rz_fuse = false, rz_done = false;
  // opts.matrix_free: the FP32 tables of the matrix-free finest-level apply
  // (laid out as MfTables<p + 1>)
  std::vector<float> mf_tab;
  // blocked solves of up to kb right-hand sides (opts.rhs_block): FP32 level
  // vectors hold kb copies [kb][...]; kr is the count the V-cycle launches
  // run with (1 outside a blocked solve)
  int kb = 1, kr = 1;
  PCycleParams<float> pc32b;   // the persistent cycle for kr > 1 (no block-0 tail)
  int pc_blocks_b = 0;
  double *Xb = nullptr, *Rb = nullptr, *Bb = nullptr, *Lb = nullptr;   // FP64 [kb][len]
  double *scal64b = nullptr, *scal32b = nullptr, *partial_b = nullptr, *scal_hb = nullptr;
  unsigned* counter_b = nullptr;                                         // [kb + 1]
  cudaGraph_t cgb_graph[kMaxRhsBlock + 1] = {};
  cudaGraphExec_t cgb_exec[kMaxRhsBlock + 1] = {};
  long long cgb_body_launches[kMaxRhsBlock + 1] = {};

  template <typename T>
  cudaError_t alloc(T** p_, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, sizeof(T) * (count ? count : 1));
    if (e == cudaSuccess) {
      allocs.push_back(q);
      *p_ = (T*)q;
    }
    return e;
  }
  int64_t fine_len() const { return (int64_t)(p + 1) * 2 * n * (n + 1); }
};

namespace {

template <typename T> LevelData<T>& ld(Level& L);
template <> LevelData<double>& ld<double>(Level& L) { return L.d64; }
template <> LevelData<float>& ld<float>(Level& L) { return L.d32; }
template <typename T> CTailParams<T>& ctailp(hdgmg_ctx* c);
template <> CTailParams<double>& ctailp<double>(hdgmg_ctx* c) { return c->cp64; }
template <> CTailParams<float>& ctailp<float>(hdgmg_ctx* c) { return c->cp32; }
template <typename T> PCycleParams<T>& pcyclep(hdgmg_ctx* c);
template <> PCycleParams<double>& pcyclep<double>(hdgmg_ctx* c) { return c->pc64; }
template <> PCycleParams<float>& pcyclep<float>(hdgmg_ctx* c) { return c->pc32; }
template <typename T> PCycleParams<T>& pcycleb(hdgmg_ctx* c);
template <> PCycleParams<double>& pcycleb<double>(hdgmg_ctx* c) { return c->pc64; }   // FP64: unblocked
template <> PCycleParams<float>& pcycleb<float>(hdgmg_ctx* c) { return c->pc32b; }
template <typename T> TailParams<T>& tailp(hdgmg_ctx* c);
template <> TailParams<double>& tailp<double>(hdgmg_ctx* c) { return c->tp64; }
template <> TailParams<float>& tailp<float>(hdgmg_ctx* c) { return c->tp32; }

// Choose the fused tail: the longest run of P1 levels at the bottom of the
// hierarchy with n <= tail_n whose vectors and operators fit in shared memory.
template <typename T>
size_t tail_layout(hdgmg_ctx* c, int start, const std::vector<int>& staged, bool stage_inv,
                   TailParams<T>* P) {
  const int last = (int)c->levels.size() - 1;
  size_t off = 0;                                   // in T units
  auto take = [&](size_t count) {
    size_t o = off;
    off += (count + 3) / 4 * 4;                     // keep 16-byte alignment for floats
    return o;
  };
  for (int k = start; k <= last; ++k) {
    const Level& L = c->levels[k];
    TailLevel<T> t;
    t.n = L.n;
    t.m = L.m;
    t.nEdge = L.nEdge;
    t.voff = (int)take(6 * (size_t)L.nEdge);
    t.staged = (k < last && staged[k]) ? 1 : 0;
    if (t.staged) {
      const size_t nC = (size_t)L.nE / 4;
      const size_t na = c->ns ? 64 : 36;
      t.a_off = (int)take(na * (size_t)L.nE);
      t.dinv_off = (int)take((c->ns ? 4 : 3) * (size_t)L.nEdge);
      t.aii_off = (int)take(na * nC);
      t.y_off = (int)take(128 * nC);
      t.pi_off = (int)take(64 * nC);
      if (c->ns) t.rt_off = (int)take(64 * nC);
    }
    if (P) P->lv[k - start] = t;
  }
  size_t bytes = (off * sizeof(T) + 15) / 16 * 16;
  const size_t ainv_off = bytes;
  if (stage_inv) bytes += sizeof(double) * (size_t)c->nf * c->nf;
  const size_t w_off = bytes;
  bytes += sizeof(double) * (size_t)(c->nf + 2);
  if (P) {
    P->ainv_off = stage_inv ? (int)ainv_off : -1;
    P->w_off = (int)w_off;
    P->smem_bytes = (int)bytes;
  }
  return bytes;
}

// Choose the fused tail: P1 levels at the bottom of the hierarchy with
// n <= tail_n.  The level vectors always live in shared memory; the level
// operators are staged there too, from the coarsest level upwards, while they
// fit -- larger levels read them from L2.
template <typename T>
void plan_tail(hdgmg_ctx* c, int tail_n) {
  const int last = (int)c->levels.size() - 1;
  const size_t cap = (size_t)kTailMaxSmem;
  std::vector<int> staged(c->levels.size(), 0);
  const bool stage_inv = tail_layout<T>(c, last, staged, true, nullptr) <= cap;
  if (tail_layout<T>(c, last, staged, stage_inv, nullptr) > cap) {
    c->tail_start = -1;                      // coarsest level alone: standalone solve
    return;
  }
  int start = last;
  while (start - 1 >= 0) {
    const int k = start - 1;
    const Level& L = c->levels[k];
    // a finest level with a BF16 operator copy keeps its launched BF16 matvecs
    if (L.nd != 2 || L.transfer != 2 || L.n > tail_n || L.A16) break;
    if (last - k + 1 > kMaxTail) break;
    staged[k] = 1;
    if (tail_layout<T>(c, k, staged, stage_inv, nullptr) > cap) {
      staged[k] = 0;
      if (tail_layout<T>(c, k, staged, stage_inv, nullptr) > cap) break;
    }
    start = k;
  }
  c->tail_start = start;
  TailParams<T>& P = tailp<T>(c);
  P.nlev = last - start + 1;
  tail_layout<T>(c, start, staged, stage_inv, &P);
  for (int k = start; k <= last; ++k) {
    LevelData<T>& D = ld<T>(c->levels[k]);
    TailLevel<T>& t = P.lv[k - start];
    t.A = D.A;
    t.Dinv = D.Dinv;
    t.AIIinv = D.AIIinv;
    t.Y = D.Y;
    t.Pi = D.Pi;
    t.Rt = D.Rt;
  }
  P.r_in = ld<T>(c->levels[start]).r;
  P.e_out = ld<T>(c->levels[start]).e;
  P.Ainv = c->cinv;
  P.fidx = c->freeidx;
  P.fedge = c->fedge;
  P.nf = c->nf;
  P.omega = (T)c->opts.omega;
  P.lc = c->opts.local_corr;
  P.ns = c->ns ? 1 : 0;
}


// Cluster tail: the P1 levels with n <= top_n down to the coarsest, split
// over `cl` CTAs.  Vectors always live in distributed shared memory; level
// operators are staged from the coarsest level upwards while they fit.
template <typename T>
size_t ctail_layout(hdgmg_ctx* c, int start, int cl, const std::vector<int>& staged,
                    CTailParams<T>* P) {
  const int last = (int)c->levels.size() - 1;
  size_t off = 0;
  auto take = [&](size_t count) {
    size_t o = off;
    off += (count + 3) / 4 * 4;
    return o;
  };
  auto cdiv = [](int a, int b) { return (a + b - 1) / b; };
  for (int k = start; k <= last; ++k) {
    const Level& L = c->levels[k];
    CTailLevel<T> t;
    t.n = L.n;
    t.m = L.m;
    t.nEdge = L.nEdge;
    t.echunk = cdiv(L.nE, cl);
    t.edchunk = cdiv(L.nEdge, cl);
    t.cchunk = (k < last) ? cdiv(L.nE / 4, cl) : 1;
    t.off_v = (int)take(6 * (size_t)t.edchunk);
    if (k < last && staged[k]) {
      t.off_A = (int)take(36 * (size_t)t.echunk);
      t.off_D = (int)take(3 * (size_t)t.edchunk);
      t.off_AII = (int)take(36 * (size_t)t.cchunk);
      t.off_Y = (int)take(128 * (size_t)t.cchunk);
      t.off_Pi = (int)take(64 * (size_t)t.cchunk);
    }
    if (P) P->lv[k - start] = t;
  }
  size_t bytes = (off * sizeof(T) + 15) / 16 * 16;
  const size_t w_off = bytes;
  bytes += sizeof(double) * (size_t)(c->nf + 2);
  if (P) {
    P->w_off = (int)w_off;
    P->smem_bytes = (int)bytes;
  }
  return bytes;
}

template <typename T>
void plan_ctail(hdgmg_ctx* c, int top_n) {
  c->ctail_start = -1;
  const int last = (int)c->levels.size() - 1;
  if (last < 1) return;
  int start = last;
  while (start - 1 >= 0) {
    const Level& L = c->levels[start - 1];
    if (L.nd != 2 || L.transfer != 2 || L.n > top_n || L.A16 || last - (start - 1) + 1 > kMaxTail)
      break;
    --start;
  }
  if (start == last) return;                 // nothing above the coarsest level to fuse
  const size_t cap = (size_t)kTailMaxSmem;
  for (int cl : {16, 8}) {
    for (int s0 = start; s0 < last; ++s0) {
      std::vector<int> staged(c->levels.size(), 0);
      if (ctail_layout<T>(c, s0, cl, staged, nullptr) > cap) continue;
      for (int k = last - 1; k >= s0; --k) {
        staged[k] = 1;
        if (ctail_layout<T>(c, s0, cl, staged, nullptr) > cap) {
          staged[k] = 0;
          break;
        }
      }
      const size_t bytes = ctail_layout<T>(c, s0, cl, staged, nullptr);
      if (ctail_max_clusters<T>(cl, (int)bytes) < 1) break;   // try a smaller cluster
      CTailParams<T>& P = ctailp<T>(c);
      P = CTailParams<T>();
      P.nlev = last - s0 + 1;
      P.cl = cl;
      ctail_layout<T>(c, s0, cl, staged, &P);
      for (int k = s0; k <= last; ++k) {
        LevelData<T>& D = ld<T>(c->levels[k]);
        CTailLevel<T>& t = P.lv[k - s0];
        t.A = D.A;
        t.Dinv = D.Dinv;
        t.AIIinv = D.AIIinv;
        t.Y = D.Y;
        t.Pi = D.Pi;
      }
      P.r_in = ld<T>(c->levels[s0]).r;
      P.e_out = ld<T>(c->levels[s0]).e;
      P.Ainv = c->cinv;
      P.fidx = c->freeidx;
      P.fedge = c->fedge;
      P.nf = c->nf;
      P.omega = (T)c->opts.omega;
      P.lc = c->opts.local_corr;
      child_injection(P.Jc);
      c->ctail_start = s0;
      return;
    }
  }
}

// Persistent P1 cycle: from the first P1 level that the launched path runs by
// fused edge sweeps (below the p-level, or level 0 when p = 1) down to the
// coarsest.  The levels with n <= tail_n (and the coarsest) run on block 0:
// staged in its shared memory when they fit (operators, inverse, vectors),
// from L2 otherwise.  The grid is sized to the first level's edges (one item
// per thread), at most one block per SM; a tail from the first level is one
// block.
constexpr size_t kPcSmemBudget = 200 * 1024;

// shared-memory layout of levels [k, last] of the block-0 tail; returns bytes
template <typename T>
size_t pcycle_tail_layout(hdgmg_ctx* c, int ls, int k, PCycleParams<T>* P) {
  const int last = (int)c->levels.size() - 1;
  const size_t sz = sizeof(T);
  const size_t na = c->ns ? 64 : 36, nd2 = c->ns ? 4 : 3;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 15) / 16 * 16;
    return (int)o;
  };
  for (int l = k; l <= last; ++l) {
    const Level& L = c->levels[l];
    const size_t nE = L.nE, ned = L.nEdge, nC = nE / 4;
    PLevel<T> q;
    q.so_v = take(6 * ned * sz);
    if (l < last) {
      q.so_A = take(na * nE * sz);
      q.so_D = take(nd2 * ned * sz);
      q.so_AII = take(na * nC * sz);
      q.so_Y = take(128 * nC * sz);
      q.so_Pi = take(64 * nC * sz);
      q.so_Rt = c->ns ? take(64 * nC * sz) : q.so_Pi;
    }
    if (P) {
      PLevel<T>& d = P->lv[l - ls];
      d.so_v = q.so_v;
      d.so_A = q.so_A;
      d.so_D = q.so_D;
      d.so_AII = q.so_AII;
      d.so_Y = q.so_Y;
      d.so_Pi = q.so_Pi;
      d.so_Rt = q.so_Rt;
    }
  }
  const int so_Ainv = take(sizeof(double) * (size_t)c->nf * c->nf);
  const int so_w = take(sizeof(double) * (size_t)(c->nf > 0 ? c->nf : 1));
  if (P) {
    // bytes moved by the bulk copies: every operator array of the staged
    // levels and the coarsest inverse
    size_t tx = sizeof(double) * (size_t)c->nf * c->nf;
    for (int l = k; l < last; ++l) {
      const Level& L = c->levels[l];
      const size_t nE = L.nE, ned = L.nEdge, nC = nE / 4;
      tx += sz * (na * nE + nd2 * ned + na * nC + 128 * nC + 64 * nC + (c->ns ? 64 * nC : 0));
    }
    P->stage_bytes = (int)tx;
    P->so_Ainv = so_Ainv;
    P->so_w = so_w;
    P->smem_bytes = (int)off;
  }
  return off;
}

template <typename T>
void plan_pcycle(hdgmg_ctx* c) {
  c->pc_start = -1;
  const hdgmg_opts& o = c->opts;
  if (o.pcycle <= 0 || o.smoother != HDGMG_SMOOTH_BLOCK_JACOBI) return;
  // the FP64 cycle's steps are FP64-pipe bound and run faster as launched
  // kernels with more threads per SM (measured at 256^2, p = 4: 17.8 ms per
  // step launched, 18.9 persistent); pcycle = 2 forces the persistent form
  if (std::is_same<T, double>::value && o.pcycle < 2) return;
  const int last = (int)c->levels.size() - 1;
  int ls = -1;
  for (int l = 0; l < last; ++l) {
    const Level& L = c->levels[l];
    if (L.nd == 2 && L.transfer == 2 && !L.A16) {
      ls = l;
      break;
    }
  }
  if (ls < 0 || last - ls + 1 > kMaxPLev || c->nf > 4096) return;
  PCycleParams<T>& P = pcyclep<T>(c);
  P = PCycleParams<T>();
  P.nlev = last - ls + 1;
  P.tail = P.nlev;
  for (int k = ls; k <= last; ++k) {
    Level& L = c->levels[k];
    LevelData<T>& D = ld<T>(L);
    PLevel<T>& q = P.lv[k - ls];
    q.n = L.n;
    q.m = L.m;
    q.g = make_p1geom(L.n);
    q.A = D.A;
    q.Dinv = D.Dinv;
    q.AIIinv = D.AIIinv;
    q.Y = D.Y;
    q.Pi = D.Pi;
    q.Rt = c->ns ? D.Rt : D.Pi;
    q.r = D.r;
    q.e = D.e;
    q.y = D.y;
    if (P.tail == P.nlev && L.n <= o.pcycle_tail_n) P.tail = k - ls;
  }
  P.so_w = 0;
  P.smem_bytes = (int)(sizeof(double) * (size_t)(c->nf > 0 ? c->nf : 1));
  if (P.tail < P.nlev) {
    // stage the tail in shared memory from the highest level that fits
    for (int k = ls + P.tail; k <= last; ++k) {
      if (pcycle_tail_layout<T>(c, ls, k, nullptr) <= kPcSmemBudget) {
        P.tail = k - ls;
        P.staged = 1;
        pcycle_tail_layout<T>(c, ls, k, &P);
        break;
      }
    }
  }
  P.Ainv = c->cinv;
  P.fidx = c->freeidx;
  P.fedge = c->fedge;
  P.nf = c->nf;
  P.dco = make_fastdiv(c->levels[last].nEdge + c->nf);
  P.omega = (T)o.omega;
  P.lc = o.local_corr;
  P.ns = c->ns ? 1 : 0;
  P.bar = c->pc_bar;
  P.err = c->err + 2;
  const int maxb = pcycle_max_blocks<T>(P.smem_bytes);
  if (maxb < 1) return;
  const int nthr = pcycle_threads<T>();
  const int want = (c->levels[ls].nEdge + nthr - 1) / nthr;
  c->pc_blocks = P.tail == 0 ? 1 : (want < maxb ? want : maxb);
  if (std::is_same<T, float>::value && c->kb > 1) {
    // blocked solves: the same levels for up to kb right-hand sides, every
    // level on the whole grid (no block-0 tail: k vector sets do not fit in
    // one block's shared memory), shared memory for the k coarse right-hand sides
    PCycleParams<T>& B = pcycleb<T>(c);
    B = P;
    B.tail = B.nlev;
    B.staged = 0;
    B.bar = c->pc_bar + 1;   // its own count: the two launch different grid sizes
    B.so_w = 0;
    B.smem_bytes = (int)(sizeof(double) * (size_t)c->kb * (c->nf > 0 ? c->nf : 1));
    const int maxbb = pcycle_max_blocks<T>(B.smem_bytes);
    const int wantb = (c->kb * c->levels[ls].nEdge + nthr - 1) / nthr;
    c->pc_blocks_b = wantb < maxbb ? wantb : maxbb;
    if (c->pc_blocks_b < 1) return;
  }
  c->pc_start = ls;
}

// A bounded grid-barrier wait of the persistent cycle ran out on the device
// (err[2] set; its copy in err_h[2] must be current): reset the barrier and the
// flag so that the context stays usable, and report it.
hdgmg_status cycle_wait_status(hdgmg_ctx* c) {
  if (c->pc_start < 0 || c->err_h[2] == 0) return HDGMG_OK;
  c->err_h[2] = 0;
  CUDA_TRY(cudaMemsetAsync(c->pc_bar, 0, 2 * sizeof(unsigned long long), c->stream));
  CUDA_TRY(cudaMemsetAsync(c->err + 2, 0, sizeof(int), c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return fail(HDGMG_ETIMEOUT, "a grid-barrier wait of the persistent V-cycle ran out");
}

hdgmg_status check_launch(const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(HDGMG_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return HDGMG_OK;
}

// ----------------------------------------------------------- V-cycle (Alg. 1)
// y += A_l e on level l (the finest level reads its BF16 copy when it has one)
template <typename T>
void level_matvec(hdgmg_ctx* c, int l, const T* x, T* y, const T* xadd = nullptr) {
  Level& L = c->levels[l];
  if constexpr (std::is_same<T, float>::value) {
    if (L.A16) {
      launch_matvec_bf16(c->stream, L.n, L.nd, c->ns, L.A16, x, y, 1.0f, xadd, c->kr);
      return;
    }
    if (l == 0 && c->opts.matrix_free) {
      launch_matvec_mf(c->stream, L.n, L.nd, c->mf_tab.data(), c->kap, x, y, 1.0f, xadd, c->kr);
      return;
    }
  }
  launch_matvec<T>(c->stream, L.n, L.nd, c->ns, ld<T>(L).A, x, y, T(1), xadd, c->kr);
}

// A P1 level run by separate launches with the fused edge sweeps (not in a
// fused tail, not the coarsest level)
bool p1_launched(hdgmg_ctx* c, int l) {
  const Level& L = c->levels[l];
  return c->opts.smoother == HDGMG_SMOOTH_BLOCK_JACOBI && L.nd == 2 && L.transfer == 2 && !L.A16 &&
         l != c->tail_start && l != c->ctail_start;
}

// m smoothing steps of the point smoothers on level l (steps 2 and 6 of
// Algorithm 1); from_zero: e is taken as zero (pre-smoothing)
template <typename T>
void smooth_point(hdgmg_ctx* c, int l, bool from_zero) {
  cudaStream_t s = c->stream;
  Level& L = c->levels[l];
  LevelData<T>& D = ld<T>(L);
  const T omega = (T)c->opts.omega;
  switch (c->opts.smoother) {
    case HDGMG_SMOOTH_POINT_JACOBI: {
      int i = 0;
      if (from_zero) {
        launch_pj_update<T>(s, L.n, L.nd, D.Dpt, D.r, D.y, D.e, omega, 1);
        i = 1;
      }
      for (; i < L.m; ++i) {
        level_matvec<T>(c, l, D.e, D.y);
        launch_pj_update<T>(s, L.n, L.nd, D.Dpt, D.r, D.y, D.e, omega, 0);
      }
      break;
    }
    case HDGMG_SMOOTH_CHEBYSHEV:
      for (int k = 0; k < L.m; ++k) {
        if (k == 0 && from_zero) {
          launch_cheb_update<T>(s, L.n, L.nd, D.Dpt, D.r, D.y, D.e, D.cd, L.cheb, 0, 1, 1);
        } else {
          level_matvec<T>(c, l, D.e, D.y);
          launch_cheb_update<T>(s, L.n, L.nd, D.Dpt, D.r, D.y, D.e, D.cd, L.cheb, k, 0, k == 0);
        }
      }
      break;
    case HDGMG_SMOOTH_LU_SGS:
      if (from_zero) cudaMemsetAsync(D.e, 0, sizeof(T) * (size_t)L.nd * L.nEdge, s);
      for (int i = 0; i < L.m; ++i) {
        for (int col = 0; col < 4; ++col)
          launch_gs_colour<T>(s, L.n, L.nd, c->ns, ld<T>(L).A, D.Dpt, D.r, D.e, col, 0);
        for (int col = 3; col >= 0; --col)
          launch_gs_colour<T>(s, L.n, L.nd, c->ns, ld<T>(L).A, D.Dpt, D.r, D.e, col, 1);
      }
      break;
    default:
      break;
  }
}

// rp_r0/rp_y0/rp_nd0: the p-level above left its restriction J_N^T (r - A e)
// pending; this level's first sweep applies it.
template <typename T>
void vcycle(hdgmg_ctx* c, int l, const T* rp_r0 = nullptr, T* rp_y0 = nullptr, int rp_nd0 = 0) {
  cudaStream_t s = c->stream;
  Level& L = c->levels[l];
  LevelData<T>& D = ld<T>(L);
  const int last = (int)c->levels.size() - 1;
  if (l == c->pc_start) {                                   // persistent P1 cycle
    const bool blocked = std::is_same<T, float>::value && c->kr > 1;
    PCycleParams<T> P = blocked ? pcycleb<T>(c) : pcyclep<T>(c);
    P.rp_r0 = rp_r0;
    P.rp_y0 = rp_y0;
    P.rp_nd0 = rp_nd0;
    P.nrhs = c->kr;
    if (c->pc_trace_armed) {
      P.trace = c->pc_trace;
      P.trace_cap = c->pc_trace_cap;
    }
    launch_pcycle<T>(s, P, blocked ? c->pc_blocks_b : c->pc_blocks);
    return;
  }
  if (l == c->ctail_start) {                                // cluster-fused P1 tail
    launch_ctail<T>(s, ctailp<T>(c));
    return;
  }
  if (l == c->tail_start) {                                 // fused P1 tail + B_1 = A_1^-1
    launch_vcycle_tail<T>(s, tailp<T>(c));
    return;
  }
  if (l == last) {                                          // B_1 = A_1^-1
    launch_coarse_solve<T>(s, L.n, c->freeidx, c->fedge, c->nf, c->cinv, D.r, D.e, c->kr);
    return;
  }
  const T omega = (T)c->opts.omega;
  const int lc = c->opts.local_corr;
  const bool ns = c->ns;
  const int k = c->kr;
  if (p1_launched(c, l)) {
    // P1 level: fused edge-centric sweeps, ping-ponging between e and y.  The
    // first sweep (from e = 0) writes y; after the 2m - 1 sweeps of the level
    // the correction is back in e.
    Level& Lc = c->levels[l + 1];
    LevelData<T>& Dc = ld<T>(Lc);
    T* bufs[2] = {D.e, D.y};
    int cur = 1;
    if (rp_r0)
      launch_bj_first_restrict_p<T>(s, L.n, rp_nd0, ns, D.Dinv, rp_r0, rp_y0, D.r, bufs[1], omega, k);
    else
      launch_bj_update<T>(s, L.n, 2, ns, D.Dinv, D.r, bufs[0], bufs[1], omega, 1, nullptr, k);
    for (int i = 1; i < L.m; ++i) {
      launch_edge_p1<T>(s, L.n, ns, D.A, D.Dinv, D.r, bufs[cur], bufs[1 - cur], omega, true, k);
      cur ^= 1;
    }
    if (lc != HDGMG_LC_NONE)
      launch_local_correction<T>(s, L.n / 2, ns, D.AIIinv, D.Y, D.r, bufs[cur], k);
    launch_edge_p1<T>(s, L.n, ns, D.A, D.Dinv, D.r, bufs[cur], bufs[1 - cur], omega, false, k);
    launch_restrict_h<T>(s, Lc.n, D.Rt, D.r, bufs[1 - cur], Dc.r, k);
    vcycle<T>(c, l + 1);
    launch_prolong_h<T>(s, Lc.n, D.Pi, Dc.e, bufs[cur], bufs[1 - cur], k);
    if (lc == HDGMG_LC_BOTH)
      launch_local_correction<T>(s, L.n / 2, ns, D.AIIinv, D.Y, D.r, bufs[cur], k);
    for (int i = 0; i < L.m; ++i) {
      launch_edge_p1<T>(s, L.n, ns, D.A, D.Dinv, D.r, bufs[cur], bufs[1 - cur], omega, true, k);
      cur ^= 1;
    }
    return;                                    // cur == 0: the correction is in D.e
  }
  const bool bj = c->opts.smoother == HDGMG_SMOOTH_BLOCK_JACOBI;
  // step 2: pre-smoothing (the first sweep starts from e = 0)
  if (bj) {
    launch_bj_update<T>(s, L.n, L.nd, ns, D.Dinv, D.r, D.y, D.e, omega, 1, nullptr, k);
    for (int i = 1; i < L.m; ++i) {
      level_matvec<T>(c, l, D.e, D.y);
      launch_bj_update<T>(s, L.n, L.nd, ns, D.Dinv, D.r, D.y, D.e, omega, 0, nullptr, k);
    }
  } else {
    smooth_point<T>(c, l, true);
  }
  // step 3: local correction (interior edges of the next level's macro-elements)
  if (L.transfer == 2 && lc != HDGMG_LC_NONE)
    launch_local_correction<T>(s, L.n / 2, ns, D.AIIinv, D.Y, D.r, D.e, k);
  // step 4: coarse-grid correction
  Level& Lc = c->levels[l + 1];
  LevelData<T>& Dc = ld<T>(Lc);
  level_matvec<T>(c, l, D.e, D.y);
  // J_N^T and J_N fused into the neighbouring kernels when the P1 level
  // below runs as separate launches
  const bool fuse_p = L.transfer == 1 && p1_launched(c, l + 1);
  const T* xadd = nullptr;
  if (fuse_p) {
    vcycle<T>(c, l + 1, D.r, D.y, L.nd);
    xadd = Dc.e;
  } else {
    if (L.transfer == 1)
      launch_restrict_p<T>(s, L.n, L.nd, D.r, D.y, Dc.r);
    else
      launch_restrict_h<T>(s, Lc.n, D.Rt, D.r, D.y, Dc.r, k);
    vcycle<T>(c, l + 1);
    if (L.transfer == 1)
      launch_prolong_p<T>(s, L.n, L.nd, Dc.e, D.e);
    else
      launch_prolong_h<T>(s, Lc.n, D.Pi, Dc.e, D.e, D.y, k);
  }
  // step 5: second local correction (symmetric cycle)
  if (L.transfer == 2 && lc == HDGMG_LC_BOTH)
    launch_local_correction<T>(s, L.n / 2, ns, D.AIIinv, D.Y, D.r, D.e, k);
  // step 6: post-smoothing (the first step also adds the pending J_N e_c)
  if (!bj) {
    smooth_point<T>(c, l, false);
    return;
  }
  for (int i = 0; i < L.m; ++i) {
    level_matvec<T>(c, l, D.e, D.y, i == 0 ? xadd : nullptr);
    if constexpr (std::is_same<T, float>::value) {
      // the PCG's r.z joins the last step of the finest level (cg_body64_fused)
      if (l == 0 && i + 1 == L.m && c->rz_fuse && k == 1 && !ns) {
        launch_bj_update_dot(s, L.n, L.nd, D.Dinv, D.r, D.y, D.e, omega, i == 0 ? xadd : nullptr,
                             c->r, c->scal, c->partial, c->counter);
        c->rz_done = true;
        continue;
      }
    }
    launch_bj_update<T>(s, L.n, L.nd, ns, D.Dinv, D.r, D.y, D.e, omega, 0, i == 0 ? xadd : nullptr,
                        k);
  }
}

// z = B_N r on FP64 fine vectors
void apply_B(hdgmg_ctx* c, const double* r, double* z) {
  cudaStream_t s = c->stream;
  Level& L0 = c->levels[0];
  const int64_t len = c->fine_len();
  if (c->opts.precision != HDGMG_PREC_FP64) {
    launch_convert<double, float>(s, len, r, L0.d32.r);
    vcycle<float>(c, 0);
    launch_convert<float, double>(s, len, L0.d32.e, z);
  } else {
    cudaMemcpyAsync(L0.d64.r, r, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
    vcycle<double>(c, 0);
    cudaMemcpyAsync(z, L0.d64.e, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
  }
}

// y = A_fine x (FP64, interior rows), y overwritten
void apply_A64(hdgmg_ctx* c, const double* x, double* y) {
  cudaMemsetAsync(y, 0, sizeof(double) * c->fine_len(), c->stream);
  launch_matvec<double>(c->stream, c->n, c->p + 1, c->ns, c->levels[0].d64.A, x, y, 1.0);
}

double dot_sync(hdgmg_ctx* c, const double* a, const double* b) {
  launch_dot(c->stream, c->fine_len(), a, b, c->partial, c->scal + 5);
  cudaMemcpyAsync(c->scal_h + 5, c->scal + 5, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  cudaStreamSynchronize(c->stream);
  return c->scal_h[5];
}

template <typename T>
hdgmg_status alloc_level(hdgmg_ctx* c, Level& L, bool vec_only_fine) {
  LevelData<T>& D = ld<T>(L);
  (void)vec_only_fine;
  const size_t nblk_ent = c->ns ? (size_t)L.nd * L.nd : (size_t)(L.nd * (L.nd + 1) / 2);
  CUDA_TRY(c->alloc(&D.A, (size_t)L.nsym * L.nE));
  CUDA_TRY(c->alloc(&D.Dinv, nblk_ent * L.nEdge));
  // blocked solves run the FP32 cycle on kb right-hand sides at once
  const size_t nvec = (size_t)L.nd * L.nEdge * (std::is_same<T, float>::value ? c->kb : 1);
  CUDA_TRY(c->alloc(&D.r, nvec));
  CUDA_TRY(c->alloc(&D.e, nvec));
  CUDA_TRY(c->alloc(&D.y, nvec));
  CUDA_TRY(cudaMemset(D.y, 0, sizeof(T) * nvec));
  CUDA_TRY(cudaMemset(D.r, 0, sizeof(T) * nvec));
  CUDA_TRY(cudaMemset(D.e, 0, sizeof(T) * nvec));
  if (c->opts.smoother != HDGMG_SMOOTH_BLOCK_JACOBI && L.transfer != 0) {
    CUDA_TRY(c->alloc(&D.Dpt, (size_t)L.nd * L.nEdge));
    if (c->opts.smoother == HDGMG_SMOOTH_CHEBYSHEV) {
      CUDA_TRY(c->alloc(&D.cd, (size_t)L.nd * L.nEdge));
      CUDA_TRY(cudaMemset(D.cd, 0, sizeof(T) * (size_t)L.nd * L.nEdge));
      if (!L.cheb) CUDA_TRY(c->alloc(&L.cheb, 2 * (size_t)L.m));
    }
  }
  if (L.transfer == 2) {
    const size_t nC = (size_t)L.nE / 4;
    CUDA_TRY(c->alloc(&D.AIIinv, (c->ns ? 64 : 36) * nC));
    CUDA_TRY(c->alloc(&D.Y, 128 * nC));
    CUDA_TRY(c->alloc(&D.Pi, 64 * nC));
    if (c->ns)
      CUDA_TRY(c->alloc(&D.Rt, 64 * nC));
    else
      D.Rt = D.Pi;                     // Q_{k-1} = I_k^T for symmetric A
  }
  return HDGMG_OK;
}

// Point smoothers: 1 / A_aa on every non-coarsest level; for Chebyshev also
// Lambda_max of D^-1 A by 30 power iterations (from the deterministic start
// vector, on the level's own vectors) and the step coefficients
//   theta = (L + L/30)/2, delta = (L - L/30)/2, sigma = theta/delta,
//   k = 0: d = D^-1 res / theta;  k >= 1: rho_k = 1/(2 sigma - rho_{k-1}),
//   d = rho_k rho_{k-1} d + (2 rho_k / delta) D^-1 res,   rho_0 = 1/sigma.
constexpr int kPowerIters = 30;

template <typename T>
hdgmg_status setup_point_smoother(hdgmg_ctx* c) {
  cudaStream_t s = c->stream;
  const int nl = (int)c->levels.size();
  for (int l = 0; l + 1 < nl; ++l) {
    Level& L = c->levels[l];
    LevelData<T>& D = ld<T>(L);
    launch_point_diag<T>(s, L.n, L.nd, c->ns, D.A, D.Dpt);
    if (c->opts.smoother != HDGMG_SMOOTH_CHEBYSHEV) continue;
    const int64_t len = (int64_t)L.nd * L.nEdge;
    launch_power_start<T>(s, L.n, L.nd, D.e);
    for (int it = 0; it < kPowerIters; ++it) {
      CUDA_TRY(cudaMemsetAsync(D.y, 0, sizeof(T) * len, s));
      launch_matvec<T>(s, L.n, L.nd, c->ns, D.A, D.e, D.y, T(1));
      launch_scale_by<T>(s, len, D.Dpt, D.y);
      launch_dot<T>(s, len, D.y, D.y, c->partial, c->scal + 7);
      launch_normalize<T>(s, len, D.y, c->scal + 7, D.e);
    }
    CUDA_TRY(cudaMemsetAsync(D.y, 0, sizeof(T) * len, s));
    CUDA_TRY(cudaMemcpyAsync(c->scal_h + 7, c->scal + 7, sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    L.lmax = std::sqrt(c->scal_h[7]);
    const double lmin = L.lmax / 30.0;
    const double theta = 0.5 * (L.lmax + lmin), delta = 0.5 * (L.lmax - lmin);
    const double sigma = theta / delta;
    std::vector<double> coef(2 * (size_t)L.m, 0.0);
    double rho = 1.0 / sigma;
    coef[1] = 1.0 / theta;
    for (int k = 1; k < L.m; ++k) {
      const double rn = 1.0 / (2.0 * sigma - rho);
      coef[2 * k] = rn * rho;
      coef[2 * k + 1] = 2.0 * rn / delta;
      rho = rn;
    }
    CUDA_TRY(cudaMemcpy(L.cheb, coef.data(), sizeof(double) * coef.size(), cudaMemcpyHostToDevice));
  }
  return check_launch("point smoother set-up");
}

template <typename T>
hdgmg_status setup_hierarchy(hdgmg_ctx* c) {
  cudaStream_t s = c->stream;
  const int nl = (int)c->levels.size();
  for (int l = 0; l + 1 < nl; ++l) {
    Level& L = c->levels[l];
    Level& Lc = c->levels[l + 1];
    LevelData<T>& D = ld<T>(L);
    LevelData<T>& Dc = ld<T>(Lc);
    launch_bj_blocks<T>(s, L.n, L.nd, c->ns, D.A, D.Dinv, c->err);
    if (L.transfer == 1)
      launch_pcoarsen<T>(s, L.nE, L.nd, c->ns, D.A, Dc.A);
    else
      launch_agglomerate<T>(s, Lc.n, c->ns, D.A, Dc.A, D.AIIinv, D.Y, D.Pi, D.Rt, c->err);
  }
  if (c->opts.smoother != HDGMG_SMOOTH_BLOCK_JACOBI)
    STATUS_TRY(setup_point_smoother<T>(c));
  Level& Lc = c->levels[nl - 1];
  if (!launch_coarse_setup_smem<T>(s, Lc.n, c->ns, ld<T>(Lc).A, c->freeidx, c->nf, c->cinv,
                                   c->err)) {
    launch_coarse_assemble<T>(s, Lc.n, c->ns, ld<T>(Lc).A, c->freeidx, c->nf, c->dense);
    if (c->ns) {
      launch_coarse_gj(s, c->nf, c->dense, c->cinv, c->err);
    } else {
      launch_coarse_factor(s, c->nf, c->dense, c->err);
      launch_coarse_inverse(s, c->nf, c->dense, c->clinv, c->cinv);
    }
  }
  return check_launch("hierarchy set-up");
}

hdgmg_status build_rhs(hdgmg_ctx* c, const double* f, const double* gD) {
  cudaStream_t s = c->stream;
  const int64_t len = c->fine_len();
  CUDA_TRY(cudaMemsetAsync(c->b, 0, sizeof(double) * len, s));
  if (c->ns)
    c->cd_basis ? launch_rhs_cdeig(s, c->refd, c->pb, c->p, c->n, c->kap, f, c->b)
                : launch_rhs_cd(s, c->refd, c->cd, c->p, c->n, c->kap, c->Lfac, f, c->b);
  else
    c->basis ? launch_rhs(s, c->refd, c->p, c->n, c->kap, c->ktau, f, c->b)
             : launch_rhs_factor(s, c->refd, c->p, c->n, c->kap, c->ktau, c->Lfac, f, c->b);
  launch_copy_boundary(s, c->n, c->p + 1, gD, c->lam);
  if (gD) {
    // the lift -A lambda_D formed in a zeroed buffer (two contributions per
    // entry, so their order cannot change the sum), then subtracted
    CUDA_TRY(cudaMemsetAsync(c->Ap, 0, sizeof(double) * len, s));
    launch_matvec<double>(s, c->n, c->p + 1, c->ns, c->levels[0].d64.A, c->lam, c->Ap, 1.0);
    launch_axpby(s, len, -1.0, c->Ap, 1.0, c->b);
  }
  return check_launch("condensed right-hand side");
}

// One PCG iteration (reordered so that the test closes the body):
//   z = B r; beta = (r.z)/rz; p = z + beta p; alpha = (r.z)/(p.Ap);
//   x += alpha p; r -= alpha Ap; test ||r||^2 <= tol^2 ||b||^2.
// FP64 form: A = the FP64 fine operator, B = the V-cycle.  FP32 form (inner
// iteration of the refinement): A = the FP32 copy, vectors FP32, scalars and
// dot products FP64; r and z are the V-cycle's own level-0 buffers.
// With the FP32 V-cycle the level-0 FP32 residual is written by the update
// kernel of the previous iteration (and once before the loop), and the
// V-cycle output is read in FP32 by the two kernels that consume z.
void cg_body64(hdgmg_ctx* c, cudaGraphConditionalHandle h) {
  cudaStream_t s = c->stream;
  const int64_t len = c->fine_len();
  Level& L0 = c->levels[0];
  const bool mixed = c->opts.precision != HDGMG_PREC_FP64;
  if (mixed) {
    vcycle<float>(c, 0);
    launch_dot_fused_mixed(s, len, c->r, L0.d32.e, c->partial, c->counter, c->scal, 1);
    launch_cg_direction_zero_mixed(s, len, c->scal, L0.d32.e, c->pv, c->Ap);
  } else {
    apply_B(c, c->r, c->z);
    launch_dot_fused<double>(s, len, c->r, c->z, c->partial, c->counter, c->scal, 1);
    launch_cg_direction_zero<double>(s, len, c->scal, c->z, c->pv, c->Ap);
  }
  launch_matvec<double>(s, c->n, c->p + 1, c->ns, L0.d64.A, c->pv, c->Ap, 1.0);
  launch_dot_fused<double>(s, len, c->pv, c->Ap, c->partial, c->counter, c->scal, 0);
  launch_cg_update_test<double>(s, len, c->scal, c->x, c->r, c->pv, c->Ap, c->partial, c->counter,
                                h, c->it_dev, c->opts.max_it, c->opts.rtol * c->opts.rtol,
                                mixed ? L0.d32.r : nullptr);
}

// The same iteration in three launches after the V-cycle (opts.pcg_fuse,
// symmetric operator): r.z and beta; then p+ = z + beta p, Ap = A p+ and
// alpha = (r.z)/(p+.Ap) in the matvec kernel (p+ formed where the elements
// gather it); then x, r, p and the test.  Ap is zero on entry (zeroed before
// the loop and by every update).
void cg_body64_fused(hdgmg_ctx* c, cudaGraphConditionalHandle h) {
  cudaStream_t s = c->stream;
  const int64_t len = c->fine_len();
  Level& L0 = c->levels[0];
  const bool mixed = c->opts.precision != HDGMG_PREC_FP64;
  const float* z32 = mixed ? L0.d32.e : nullptr;
  const double* z64 = mixed ? nullptr : c->z;
  if (mixed) {
    c->rz_fuse = true;
    c->rz_done = false;
    vcycle<float>(c, 0);
    c->rz_fuse = false;
    if (!c->rz_done) launch_dot_fused_mixed(s, len, c->r, z32, c->partial, c->counter, c->scal, 1);
  } else {
    apply_B(c, c->r, c->z);
    launch_dot_fused<double>(s, len, c->r, c->z, c->partial, c->counter, c->scal, 1);
  }
  launch_cg_matvec(s, c->n, c->p + 1, L0.d64.A, z32, z64, c->pv, c->Ap, c->scal, c->partial,
                   c->counter);
  launch_cg_update_dir_test(s, len, c->scal, c->x, c->r, c->pv, c->Ap, z32, z64, c->partial,
                            c->counter, h, c->it_dev, c->opts.max_it, c->opts.rtol * c->opts.rtol,
                            mixed ? L0.d32.r : nullptr);
}

bool pcg_fused(const hdgmg_ctx* c) { return c->opts.pcg_fuse && !c->ns; }

void cg_body32(hdgmg_ctx* c, cudaGraphConditionalHandle h) {
  cudaStream_t s = c->stream;
  const int64_t len = c->fine_len();
  Level& L0 = c->levels[0];
  float* rs = L0.d32.r;
  float* zs = L0.d32.e;
  vcycle<float>(c, 0);
  launch_dot_fused<float>(s, len, rs, zs, c->partial, c->counter, c->scal32, 1);
  launch_cg_direction_zero<float>(s, len, c->scal32, zs, c->ps, c->Aps);
  launch_matvec<float>(s, c->n, c->p + 1, c->ns, L0.d32.A, c->ps, c->Aps, 1.0f);
  launch_dot_fused<float>(s, len, c->ps, c->Aps, c->partial, c->counter, c->scal32, 0);
  launch_cg_update_test<float>(s, len, c->scal32, c->xs, rs, c->ps, c->Aps, c->partial, c->counter,
                               h, c->it_dev, c->opts.max_it,
                               c->opts.inner_rtol * c->opts.inner_rtol, nullptr);
}

// Keep the finest operator the V-cycle reads (twice per cycle) in L2 across the
// iterations of a Krylov loop: an access-policy window on the capture stream,
// which the captured kernel nodes inherit.  The set-aside for persisting lines
// is a limit of this process's context (capped by the device); hdgmg_destroy
// resets the persisting lines.
void set_l2_window(hdgmg_ctx* c) {
  if (c->opts.l2_persist_mb <= 0) return;
  int dev = 0, maxp = 0, maxw = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, dev);
  cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxAccessPolicyWindowSize, dev);
  if (maxp <= 0 || maxw <= 0) return;
  Level& L0 = c->levels[0];
  const size_t n = (size_t)L0.nsym * L0.nE;
  void* base;
  size_t bytes;
  if (L0.A16) {
    base = L0.A16;
    bytes = n * sizeof(__nv_bfloat16);
  } else if (c->opts.precision != HDGMG_PREC_FP64) {
    base = L0.d32.A;
    bytes = n * sizeof(float);
  } else {
    base = L0.d64.A;
    bytes = n * sizeof(double);
  }
  size_t lim = (size_t)c->opts.l2_persist_mb << 20;
  if (lim > (size_t)maxp) lim = (size_t)maxp;
  if (bytes > (size_t)maxw) bytes = (size_t)maxw;
  if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, lim) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  cudaStreamAttrValue v = {};
  v.accessPolicyWindow.base_ptr = base;
  v.accessPolicyWindow.num_bytes = bytes;
  v.accessPolicyWindow.hitRatio = lim >= bytes ? 1.0f : (float)((double)lim / (double)bytes);
  v.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
  v.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
  if (cudaStreamSetAttribute(c->cap_stream, cudaStreamAttributeAccessPolicyWindow, &v) == cudaSuccess)
    c->l2_window = true;
  else
    cudaGetLastError();
}

hdgmg_status build_loop_graph(hdgmg_ctx* c, void (*body)(hdgmg_ctx*, cudaGraphConditionalHandle),
                              cudaGraph_t* graph_out, cudaGraphExec_t* exec_out,
                              long long* body_launches) {
  if (*exec_out) return HDGMG_OK;
  if (!c->cap_stream) {
    CUDA_TRY(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    set_l2_window(c);
  }
  cudaGraph_t g = nullptr;
  CUDA_TRY(cudaGraphCreate(&g, 0));
  *graph_out = g;
  cudaGraphConditionalHandle h;
  CUDA_TRY(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  CUDA_TRY(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
  cudaGraph_t bodyg = np.conditional.phGraph_out[0];
  cudaStream_t saved = c->stream;
  c->stream = c->cap_stream;
  const long long l0 = launch_count();
  CUDA_TRY(cudaStreamBeginCaptureToGraph(c->cap_stream, bodyg, nullptr, nullptr, 0,
                                         cudaStreamCaptureModeRelaxed));
  body(c, h);
  cudaGraph_t captured = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(c->cap_stream, &captured);
  c->stream = saved;
  if (ce != cudaSuccess)
    return fail(HDGMG_ECUDA, std::string("capture of the PCG loop: ") + cudaGetErrorString(ce));
  *body_launches = launch_count() - l0;
  c->capture_launches += *body_launches;    // captured, not executed
  CUDA_TRY(cudaGraphInstantiate(exec_out, g, 0));
  return HDGMG_OK;
}

// FP64 outer iteration with the FP32 PCG as the inner solver (iterative
// refinement): r = b - A x in FP64, solve A d = r / ||r|| in FP32 to
// inner_rtol, x += ||r|| d.  Returns the number of inner iterations.
hdgmg_status refine_solve(hdgmg_ctx* c, double nb, int* iters, int* outer, double* rel,
                          bool* conv, bool* breakdown) {
  cudaStream_t s = c->stream;
  const int64_t len = c->fine_len();
  const hdgmg_opts& o = c->opts;
  STATUS_TRY(build_loop_graph(c, cg_body32, &c->cg32_graph, &c->cg32_exec, &c->cg32_body_launches));
  Level& L0 = c->levels[0];
  *iters = 0;
  *outer = 0;
  *conv = false;
  *breakdown = false;
  for (;;) {
    // r = b - A x with A x formed in a zeroed buffer (deterministic sum)
    CUDA_TRY(cudaMemsetAsync(c->Ap, 0, sizeof(double) * len, s));
    launch_matvec<double>(s, c->n, c->p + 1, c->ns, L0.d64.A, c->x, c->Ap, 1.0);
    CUDA_TRY(cudaMemcpyAsync(c->r, c->b, sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
    launch_axpby(s, len, -1.0, c->Ap, 1.0, c->r);
    launch_dot<double>(s, len, c->r, c->r, c->partial, c->scal + 7);
    CUDA_TRY(cudaMemcpyAsync(c->scal_h + 7, c->scal + 7, sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    const double rr = c->scal_h[7];
    *rel = std::sqrt(rr) / nb;
    if (!std::isfinite(rr)) { *breakdown = true; break; }
    if (*rel <= o.rtol) { *conv = true; break; }
    if (*iters >= o.max_it || !(rr > 0.0)) break;
    // inner FP32 PCG on the normalised residual
    launch_scale_to_f32(s, len, c->r, c->scal + 7, L0.d32.r);
    CUDA_TRY(cudaMemsetAsync(c->xs, 0, sizeof(float) * len, s));
    CUDA_TRY(cudaMemsetAsync(c->ps, 0, sizeof(float) * len, s));
    CUDA_TRY(cudaMemsetAsync(c->it_dev, 0, sizeof(int), s));
    c->init_h[2] = 1.0;
    c->init_h[3] = 1.0;
    CUDA_TRY(cudaMemcpyAsync(c->scal32 + 0, &c->init_h[2], sizeof(double), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c->scal32 + 6, &c->init_h[3], sizeof(double), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaGraphLaunch(c->cg32_exec, s));
    launch_add_f32(s, len, c->scal + 7, c->xs, c->x);
    CUDA_TRY(cudaMemcpyAsync(c->it_h, c->it_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    *iters += *c->it_h;
    c->launches_solve += c->cg32_body_launches * (*c->it_h);
    ++*outer;
  }
  return HDGMG_OK;
}

// ------------------------------------------- blocked right-hand sides
// One iteration of k = c->kr simultaneous FP32 PCGs (the inner solver of the
// blocked refinement): one V-cycle, FP32 matvec and vector pass serve every
// right-hand side, each with its own scalars (scal32b[8 j ...]); a right-hand
// side that has reached the inner tolerance is frozen; the loop stops when
// all have (cg_update_test_block).
void cg_body_block(hdgmg_ctx* c, cudaGraphConditionalHandle h) {
  cudaStream_t s = c->stream;
  const int64_t len = c->fine_len();
  const int k = c->kr;
  Level& L0 = c->levels[0];
  float* rs = L0.d32.r;
  float* zs = L0.d32.e;
  vcycle<float>(c, 0);
  launch_dot_fused<float>(s, len, rs, zs, c->partial_b, c->counter_b, c->scal32b, 1, k);
  launch_cg_direction_zero<float>(s, len, c->scal32b, zs, c->ps, c->Aps, k);
  launch_matvec<float>(s, c->n, c->p + 1, c->ns, L0.d32.A, c->ps, c->Aps, 1.0f, nullptr, k);
  launch_dot_fused<float>(s, len, c->ps, c->Aps, c->partial_b, c->counter_b, c->scal32b, 0, k);
  launch_cg_update_test_block<float>(s, len, k, c->scal32b, c->xs, rs, c->ps, c->Aps, c->partial_b,
                                     c->counter_b, h, c->it_dev, c->opts.max_it,
                                     c->opts.inner_rtol * c->opts.inner_rtol);
}

// FP64 iterative refinement around the blocked FP32 PCG for k right-hand
// sides (b_j in Bb, solutions accumulated in Xb): r_j = b_j - A x_j in FP64,
// stop when every ||r_j|| <= rtol ||b_j|| (or breakdown / max_it inner
// iterations), else solve A d_j = r_j / ||r_j|| in FP32 to inner_rtol for all
// j at once and x_j += ||r_j|| d_j.  rel[j]: final relative residuals.
hdgmg_status refine_solve_block(hdgmg_ctx* c, int k, const double* nb, int* iters, int* outer,
                                double* rel, bool* conv, bool* breakdown) {
  cudaStream_t s = c->stream;
  const int64_t len = c->fine_len();
  const hdgmg_opts& o = c->opts;
  Level& L0 = c->levels[0];
  if (!c->cgb_exec[k]) {
    const int saved = c->kr;
    c->kr = k;
    const hdgmg_status st = build_loop_graph(c, cg_body_block, &c->cgb_graph[k], &c->cgb_exec[k],
                                             &c->cgb_body_launches[k]);
    c->kr = saved;
    STATUS_TRY(st);
  }
  *iters = 0;
  *outer = 0;
  *conv = false;
  *breakdown = false;
  for (;;) {
    // R = B - A X with A X formed in the zeroed R (deterministic sums)
    CUDA_TRY(cudaMemsetAsync(c->Rb, 0, sizeof(double) * len * k, s));
    launch_matvec<double>(s, c->n, c->p + 1, c->ns, L0.d64.A, c->Xb, c->Rb, 1.0, nullptr, k);
    launch_axpby(s, len * k, 1.0, c->Bb, -1.0, c->Rb);
    launch_dot_fused<double>(s, len, c->Rb, c->Rb, c->partial_b, c->counter_b, c->scal64b, 2, k);
    CUDA_TRY(cudaMemcpyAsync(c->scal_hb, c->scal64b, sizeof(double) * 8 * k, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    bool all = true;
    for (int j = 0; j < k; ++j) {
      const double rr = c->scal_hb[8 * j + 5];
      rel[j] = nb[j] > 0.0 ? std::sqrt(rr) / nb[j] : 0.0;
      if (!std::isfinite(rr)) *breakdown = true;
      // a solved right-hand side (or a zero one) gets a zero inner right-hand side
      if (!(rel[j] > o.rtol)) c->scal_hb[8 * j + 5] = 0.0;
      else all = false;
    }
    if (*breakdown) break;
    if (all) {
      *conv = true;
      break;
    }
    if (*iters >= o.max_it) break;
    // inner blocked FP32 PCG on the normalised residuals
    CUDA_TRY(cudaMemcpyAsync(c->scal64b, c->scal_hb, sizeof(double) * 8 * k, cudaMemcpyHostToDevice, s));
    launch_scale_to_f32(s, len, c->Rb, c->scal64b + 5, L0.d32.r, k, 8);
    CUDA_TRY(cudaMemsetAsync(c->xs, 0, sizeof(float) * len * k, s));
    CUDA_TRY(cudaMemsetAsync(c->ps, 0, sizeof(float) * len * k, s));
    CUDA_TRY(cudaMemsetAsync(c->it_dev, 0, sizeof(int) * 2, s));
    // inner scalars in the second half of the staging buffer (the first half
    // may still be in flight to scal64b)
    double* q0 = c->scal_hb + 8 * c->kb;
    for (int j = 0; j < k; ++j) {
      double* q = q0 + 8 * j;              // rz = 1 (p = 0 makes beta irrelevant), ref norm^2 = 1
      const bool solved = c->scal_hb[8 * j + 5] == 0.0;
      for (int t = 0; t < 8; ++t) q[t] = 0.0;
      q[0] = 1.0;
      q[6] = 1.0;
      q[7] = solved ? 1.0 : 0.0;
    }
    CUDA_TRY(cudaMemcpyAsync(c->scal32b, q0, sizeof(double) * 8 * k, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaGraphLaunch(c->cgb_exec[k], s));
    launch_add_f32(s, len, c->scal64b + 5, c->xs, c->Xb, k, 8);
    CUDA_TRY(cudaMemcpyAsync(c->it_h, c->it_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    *iters += *c->it_h;
    c->launches_solve += c->cgb_body_launches[k] * (*c->it_h);
    ++*outer;
    STATUS_TRY(check_launch("blocked refinement"));
  }
  return HDGMG_OK;
}

// Solve k <= kb right-hand sides together: condensed right-hand sides one by
// one (into Bb, boundary traces into Lb), the blocked refinement, then
// lambda_j = boundary + x_j and the local recovery of each.
hdgmg_status solve_block(hdgmg_ctx* c, int k, const double* f, const double* gD, double* lam,
                         double* u, double* q, hdgmg_info* info) {
  cudaStream_t s = c->stream;
  const int64_t len = c->fine_len();
  const size_t nvE = (size_t)c->nv * c->n * c->n;
  double nb[kMaxRhsBlock], rel[kMaxRhsBlock];
  for (int j = 0; j < k; ++j) {
    STATUS_TRY(build_rhs(c, f + j * nvE, gD ? gD + j * len : nullptr));
    CUDA_TRY(cudaMemcpyAsync(c->Bb + j * len, c->b, sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c->Lb + j * len, c->lam, sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
  }
  launch_dot_fused<double>(s, len, c->Bb, c->Bb, c->partial_b, c->counter_b, c->scal64b, 2, k);
  CUDA_TRY(cudaMemcpyAsync(c->scal_hb, c->scal64b, sizeof(double) * 8 * k, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemsetAsync(c->Xb, 0, sizeof(double) * len * k, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  bool bad_b = false;
  for (int j = 0; j < k; ++j) {
    nb[j] = std::sqrt(c->scal_hb[8 * j + 5]);
    if (!std::isfinite(nb[j])) bad_b = true;
  }
  int it = 0, outer = 0;
  bool conv = true, breakdown = bad_b;
  if (!bad_b) STATUS_TRY(refine_solve_block(c, k, nb, &it, &outer, rel, &conv, &breakdown));
  double worst = 0.0;
  for (int j = 0; j < k; ++j) worst = rel[j] > worst || !(rel[j] == rel[j]) ? rel[j] : worst;
  for (int j = 0; j < k; ++j) {
    double* lj = lam + j * len;
    CUDA_TRY(cudaMemcpyAsync(lj, c->Lb + j * len, sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
    launch_axpby(s, len, 1.0, c->Xb + j * len, 1.0, lj);
    double* uj = u ? u + j * nvE : nullptr;
    double* qj = q ? q + 2 * j * nvE : nullptr;
    if (uj || qj)
      c->basis ? launch_recover(s, c->refd, c->p, c->n, c->kap, c->ktau, f + j * nvE, lj, uj, qj)
               : launch_recover_factor(s, c->refd, c->p, c->n, c->kap, c->ktau, c->Lfac, f + j * nvE,
                                       lj, uj, qj);
  }
  STATUS_TRY(check_launch("blocked solve"));
  if (c->pc_start >= 0)
    CUDA_TRY(cudaMemcpyAsync(c->err_h + 2, c->err + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  STATUS_TRY(cycle_wait_status(c));
  c->refinements = outer;
  if (info) {
    info->iters = it;
    info->converged = conv ? 1 : 0;
    info->rel_res = worst;
    info->refinements = outer;
  }
  if (breakdown) return fail(HDGMG_EBREAKDOWN, "NaN/Inf in the blocked outer iteration");
  if (!conv) return fail(HDGMG_ENOCONV, "blocked refinement did not reach rtol");
  return HDGMG_OK;
}

// One Arnoldi step of right-preconditioned flexible GMRES (all on the
// device; the index j is read from device memory by every kernel).
void gm_body(hdgmg_ctx* c, cudaGraphConditionalHandle h) {
  cudaStream_t s = c->stream;
  const int64_t len = c->fine_len();
  const int m = c->opts.gmres_restart;
  launch_gm_select(s, len, c->gmV, c->gmj, 0, c->pv);          // v_j
  apply_B(c, c->pv, c->z);                                     // z_j = B v_j
  launch_gm_store(s, len, c->z, c->gmZ, c->gmj, 0);            // Z[j] = z_j
  apply_A64(c, c->z, c->Ap);                                   // w = A z_j
  launch_gm_orthogonalize(s, len, c->gmV, c->gmj, c->Ap, c->gmpart, m + 1, c->gmH, c->gmh, m + 1, 0);
  launch_gm_orthogonalize(s, len, c->gmV, c->gmj, c->Ap, c->gmpart, m + 1, c->gmH, c->gmh, m + 1, 1);
  launch_dot_fused<double>(s, len, c->Ap, c->Ap, c->partial, c->counter, c->scal, 2);
  launch_gm_normalize(s, len, c->Ap, c->scal + 5, c->gmV, c->gmj);
  launch_gm_givens(s, c->gmH, m + 1, c->gmcs, c->gmsn, c->gmg, c->gmj, m, c->gmtol, c->scal + 5, h,
                   c->gmtot, c->opts.max_it);
}

hdgmg_status gmres_buffers(hdgmg_ctx* c) {
  if (c->gmV) return HDGMG_OK;
  const int m = c->opts.gmres_restart;
  const int64_t len = c->fine_len();
  CUDA_TRY(c->alloc(&c->gmV, (size_t)(m + 1) * len));
  CUDA_TRY(c->alloc(&c->gmZ, (size_t)m * len));
  CUDA_TRY(c->alloc(&c->gmH, (size_t)(m + 1) * m));
  CUDA_TRY(c->alloc(&c->gmcs, (size_t)m));
  CUDA_TRY(c->alloc(&c->gmsn, (size_t)m));
  CUDA_TRY(c->alloc(&c->gmg, (size_t)m + 1));
  CUDA_TRY(c->alloc(&c->gmh, (size_t)m + 1));
  CUDA_TRY(c->alloc(&c->gmpart, (size_t)(m + 1) * gm_partial_blocks()));
  CUDA_TRY(c->alloc(&c->gmtol, 2));
  CUDA_TRY(c->alloc(&c->gmj, 2));
  CUDA_TRY(c->alloc(&c->gmtot, 2));
  CUDA_TRY(cudaMallocHost(&c->gmh_host, sizeof(double) * ((size_t)(m + 1) * m + 2 * (m + 1) + 8)));
  return HDGMG_OK;
}

// FGMRES(m) with the V-cycle as right preconditioner; restarts recompute the
// true FP64 residual.  Returns the total number of Arnoldi steps.
hdgmg_status gmres_solve(hdgmg_ctx* c, double nb, int* iters, double* rel, bool* conv,
                         bool* breakdown) {
  cudaStream_t s = c->stream;
  const int64_t len = c->fine_len();
  const hdgmg_opts& o = c->opts;
  const int m = o.gmres_restart;
  STATUS_TRY(gmres_buffers(c));
  STATUS_TRY(build_loop_graph(c, gm_body, &c->gm_graph, &c->gm_exec, &c->gm_body_launches));
  *iters = 0;
  *conv = false;
  *breakdown = false;
  CUDA_TRY(cudaMemsetAsync(c->gmtot, 0, sizeof(int), s));
  double* Hh = c->gmh_host;
  double* gh = Hh + (size_t)(m + 1) * m;
  double* yh = gh + (m + 1);
  int* jh = reinterpret_cast<int*>(yh + (m + 1));
  for (int cycle = 0; cycle < o.max_it; ++cycle) {
    // r = b - A x, its norm, v_0 = r / ||r||
    CUDA_TRY(cudaMemsetAsync(c->Ap, 0, sizeof(double) * len, s));
    launch_matvec<double>(s, c->n, c->p + 1, c->ns, c->levels[0].d64.A, c->x, c->Ap, 1.0);
    CUDA_TRY(cudaMemcpyAsync(c->r, c->b, sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
    launch_axpby(s, len, -1.0, c->Ap, 1.0, c->r);
    const double rr = dot_sync(c, c->r, c->r);
    *rel = std::sqrt(rr) / nb;
    if (!std::isfinite(rr)) { *breakdown = true; return HDGMG_OK; }
    if (*rel <= o.rtol) { *conv = true; return HDGMG_OK; }
    if (*iters >= o.max_it) return HDGMG_OK;
    const double beta = std::sqrt(rr);
    launch_axpby(s, len, 1.0 / beta, c->r, 0.0, c->gmV);
    CUDA_TRY(cudaMemsetAsync(c->gmH, 0, sizeof(double) * (size_t)(m + 1) * m, s));
    CUDA_TRY(cudaMemsetAsync(c->gmg, 0, sizeof(double) * (size_t)(m + 1), s));
    CUDA_TRY(cudaMemsetAsync(c->gmj, 0, sizeof(int), s));
    c->init_h[4] = beta;
    c->init_h[5] = o.rtol * nb;
    CUDA_TRY(cudaMemcpyAsync(c->gmg, &c->init_h[4], sizeof(double), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c->gmtol, &c->init_h[5], sizeof(double), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaGraphLaunch(c->gm_exec, s));
    CUDA_TRY(cudaMemcpyAsync(jh, c->gmj, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(Hh, c->gmH, sizeof(double) * (size_t)(m + 1) * m, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(gh, c->gmg, sizeof(double) * (size_t)(m + 1), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    const int j = *jh;
    *iters += j;
    c->launches_solve += c->gm_body_launches * j;
    // y = R^-1 g (upper triangular, column-major R = H[:, 0..j-1])
    for (int i = j - 1; i >= 0; --i) {
      double sacc = gh[i];
      for (int k = i + 1; k < j; ++k) sacc -= Hh[(size_t)k * (m + 1) + i] * yh[k];
      const double d = Hh[(size_t)i * (m + 1) + i];
      yh[i] = d != 0.0 ? sacc / d : 0.0;
    }
    CUDA_TRY(cudaMemcpyAsync(c->gmh, yh, sizeof(double) * (size_t)j, cudaMemcpyHostToDevice, s));
    launch_gm_update(s, len, c->gmZ, j, c->gmh, c->x);
    STATUS_TRY(check_launch("gmres update"));
  }
  return HDGMG_OK;
}

hdgmg_status solve_one(hdgmg_ctx* c, const double* f, const double* gD, double* lam_out,
                       double* u, double* q, hdgmg_info* info) {
  cudaStream_t s = c->stream;
  const int64_t len = c->fine_len();
  const hdgmg_opts& o = c->opts;
  c->refinements = 0;
  STATUS_TRY(build_rhs(c, f, gD));
  CUDA_TRY(cudaMemsetAsync(c->x, 0, sizeof(double) * len, s));
  const double bb = dot_sync(c, c->b, c->b);
  const double nb = std::sqrt(bb);
  int it = 0;
  double rel = 0.0;
  bool conv = true, breakdown = false;
  if (!(nb > 0.0)) {
    conv = true;
    if (!std::isfinite(bb)) breakdown = true;
  } else if (o.krylov == HDGMG_KRYLOV_GMRES) {
    STATUS_TRY(gmres_solve(c, nb, &it, &rel, &conv, &breakdown));
  } else if (o.krylov == HDGMG_KRYLOV_CG && o.precision == HDGMG_PREC_FP32_IR) {
    int outer = 0;
    STATUS_TRY(refine_solve(c, nb, &it, &outer, &rel, &conv, &breakdown));
    c->refinements = outer;
  } else if (o.krylov == HDGMG_KRYLOV_CG && o.pcg_graph == 0) {
    // the same PCG, each iteration's kernels launched from the host, which
    // reads the stop flag back after every iteration (for per-kernel
    // profiling: the kernels are not hidden inside a graph)
    CUDA_TRY(cudaMemcpyAsync(c->r, c->b, sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
    if (o.precision != HDGMG_PREC_FP64)
      launch_convert<double, float>(s, len, c->r, c->levels[0].d32.r);
    CUDA_TRY(cudaMemsetAsync(c->pv, 0, sizeof(double) * len, s));
    CUDA_TRY(cudaMemsetAsync(c->it_dev, 0, sizeof(int) * 2, s));
    c->init_h[0] = 1.0;
    c->init_h[1] = bb;
    CUDA_TRY(cudaMemcpyAsync(c->scal + 0, &c->init_h[0], sizeof(double), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c->scal + 6, &c->init_h[1], sizeof(double), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemsetAsync(c->Ap, 0, sizeof(double) * len, s));
    for (;;) {
      pcg_fused(c) ? cg_body64_fused(c, 0) : cg_body64(c, 0);
      STATUS_TRY(check_launch("PCG iteration"));
      CUDA_TRY(cudaMemcpyAsync(c->it_h, c->it_dev, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
      CUDA_TRY(cudaStreamSynchronize(s));
      if (c->it_h[1] || c->it_h[0] >= o.max_it) break;
    }
    CUDA_TRY(cudaMemcpyAsync(c->scal_h + 5, c->scal + 5, sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    it = *c->it_h;
    const double rr = c->scal_h[5];
    rel = std::sqrt(rr) / nb;
    breakdown = !std::isfinite(rr);
    conv = !breakdown && rel <= o.rtol;
  } else if (o.krylov == HDGMG_KRYLOV_CG) {
    // preconditioned CG with the V-cycle B_N (Sec. 3.6; symmetric cycle), the
    // whole iteration loop replayed as one CUDA graph
    STATUS_TRY(build_loop_graph(c, pcg_fused(c) ? cg_body64_fused : cg_body64, &c->cg_graph,
                                &c->cg_exec, &c->cg_body_launches));
    CUDA_TRY(cudaMemcpyAsync(c->r, c->b, sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
    if (o.precision != HDGMG_PREC_FP64)
      launch_convert<double, float>(s, len, c->r, c->levels[0].d32.r);
    CUDA_TRY(cudaMemsetAsync(c->pv, 0, sizeof(double) * len, s));
    CUDA_TRY(cudaMemsetAsync(c->Ap, 0, sizeof(double) * len, s));
    CUDA_TRY(cudaMemsetAsync(c->it_dev, 0, sizeof(int), s));
    c->init_h[0] = 1.0;      // rz of the previous iteration (p = 0 makes beta irrelevant)
    c->init_h[1] = bb;
    CUDA_TRY(cudaMemcpyAsync(c->scal + 0, &c->init_h[0], sizeof(double), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c->scal + 6, &c->init_h[1], sizeof(double), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaGraphLaunch(c->cg_exec, s));
    CUDA_TRY(cudaMemcpyAsync(c->it_h, c->it_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(c->scal_h + 5, c->scal + 5, sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    it = *c->it_h;
    c->launches_solve += c->cg_body_launches * it;
    const double rr = c->scal_h[5];
    rel = std::sqrt(rr) / nb;
    breakdown = !std::isfinite(rr);
    conv = !breakdown && rel <= o.rtol;
  } else {
    // multigrid as a fixed-point solver: x <- x + B_N (b - A x)  (Sec. 3.6)
    conv = false;
    for (it = 1; it <= o.max_it; ++it) {
      apply_A64(c, c->x, c->Ap);
      CUDA_TRY(cudaMemcpyAsync(c->r, c->b, sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
      launch_axpby(s, len, -1.0, c->Ap, 1.0, c->r);
      const double rr = dot_sync(c, c->r, c->r);
      rel = std::sqrt(rr) / nb;
      if (!std::isfinite(rr)) { breakdown = true; break; }
      if (rel > 1e8) break;
      if (rel <= o.rtol) { conv = true; break; }
      apply_B(c, c->r, c->z);
      launch_axpby(s, len, 1.0, c->z, 1.0, c->x);
    }
    // iterations = V-cycles applied before the converged check
    if (conv) it = it - 1;
    if (it > o.max_it) it = o.max_it;
  }
  // the persistent cycle's expired-wait flag is read back with the final
  // residual
  if (c->pc_start >= 0)
    CUDA_TRY(cudaMemcpyAsync(c->err_h + 2, c->err + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
  // true FP64 residual of the final iterate
  if (nb > 0.0) {
    apply_A64(c, c->x, c->Ap);
    CUDA_TRY(cudaMemcpyAsync(c->r, c->b, sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
    launch_axpby(s, len, -1.0, c->Ap, 1.0, c->r);
    rel = std::sqrt(dot_sync(c, c->r, c->r)) / nb;
    conv = conv && rel <= o.rtol * 10.0;
  } else if (c->pc_start >= 0) {
    CUDA_TRY(cudaStreamSynchronize(s));
  }
  STATUS_TRY(cycle_wait_status(c));
  // lambda = boundary data + interior solution
  CUDA_TRY(cudaMemcpyAsync(lam_out, c->lam, sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
  launch_axpby(s, len, 1.0, c->x, 1.0, lam_out);
  if ((u || q) && c->ns)
    c->cd_basis
        ? launch_recover_cdeig(s, c->refd, c->cd, c->pb, c->p, c->n, c->kap, f, lam_out, u, q)
        : launch_recover_cd(s, c->refd, c->cd, c->p, c->n, c->kap, c->Lfac, f, lam_out, u, q);
  else if (u || q)
    c->basis ? launch_recover(s, c->refd, c->p, c->n, c->kap, c->ktau, f, lam_out, u, q)
             : launch_recover_factor(s, c->refd, c->p, c->n, c->kap, c->ktau, c->Lfac, f, lam_out,
                                     u, q);
  STATUS_TRY(check_launch("solve"));
  if (info) {
    info->iters = it;
    info->converged = conv ? 1 : 0;
    info->rel_res = rel;
    info->refinements = c->refinements;
  }
  if (breakdown) return fail(HDGMG_EBREAKDOWN, "NaN/Inf in the outer iteration");
  if (!conv) return fail(HDGMG_ENOCONV, "outer iteration did not reach rtol");
  return HDGMG_OK;
}

}  // namespace

namespace {

hdgmg_status adjoint_buffers(hdgmg_ctx* c) {
  if (c->adj_f) return HDGMG_OK;
  const size_t nvE = (size_t)c->nv * c->n * c->n;
  const int64_t len = c->fine_len();
  CUDA_TRY(c->alloc(&c->adj_f, nvE));
  CUDA_TRY(c->alloc(&c->adj_lam, len));
  CUDA_TRY(c->alloc(&c->adj_u, nvE));
  CUDA_TRY(c->alloc(&c->fwd_lam, len));
  CUDA_TRY(c->alloc(&c->fwd_u, nvE));
  CUDA_TRY(c->alloc(&c->mis_d, nvE));
  CUDA_TRY(c->alloc(&c->mis_g, nvE));
  return HDGMG_OK;
}

// Adjoint of the solve for the sensitivity g_u = dL/du: one more solve of the
// (symmetric) trace system with right-hand side from g_u and homogeneous
// Dirichlet data, its local recovery, and the per-element contraction.
hdgmg_status adjoint_core(hdgmg_ctx* c, const double* lam, const double* u, const double* g_u,
                          double* dlogk, double* df, hdgmg_info* info) {
  cudaStream_t s = c->stream;
  const int nE = c->n * c->n;
  launch_adjoint_source(s, c->refd, c->nv, nE, g_u, c->adj_f);
  hdgmg_status st = solve_one(c, c->adj_f, nullptr, c->adj_lam, c->adj_u, nullptr, info);
  if (st != HDGMG_OK && st != HDGMG_ENOCONV) return st;
  launch_grad_contract(s, c->refd, c->p, c->n, c->kap, lam, u, c->adj_lam, c->adj_u, dlogk, df);
  STATUS_TRY(check_launch("adjoint contraction"));
  CUDA_TRY(cudaStreamSynchronize(s));
  return st;
}

}  // namespace

extern "C" {

void hdgmg_default_opts(hdgmg_opts* o) {
  if (!o) return;
  o->coarsest_n = 2;
  o->m_fine = 1;
  o->m_growth = 2;
  o->m_max = 0;
  o->local_corr = HDGMG_LC_BOTH;
  o->omega = 1.0;
  o->krylov = HDGMG_KRYLOV_CG;
  o->max_it = 200;
  o->rtol = 1e-10;
  o->precision = HDGMG_PREC_FP64;
  o->inner_rtol = 1e-5;
  o->cluster_tail_n = 0;
  o->gmres_restart = 30;
  o->smoother = HDGMG_SMOOTH_BLOCK_JACOBI;
  o->condensation = HDGMG_CONDENSE_AUTO;
  o->l2_persist_mb = 64;
  o->pcycle = 1;
  o->pcycle_tail_n = 16;
  o->pcg_graph = 1;
  o->rhs_block = 0;
  o->pcg_fuse = 1;
  o->matrix_free = 0;
}

const char* hdgmg_last_error(void) { return g_last_error.c_str(); }

void hdgmg_destroy(hdgmg_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->l2_window) cudaCtxResetPersistingL2Cache();   // demote this run's persisting lines
  for (void* p : c->allocs) cudaFree(p);
  if (c->err_h) cudaFreeHost(c->err_h);
  if (c->pc_trace) cudaFree(c->pc_trace);
  if (c->scal_h) cudaFreeHost(c->scal_h);
  if (c->init_h) cudaFreeHost(c->init_h);
  if (c->it_h) cudaFreeHost(c->it_h);
  if (c->cg_exec) cudaGraphExecDestroy(c->cg_exec);
  if (c->cg_graph) cudaGraphDestroy(c->cg_graph);
  if (c->cg32_exec) cudaGraphExecDestroy(c->cg32_exec);
  if (c->gm_exec) cudaGraphExecDestroy(c->gm_exec);
  if (c->gm_graph) cudaGraphDestroy(c->gm_graph);
  if (c->gmh_host) cudaFreeHost(c->gmh_host);
  if (c->scal_hb) cudaFreeHost(c->scal_hb);
  for (int k = 0; k <= kMaxRhsBlock; ++k) {
    if (c->cgb_exec[k]) cudaGraphExecDestroy(c->cgb_exec[k]);
    if (c->cgb_graph[k]) cudaGraphDestroy(c->cgb_graph[k]);
  }
  if (c->cg32_graph) cudaGraphDestroy(c->cg32_graph);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->evk0) cudaEventDestroy(c->evk0);
  if (c->evk1) cudaEventDestroy(c->evk1);
  delete c;
}

hdgmg_status hdgmg_create(hdgmg_ctx** out, const hdgmg_problem* prob, const hdgmg_opts* opts,
                          void* stream) {
  if (!out) return fail(HDGMG_EINVAL, "ctx pointer is NULL");
  *out = nullptr;
  if (!prob) return fail(HDGMG_EINVAL, "problem is NULL");
  hdgmg_opts o;
  if (opts)
    o = *opts;
  else
    hdgmg_default_opts(&o);
  const hdgmg_problem& P = *prob;
  if (P.p < 1 || P.p > 8) return fail(HDGMG_EINVAL, "p must be in 1..8");
  if (P.n < 2) return fail(HDGMG_EINVAL, "n must be >= 2");
  if (!(P.x1 > P.x0) || !(P.y1 > P.y0)) return fail(HDGMG_EINVAL, "empty domain");
  if (!(P.tau_c > 0.0)) return fail(HDGMG_EINVAL, "tau_c must be positive");
  if (P.tau_mode != HDGMG_TAU_CONST && P.tau_mode != HDGMG_TAU_OVER_H &&
      P.tau_mode != HDGMG_TAU_KAPPA_OVER_H)
    return fail(HDGMG_EINVAL, "unknown tau_mode");
  if (P.scheme < HDGMG_SCHEME_HDG || P.scheme > HDGMG_SCHEME_IIPG)
    return fail(HDGMG_EINVAL, "unknown scheme");
  if (P.scheme != HDGMG_SCHEME_HDG && P.pde != HDGMG_PDE_DIFFUSION)
    return fail(HDGMG_EINVAL, "the interior penalty schemes are for diffusion only");
  if (P.pde != HDGMG_PDE_DIFFUSION && P.pde != HDGMG_PDE_CONVDIFF)
    return fail(HDGMG_EINVAL, "unknown pde");
  if (P.pde == HDGMG_PDE_CONVDIFF && (!std::isfinite(P.beta_x) || !std::isfinite(P.beta_y)))
    return fail(HDGMG_EINVAL, "beta must be finite");
  if (o.coarsest_n < 2) return fail(HDGMG_EINVAL, "coarsest_n must be >= 2");
  if (o.m_fine < 1 || o.m_growth < 1 || o.m_max < 0) return fail(HDGMG_EINVAL, "bad smoothing schedule");
  if (o.local_corr < 0 || o.local_corr > 2) return fail(HDGMG_EINVAL, "unknown local_corr");
  if (o.krylov < 0 || o.krylov > 2) return fail(HDGMG_EINVAL, "unknown krylov");
  if (o.krylov == HDGMG_KRYLOV_GMRES && (o.gmres_restart < 1 || o.gmres_restart > 256))
    return fail(HDGMG_EINVAL, "gmres_restart must be in 1..256");
  if (o.precision < 0 || o.precision > 3) return fail(HDGMG_EINVAL, "unknown precision");
  if (o.smoother < 0 || o.smoother > 3) return fail(HDGMG_EINVAL, "unknown smoother");
  if (o.condensation < HDGMG_CONDENSE_AUTO || o.condensation > HDGMG_CONDENSE_FACTOR)
    return fail(HDGMG_EINVAL, "unknown condensation");
  if (o.l2_persist_mb < 0) return fail(HDGMG_EINVAL, "l2_persist_mb must be >= 0");
  if (o.rhs_block < 0 || o.rhs_block > kMaxRhsBlock)
    return fail(HDGMG_EINVAL, "rhs_block must be in 0..16");
  if (o.pcg_fuse < 0 || o.pcg_fuse > 1) return fail(HDGMG_EINVAL, "pcg_fuse must be 0 or 1");
  if (o.matrix_free < 0 || o.matrix_free > 1) return fail(HDGMG_EINVAL, "matrix_free must be 0 or 1");
  const bool nonsym = P.pde == HDGMG_PDE_CONVDIFF || P.scheme == HDGMG_SCHEME_NIPG ||
                      P.scheme == HDGMG_SCHEME_IIPG;
  if (nonsym && o.krylov == HDGMG_KRYLOV_CG)
    return fail(HDGMG_EINVAL,
                "krylov CG needs a symmetric operator; use GMRES for convection-diffusion, NIPG-H, IIPG-H");
  if (!(o.omega > 0.0) || !(o.rtol > 0.0) || o.max_it < 1) return fail(HDGMG_EINVAL, "bad omega/rtol/max_it");
  if (!(o.inner_rtol > 0.0) || !(o.inner_rtol < 1.0)) return fail(HDGMG_EINVAL, "inner_rtol must be in (0,1)");
  if (o.rhs_block > 1 &&
      (nonsym || o.krylov != HDGMG_KRYLOV_CG || o.smoother != HDGMG_SMOOTH_BLOCK_JACOBI ||
       (o.precision != HDGMG_PREC_FP32 && o.precision != HDGMG_PREC_FP32_IR)))
    return fail(HDGMG_EINVAL,
                "rhs_block > 1 needs a symmetric operator, krylov CG, block-Jacobi and the FP32 "
                "cycle (precision FP32 or FP32_IR)");
  int nn = P.n;
  while (nn > o.coarsest_n) {
    if (nn % 2) return fail(HDGMG_EINVAL, "n must halve evenly down to coarsest_n");
    nn /= 2;
  }
  if (nn < 2) return fail(HDGMG_EINVAL, "coarsest mesh would be smaller than 2 x 2");
  if ((int64_t)P.n * P.n > (1ll << 26)) return fail(HDGMG_EINVAL, "n too large");

  if (o.matrix_free &&
      (nonsym || o.condensation == HDGMG_CONDENSE_FACTOR || P.p + 1 > kMfMaxNd ||
       (o.precision != HDGMG_PREC_FP32 && o.precision != HDGMG_PREC_FP32_IR)))
    return fail(HDGMG_EINVAL, "matrix_free needs the symmetric basis condensation, p <= 6 and "
                              "precision FP32 or FP32_IR");
  hdgmg_ctx* c = new hdgmg_ctx();
  c->prob = P;
  c->opts = o;
  c->kb = o.rhs_block > 1 ? o.rhs_block : 1;
  c->ns = nonsym;
  c->basis = !nonsym && o.condensation != HDGMG_CONDENSE_FACTOR;
  c->stream = (cudaStream_t)stream;
  c->n = P.n;
  c->p = P.p;
  c->hx = (P.x1 - P.x0) / P.n;
  c->hy = (P.y1 - P.y0) / P.n;
  c->hmin = c->hx < c->hy ? c->hx : c->hy;
  c->ref = build_ref_element(P.p, c->hx, c->hy);
  if (P.scheme != HDGMG_SCHEME_HDG)
    make_ipdg_tables(c->ref, P.scheme == HDGMG_SCHEME_SIPG ? 1.0 : P.scheme == HDGMG_SCHEME_NIPG ? -1.0 : 0.0);
  if (P.tau_mode == HDGMG_TAU_KAPPA_OVER_H)
    fold_kappa_tau(c->ref, P.tau_c / c->hmin);
  else
    c->ktau = P.tau_mode == HDGMG_TAU_OVER_H ? P.tau_c / c->hmin : P.tau_c;
  c->nv = c->ref.nv;
  c->nt = c->ref.nt;
  auto cleanup = [&](hdgmg_status st) {
    hdgmg_destroy(c);
    return st;
  };
#define CTRY(call)                                                                       \
  do {                                                                                   \
    cudaError_t e__ = (call);                                                            \
    if (e__ != cudaSuccess)                                                              \
      return cleanup(fail(e__ == cudaErrorMemoryAllocation ? HDGMG_ENOMEM : HDGMG_ECUDA,  \
                          std::string(#call) + ": " + cudaGetErrorString(e__)));         \
  } while (0)
  // reference tables
  auto upload = [&](double** dst, const std::vector<double>& v) -> cudaError_t {
    cudaError_t e = c->alloc(dst, v.size());
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dst, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice);
  };
  CTRY(upload(&c->refd.M, c->ref.M));
  CTRY(upload(&c->refd.G, c->ref.G));
  CTRY(upload(&c->refd.E, c->ref.E));
  CTRY(upload(&c->refd.H, c->ref.H));
  CTRY(upload(&c->refd.F, c->ref.F));
  CTRY(upload(&c->refd.K, c->ref.K));
  CTRY(upload(&c->refd.BxT, c->ref.BxT));
  CTRY(upload(&c->refd.ByT, c->ref.ByT));
  CTRY(upload(&c->refd.Cx, c->ref.Cx));
  CTRY(upload(&c->refd.Cy, c->ref.Cy));
  CTRY(upload(&c->refd.Ef, c->ref.Ef));
  CTRY(upload(&c->refd.Hv, c->ref.Hv));
  if (c->basis) {
    // the basis that diagonalises every element's volume block
    EigBasis eb;
    if (!build_eig_basis(c->ref, c->ktau, c->hmin, eb))
      return cleanup(fail(HDGMG_EINVAL, "no positive-definite combination of the volume forms"));
    for (double& v : eb.e) v *= c->ktau;    // the kernels take tau e and tau Q
    for (double& v : eb.Q) v *= c->ktau;
    if (o.matrix_free) {
      const int nd = c->p + 1, nt = 4 * nd, nv = nd * nd;
      c->mf_tab.clear();
      for (double v : c->ref.K) c->mf_tab.push_back((float)v);
      for (double v : eb.P) c->mf_tab.push_back((float)v);
      for (double v : eb.Q) c->mf_tab.push_back((float)v);   // tau Q
      for (double v : eb.g) c->mf_tab.push_back((float)v);
      for (double v : eb.e) c->mf_tab.push_back((float)v);   // tau e
      c->mf_tab.push_back((float)c->ktau);
      if ((int)c->mf_tab.size() != mf_table_size(nd) || (int)c->ref.K.size() != nt * nt ||
          (int)eb.P.size() != nv * nt)
        return cleanup(fail(HDGMG_EINVAL, "matrix-free tables: unexpected basis sizes"));
    }
    CTRY(upload(&c->refd.Phi, eb.Phi));
    CTRY(upload(&c->refd.eg, eb.g));
    CTRY(upload(&c->refd.ee, eb.e));
    CTRY(upload(&c->refd.P, eb.P));
    CTRY(upload(&c->refd.Q, eb.Q));
  }
  if (c->ns) {
    std::vector<double> S0, W0, V0, ad;
    const bool conv = P.pde == HDGMG_PDE_CONVDIFF;
    build_cd_tables(c->ref, c->ktau, conv ? P.beta_x : 0.0, conv ? P.beta_y : 0.0, S0, W0, V0, ad);
    c->cdS0 = S0;
    c->cdW0 = W0;
    c->cdV0 = V0;
    c->cdad = ad;
    CTRY(upload(&c->cd.S0, S0));
    CTRY(upload(&c->cd.W0, W0));
    CTRY(upload(&c->cd.V0, V0));
    CTRY(upload(&c->cd.adiag, ad));
  }
  // levels
  {
    Level L;
    L.n = P.n;
    L.nd = P.p + 1;
    c->levels.push_back(L);
    if (P.p > 1) {
      Level Lp;
      Lp.n = P.n;
      Lp.nd = 2;
      c->levels.back().transfer = 1;
      c->levels.push_back(Lp);
    }
    while (c->levels.back().n > o.coarsest_n) {
      Level Lh;
      Lh.n = c->levels.back().n / 2;
      Lh.nd = 2;
      c->levels.back().transfer = 2;
      c->levels.push_back(Lh);
    }
    int m = o.m_fine;
    for (Level& Lv : c->levels) {
      Lv.nl = 4 * Lv.nd;
      Lv.nsym = c->ns ? Lv.nl * Lv.nl : Lv.nl * (Lv.nl + 1) / 2;
      Lv.nE = Lv.n * Lv.n;
      Lv.nEdge = 2 * Lv.n * (Lv.n + 1);
      Lv.m = m;
      m *= o.m_growth;
      if (o.m_max > 0 && m > o.m_max) m = o.m_max;
    }
  }
  const bool fp32 = o.precision != HDGMG_PREC_FP64;
  for (size_t l = 0; l < c->levels.size(); ++l) {
    Level& L = c->levels[l];
    hdgmg_status st;
    if (fp32) {
      st = alloc_level<float>(c, L, false);
      if (st == HDGMG_OK && l == 0) {
        if (c->alloc(&L.d64.A, (size_t)L.nsym * L.nE) != cudaSuccess) st = fail(HDGMG_ENOMEM, "A64");
        if (st == HDGMG_OK && o.precision == HDGMG_PREC_BF16 &&
            c->alloc(&L.A16, (size_t)L.nsym * L.nE) != cudaSuccess)
          st = fail(HDGMG_ENOMEM, "A16");
      }
    } else {
      st = alloc_level<double>(c, L, false);
    }
    if (st != HDGMG_OK) return cleanup(st);
  }
  const int64_t len = c->fine_len();
  CTRY(c->alloc(&c->logk, (size_t)P.n * P.n));
  CTRY(c->alloc(&c->kap, (size_t)P.n * P.n));
  if (!c->basis && !c->ns)
    CTRY(c->alloc(&c->Lfac, (size_t)c->nv * (c->nv + 1) / 2 * P.n * P.n));
  // ns: the LU factors (nv^2 doubles per element) are allocated by the first
  // set-up that needs them (the pencil basis, when accurate, needs none)
  CTRY(c->alloc(&c->err, 4));
  CTRY(cudaMallocHost(&c->err_h, sizeof(int) * 4));
  CTRY(c->alloc(&c->x, len));
  CTRY(c->alloc(&c->r, len));
  CTRY(c->alloc(&c->z, len));
  CTRY(c->alloc(&c->pv, len));
  CTRY(c->alloc(&c->Ap, len));
  CTRY(c->alloc(&c->b, len));
  CTRY(c->alloc(&c->lam, len));
  CTRY(c->alloc(&c->partial, kDotBlocks));
  CTRY(c->alloc(&c->counter, 4));
  CTRY(cudaMemset(c->counter, 0, sizeof(unsigned) * 4));
  CTRY(c->alloc(&c->scal, 8));
  CTRY(c->alloc(&c->scal32, 8));
  if (fp32) {
    CTRY(c->alloc(&c->xs, len * c->kb));
    CTRY(c->alloc(&c->ps, len * c->kb));
    CTRY(c->alloc(&c->Aps, len * c->kb));
  }
  if (c->kb > 1) {
    const size_t kb = (size_t)c->kb;
    CTRY(c->alloc(&c->Xb, len * kb));
    CTRY(c->alloc(&c->Rb, len * kb));
    CTRY(c->alloc(&c->Bb, len * kb));
    CTRY(c->alloc(&c->Lb, len * kb));
    CTRY(c->alloc(&c->scal64b, 8 * kb));
    CTRY(c->alloc(&c->scal32b, 8 * kb));
    CTRY(c->alloc(&c->partial_b, (size_t)kDotBlocks * kb));
    CTRY(c->alloc(&c->counter_b, kb + 1));
    CTRY(cudaMemset(c->counter_b, 0, sizeof(unsigned) * (kb + 1)));
    CTRY(cudaMallocHost(&c->scal_hb, sizeof(double) * 16 * kb));   // two halves: 64b, 32b
  }
  CTRY(cudaMallocHost(&c->scal_h, sizeof(double) * 8));
  CTRY(cudaMallocHost(&c->init_h, sizeof(double) * 8));
  CTRY(cudaMallocHost(&c->it_h, sizeof(int) * 2));
  CTRY(c->alloc(&c->it_dev, 2));
  // coarsest level: free-dof numbering of its interior edges
  {
    const Level& Lc = c->levels.back();
    std::vector<int> fidx(Lc.nEdge, -1);
    int nfe = 0;
    const int n = Lc.n, nvert = n * (n + 1);
    for (int e = 0; e < Lc.nEdge; ++e) {
      bool bnd;
      if (e < nvert) {
        const int i = e % (n + 1);
        bnd = (i == 0 || i == n);
      } else {
        const int j = (e - nvert) / n;
        bnd = (j == 0 || j == n);
      }
      if (!bnd) fidx[e] = nfe++;
    }
    c->nf = 2 * nfe;
    CTRY(c->alloc(&c->freeidx, fidx.size()));
    CTRY(cudaMemcpy(c->freeidx, fidx.data(), sizeof(int) * fidx.size(), cudaMemcpyHostToDevice));
    std::vector<int> fedge(nfe > 0 ? nfe : 1, 0);
    for (int e = 0; e < Lc.nEdge; ++e)
      if (fidx[e] >= 0) fedge[fidx[e]] = e;
    CTRY(c->alloc(&c->fedge, fedge.size()));
    CTRY(cudaMemcpy(c->fedge, fedge.data(), sizeof(int) * fedge.size(), cudaMemcpyHostToDevice));
    CTRY(c->alloc(&c->dense, (size_t)c->nf * c->nf));
    CTRY(c->alloc(&c->clinv, (size_t)c->nf * c->nf));
    CTRY(c->alloc(&c->cinv, (size_t)c->nf * c->nf));
  }
  // The cluster tail is opt-in: measured on GB300 (256^2, p = 4) its
  // distributed-shared-memory steps and cluster barriers cost more per step
  // than the single-block tail plus separate launches of the larger levels.
  const int ct = o.cluster_tail_n;
  // (the cluster tail exists for symmetric operators only)
  if (fp32) {
    plan_tail<float>(c, 32);
    if (ct > 0 && !c->ns) plan_ctail<float>(c, ct);
  } else {
    plan_tail<double>(c, 16);
    if (ct > 0 && !c->ns) plan_ctail<double>(c, ct);
  }
  if (c->ctail_start >= 0 && c->tail_start >= 0 && c->tail_start < c->ctail_start)
    c->ctail_start = -1;                     // keep whichever fuses more levels
  if (o.smoother != HDGMG_SMOOTH_BLOCK_JACOBI || c->kb > 1) {
    c->tail_start = -1;                      // the fused tails implement block-Jacobi only, and
    c->ctail_start = -1;                     // one right-hand side at a time
  }
  CTRY(c->alloc(&c->pc_bar, 2));
  CTRY(cudaMemset(c->pc_bar, 0, 2 * sizeof(unsigned long long)));
  if (fp32)
    plan_pcycle<float>(c);
  else
    plan_pcycle<double>(c);
  if (c->pc_start >= 0) {                    // the persistent cycle replaces both tails
    c->tail_start = -1;
    c->ctail_start = -1;
  }
  CTRY(cudaEventCreate(&c->ev0));
  CTRY(cudaEventCreate(&c->ev1));
  CTRY(cudaEventCreate(&c->evk0));
  CTRY(cudaEventCreate(&c->evk1));
  CTRY(cudaDeviceSynchronize());
#undef CTRY
  *out = c;
  return HDGMG_OK;
}

// Non-symmetric volume blocks: decide per set-up between the pencil basis
// and local LU.  eps0 = kappa's geometric mean rounded to a quarter power of
// two (so that repeated set-ups with similar kappa reuse the basis); the basis
// is used when A_e through it agrees with a direct dense solve to 1e-11 at the
// smallest and largest kappa of this set-up.
hdgmg_status prepare_pencil(hdgmg_ctx* c, const double* log_kappa) {
  c->cd_basis = false;
  if (c->opts.condensation == HDGMG_CONDENSE_FACTOR) return HDGMG_OK;
  const int nE = c->n * c->n;
  std::vector<double> lk(nE);
  CUDA_TRY(cudaMemcpyAsync(lk.data(), log_kappa, sizeof(double) * nE, cudaMemcpyDeviceToHost,
                           c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  double lo = lk[0], hi = lk[0], sum = 0.0;
  for (double v : lk) {
    if (!std::isfinite(v)) return HDGMG_OK;          // the LU path reports it
    lo = std::min(lo, v);
    hi = std::max(hi, v);
    sum += v;
  }
  const double l2 = sum / nE / std::log(2.0);
  const double eps0 = std::exp2(std::round(4.0 * l2) / 4.0);
  if (!c->pb_valid || c->pb.eps0 != eps0) {
    EigBasisNS E;
    c->pb_valid = false;
    if (build_eig_basis_ns(c->ref, c->cdS0, c->cdW0, c->cdV0, eps0, E)) {
      auto put = [&](double** dst, const std::vector<double>& v) -> cudaError_t {
        if (!*dst) {
          cudaError_t e = c->alloc(dst, v.size());
          if (e != cudaSuccess) return e;
        }
        return cudaMemcpy(*dst, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice);
      };
      CUDA_TRY(put(&c->pb.X, E.X));
      CUDA_TRY(put(&c->pb.R, E.R));
      CUDA_TRY(put(&c->pb.Pv1, E.Pv1));
      CUDA_TRY(put(&c->pb.Pv0, E.Pv0));
      CUDA_TRY(put(&c->pb.Pw1, E.Pw1));
      CUDA_TRY(put(&c->pb.Pw0, E.Pw0));
      CUDA_TRY(put(&c->pb.la, E.la));
      CUDA_TRY(put(&c->pb.lb, E.lb));
      if (!c->pb.kind) CUDA_TRY(c->alloc(&c->pb.kind, E.kind.size()));
      CUDA_TRY(cudaMemcpy(c->pb.kind, E.kind.data(), sizeof(int) * E.kind.size(),
                          cudaMemcpyHostToDevice));
      c->pb.eps0 = eps0;
      c->pb_valid = true;
      c->pb_host = E;
    }
  }
  if (c->pb_valid) {
    const double err = std::max(
        check_eig_basis_ns(c->ref, c->cdS0, c->cdW0, c->cdV0, c->cdad, c->pb_host, std::exp(lo)),
        check_eig_basis_ns(c->ref, c->cdS0, c->cdW0, c->cdV0, c->cdad, c->pb_host, std::exp(hi)));
    c->cd_basis = err <= 1e-11;
  }
  if (!c->cd_basis && c->opts.condensation == HDGMG_CONDENSE_BASIS)
    return fail(HDGMG_EINVAL, "condensation BASIS: the pencil basis is not accurate for this kappa");
  return HDGMG_OK;
}

hdgmg_status hdgmg_setup(hdgmg_ctx* c, const double* log_kappa) {
  if (!c || !log_kappa) return fail(HDGMG_EINVAL, "NULL argument");
  cudaStream_t s = c->stream;
  const int nE = c->n * c->n;
  const long long l0 = launch_count();
  CUDA_TRY(cudaEventRecord(c->ev0, s));
  CUDA_TRY(cudaMemcpyAsync(c->logk, log_kappa, sizeof(double) * nE, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemsetAsync(c->err, 0, sizeof(int) * 4, s));
  CUDA_TRY(cudaMemsetAsync(c->pc_bar, 0, 2 * sizeof(unsigned long long), s));
  Level& L0 = c->levels[0];
  if (c->ns) {
    STATUS_TRY(prepare_pencil(c, log_kappa));
    if (!c->cd_basis && !c->Lfac) CUDA_TRY(c->alloc(&c->Lfac, (size_t)c->nv * c->nv * nE));
  }
  launch_kappa(s, nE, c->logk, c->kap);
  // the first set-up of a (kernel, p) pair times the candidate block sizes
  // before the condensation proper (outside the timed condensation events)
  for (int pass = 0; pass < 2; ++pass) {
    const bool tune_only = pass == 0;
    if (!tune_only) CUDA_TRY(cudaEventRecord(c->evk0, s));
    if (c->ns)
      c->condense_threads =
          c->cd_basis ? launch_condense_cdeig(s, c->refd, c->cd, c->pb, c->p, nE, c->kap, L0.d64.A,
                                              c->err, tune_only)
                      : launch_condense_cd(s, c->refd, c->cd, c->p, nE, c->kap, L0.d64.A, c->Lfac,
                                           c->err, tune_only);
    else
      c->condense_threads =
          c->basis ? launch_condense(s, c->refd, c->p, nE, c->kap, c->ktau, L0.d64.A, c->err, tune_only)
                   : launch_condense_factor(s, c->refd, c->p, nE, c->kap, c->ktau, L0.d64.A, c->Lfac,
                                            c->err, tune_only);
  }
  CUDA_TRY(cudaEventRecord(c->evk1, s));
  STATUS_TRY(check_launch("condensation"));
  if (c->opts.precision != HDGMG_PREC_FP64) {
    launch_convert<double, float>(s, (int64_t)L0.nsym * L0.nE, L0.d64.A, L0.d32.A);
    if (L0.A16) launch_to_bf16(s, (int64_t)L0.nsym * L0.nE, L0.d64.A, L0.A16);
    STATUS_TRY(setup_hierarchy<float>(c));
  } else {
    STATUS_TRY(setup_hierarchy<double>(c));
  }
  CUDA_TRY(cudaEventRecord(c->ev1, s));
  CUDA_TRY(cudaMemcpyAsync(c->err_h, c->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  c->t_setup_ms = ms;
  cudaEventElapsedTime(&ms, c->evk0, c->evk1);
  c->t_condense_ms = ms;
  c->launches_setup = launch_count() - l0;
  if (c->err_h[0]) {
    c->setup_done = false;
    char buf[128];
    snprintf(buf, sizeof(buf), "non-positive pivot in set-up (flags 0x%x)", c->err_h[0]);
    return fail(HDGMG_EBREAKDOWN, buf);
  }
  c->setup_done = true;
  return HDGMG_OK;
}

}  // extern "C"

namespace hdgmg {
// Make the condensation autotuner's choice for this context's (kernel, p)
// on its stream, synchronously; the batch set-up calls it for one problem of
// each kind before running the set-ups concurrently, so that concurrent work
// does not disturb the timings.
hdgmg_status tune_condensation(hdgmg_ctx* c, const double* log_kappa) {
  cudaStream_t s = c->stream;
  const int nE = c->n * c->n;
  CUDA_TRY(cudaMemcpyAsync(c->logk, log_kappa, sizeof(double) * nE, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemsetAsync(c->err, 0, sizeof(int) * 4, s));
  launch_kappa(s, nE, c->logk, c->kap);
  Level& L0 = c->levels[0];
  if (c->ns) {
    STATUS_TRY(prepare_pencil(c, log_kappa));
    if (c->cd_basis) {
      launch_condense_cdeig(s, c->refd, c->cd, c->pb, c->p, nE, c->kap, L0.d64.A, c->err, true);
    } else {
      if (!c->Lfac) CUDA_TRY(c->alloc(&c->Lfac, (size_t)c->nv * c->nv * nE));
      launch_condense_cd(s, c->refd, c->cd, c->p, nE, c->kap, L0.d64.A, c->Lfac, c->err, true);
    }
  } else
    c->basis ? launch_condense(s, c->refd, c->p, nE, c->kap, c->ktau, L0.d64.A, c->err, true)
             : launch_condense_factor(s, c->refd, c->p, nE, c->kap, c->ktau, L0.d64.A, c->Lfac,
                                      c->err, true);
  CUDA_TRY(cudaStreamSynchronize(s));
  return check_launch("condensation tuning");
}
bool condensation_kind(const hdgmg_ctx* c, int* p, int* ns) {
  *p = c->p;
  *ns = c->ns ? 1 : 0;
  return true;
}
}  // namespace hdgmg

extern "C" {

hdgmg_status hdgmg_solve(hdgmg_ctx* c, int32_t nrhs, const double* f, const double* g_D,
                         double* lambda, double* u, double* q, hdgmg_info* info) {
  if (!c) return fail(HDGMG_EINVAL, "NULL argument");
  if (nrhs < 0) return fail(HDGMG_EINVAL, "nrhs < 0");
  if (nrhs == 0) {                          // nothing to solve (the pointers may be NULL)
    if (info) {
      info->iters = 0;
      info->converged = 1;
      info->rel_res = 0.0;
    }
    return HDGMG_OK;
  }
  if (!f || !lambda) return fail(HDGMG_EINVAL, "NULL argument");
  if (!c->setup_done) return fail(HDGMG_EINVAL, "hdgmg_setup has not succeeded");
  const size_t nE = (size_t)c->n * c->n;
  const int64_t len = c->fine_len();
  hdgmg_status last = HDGMG_OK;
  const long long l0 = launch_count(), cap0 = c->capture_launches;
  c->launches_solve = 0;
  CUDA_TRY(cudaEventRecord(c->ev0, c->stream));
  if (c->kb > 1 && nrhs > 1) {
    // blocks of up to kb right-hand sides solved together
    for (int k0 = 0; k0 < nrhs; k0 += c->kb) {
      const int k = nrhs - k0 < c->kb ? nrhs - k0 : c->kb;
      hdgmg_status st = solve_block(c, k, f + (size_t)k0 * c->nv * nE,
                                    g_D ? g_D + (size_t)k0 * len : nullptr, lambda + (size_t)k0 * len,
                                    u ? u + (size_t)k0 * c->nv * nE : nullptr,
                                    q ? q + (size_t)k0 * 2 * c->nv * nE : nullptr, info);
      if (st == HDGMG_ECUDA || st == HDGMG_EINVAL || st == HDGMG_ENOMEM || st == HDGMG_ETIMEOUT)
        return st;
      if (st != HDGMG_OK) last = st;
    }
  } else {
    for (int k = 0; k < nrhs; ++k) {
      hdgmg_status st = solve_one(c, f + (size_t)k * c->nv * nE, g_D ? g_D + (size_t)k * len : nullptr,
                                  lambda + (size_t)k * len, u ? u + (size_t)k * c->nv * nE : nullptr,
                                  q ? q + (size_t)k * 2 * c->nv * nE : nullptr, info);
      if (st == HDGMG_ECUDA || st == HDGMG_EINVAL || st == HDGMG_ENOMEM) return st;
      if (st != HDGMG_OK) last = st;
    }
  }
  CUDA_TRY(cudaEventRecord(c->ev1, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (info) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    info->t_solve_ms = ms;
    info->t_setup_ms = c->t_setup_ms;
    info->t_condense_ms = c->t_condense_ms;
    info->condense_threads = c->condense_threads / 16;
    info->condense_elements_per_block = c->condense_threads % 16;
    info->condense_kind =
        (c->ns ? c->cd_basis : c->basis) ? HDGMG_CONDENSE_BASIS : HDGMG_CONDENSE_FACTOR;
    info->n_levels = (int)c->levels.size();
    info->trace_dofs = (int64_t)2 * c->n * (c->n - 1) * (c->p + 1);
  }
  c->launches_solve += launch_count() - l0 - (c->capture_launches - cap0);
  if (info) info->kernel_launches = c->launches_setup + c->launches_solve;
  if (last != HDGMG_OK) return last;
  return HDGMG_OK;
}

hdgmg_status hdgmg_run_host(hdgmg_ctx* c, const double* log_kappa, const double* f,
                            const double* g_D, double* lambda, double* u, double* q,
                            hdgmg_info* info) {
  if (!c || !log_kappa || !f || !lambda) return fail(HDGMG_EINVAL, "NULL argument");
  cudaStream_t s = c->stream;
  const size_t nE = (size_t)c->n * c->n;
  const int64_t len = c->fine_len();
  if (!c->st_f) {
    CUDA_TRY(c->alloc(&c->st_f, (size_t)c->nv * nE));
    CUDA_TRY(c->alloc(&c->st_g, len));
    CUDA_TRY(c->alloc(&c->st_l, len));
    CUDA_TRY(c->alloc(&c->st_u, (size_t)c->nv * nE));
    CUDA_TRY(c->alloc(&c->st_q, (size_t)2 * c->nv * nE));
  }
  // log_kappa lands in the context's own copy through the staging of setup
  CUDA_TRY(cudaMemcpyAsync(c->st_u, log_kappa, sizeof(double) * nE, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(c->st_f, f, sizeof(double) * c->nv * nE, cudaMemcpyHostToDevice, s));
  if (g_D) CUDA_TRY(cudaMemcpyAsync(c->st_g, g_D, sizeof(double) * len, cudaMemcpyHostToDevice, s));
  STATUS_TRY(hdgmg_setup(c, c->st_u));
  hdgmg_status st = hdgmg_solve(c, 1, c->st_f, g_D ? c->st_g : nullptr, c->st_l, u ? c->st_u : nullptr,
                                q ? c->st_q : nullptr, info);
  if (st == HDGMG_ECUDA || st == HDGMG_EINVAL || st == HDGMG_ENOMEM) return st;
  CUDA_TRY(cudaMemcpyAsync(lambda, c->st_l, sizeof(double) * len, cudaMemcpyDeviceToHost, s));
  if (u) CUDA_TRY(cudaMemcpyAsync(u, c->st_u, sizeof(double) * c->nv * nE, cudaMemcpyDeviceToHost, s));
  if (q) CUDA_TRY(cudaMemcpyAsync(q, c->st_q, sizeof(double) * 2 * c->nv * nE, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return st;
}

hdgmg_status hdgmg_adjoint(hdgmg_ctx* c, const double* lambda, const double* u, const double* g_u,
                           double* dL_dlogk, double* dL_df, hdgmg_info* info) {
  if (!c || !lambda || !u || !g_u) return fail(HDGMG_EINVAL, "NULL argument");
  if (c->ns) return fail(HDGMG_EINVAL, "the adjoint is for the symmetric diffusion operator");
  if (!c->setup_done) return fail(HDGMG_EINVAL, "hdgmg_setup has not succeeded");
  STATUS_TRY(adjoint_buffers(c));
  return adjoint_core(c, lambda, u, g_u, dL_dlogk, dL_df, info);
}

hdgmg_status hdgmg_gradient(hdgmg_ctx* c, const double* f, const double* g_D, const double* u_obs,
                            double* J, double* dJ_dlogk, double* dJ_df, hdgmg_info* info) {
  if (!c || !f || !u_obs) return fail(HDGMG_EINVAL, "NULL argument");
  if (c->ns) return fail(HDGMG_EINVAL, "the adjoint is for the symmetric diffusion operator");
  if (!c->setup_done) return fail(HDGMG_EINVAL, "hdgmg_setup has not succeeded");
  STATUS_TRY(adjoint_buffers(c));
  cudaStream_t s = c->stream;
  const int nE = c->n * c->n;
  hdgmg_status st = solve_one(c, f, g_D, c->fwd_lam, c->fwd_u, nullptr, info);
  if (st != HDGMG_OK && st != HDGMG_ENOCONV) return st;
  launch_misfit(s, c->refd, c->nv, nE, c->fwd_u, u_obs, c->mis_d, c->mis_g);
  launch_dot<double>(s, (int64_t)c->nv * nE, c->mis_d, c->mis_g, c->partial, c->scal + 7);
  CUDA_TRY(cudaMemcpyAsync(c->scal_h + 7, c->scal + 7, sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (J) *J = 0.5 * c->scal_h[7];
  hdgmg_status st2 = adjoint_core(c, c->fwd_lam, c->fwd_u, c->mis_g, dJ_dlogk, dJ_df, info);
  return st2 != HDGMG_OK ? st2 : st;
}

hdgmg_status hdgmg_num_levels(hdgmg_ctx* c, int32_t* n_levels) {
  if (!c || !n_levels) return fail(HDGMG_EINVAL, "NULL argument");
  *n_levels = (int32_t)c->levels.size();
  return HDGMG_OK;
}

hdgmg_status hdgmg_level_shape(hdgmg_ctx* c, int32_t level, int32_t* n, int32_t* nd) {
  if (!c || !n || !nd) return fail(HDGMG_EINVAL, "NULL argument");
  if (level < 0 || level >= (int)c->levels.size()) return fail(HDGMG_EINVAL, "level out of range");
  *n = c->levels[level].n;
  *nd = c->levels[level].nd;
  return HDGMG_OK;
}

hdgmg_status hdgmg_copy_element_matrices(hdgmg_ctx* c, int32_t level, double* out) {
  if (!c || !out) return fail(HDGMG_EINVAL, "NULL argument");
  if (level < 0 || level >= (int)c->levels.size()) return fail(HDGMG_EINVAL, "level out of range");
  if (!c->setup_done) return fail(HDGMG_EINVAL, "hdgmg_setup has not succeeded");
  Level& L = c->levels[level];
  if (level == 0 || c->opts.precision == HDGMG_PREC_FP64)
    launch_unpack<double>(c->stream, L.nl, L.nE, c->ns, L.d64.A, out);
  else
    launch_unpack<float>(c->stream, L.nl, L.nE, c->ns, L.d32.A, out);
  STATUS_TRY(check_launch("copy element matrices"));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return HDGMG_OK;
}

hdgmg_status hdgmg_apply_operator(hdgmg_ctx* c, int32_t level, const double* x, double* y) {
  if (!c || !x || !y) return fail(HDGMG_EINVAL, "NULL argument");
  if (level < 0 || level >= (int)c->levels.size()) return fail(HDGMG_EINVAL, "level out of range");
  if (!c->setup_done) return fail(HDGMG_EINVAL, "hdgmg_setup has not succeeded");
  cudaStream_t s = c->stream;
  Level& L = c->levels[level];
  const int64_t len = (int64_t)L.nd * L.nEdge;
  if (level == 0 || c->opts.precision == HDGMG_PREC_FP64) {
    double *xm = nullptr, *ym = nullptr;
    CUDA_TRY(cudaMalloc(&xm, sizeof(double) * len));
    CUDA_TRY(cudaMalloc(&ym, sizeof(double) * len));
    cudaMemcpyAsync(xm, x, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
    launch_mask<double>(s, L.n, L.nd, xm);
    cudaMemsetAsync(ym, 0, sizeof(double) * len, s);
    launch_matvec<double>(s, L.n, L.nd, c->ns, L.d64.A, xm, ym, 1.0);
    cudaMemcpyAsync(y, ym, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
    cudaStreamSynchronize(s);
    cudaFree(xm);
    cudaFree(ym);
  } else {
    float *xm = nullptr, *ym = nullptr;
    CUDA_TRY(cudaMalloc(&xm, sizeof(float) * len));
    CUDA_TRY(cudaMalloc(&ym, sizeof(float) * len));
    launch_convert<double, float>(s, len, x, xm);
    launch_mask<float>(s, L.n, L.nd, xm);
    cudaMemsetAsync(ym, 0, sizeof(float) * len, s);
    launch_matvec<float>(s, L.n, L.nd, c->ns, L.d32.A, xm, ym, 1.0f);
    launch_convert<float, double>(s, len, ym, y);
    cudaStreamSynchronize(s);
    cudaFree(xm);
    cudaFree(ym);
  }
  return check_launch("apply operator");
}

hdgmg_status hdgmg_apply_vcycle(hdgmg_ctx* c, const double* r, double* e) {
  if (!c || !r || !e) return fail(HDGMG_EINVAL, "NULL argument");
  if (!c->setup_done) return fail(HDGMG_EINVAL, "hdgmg_setup has not succeeded");
  cudaStream_t s = c->stream;
  const int64_t len = c->fine_len();
  CUDA_TRY(cudaMemcpyAsync(c->r, r, sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
  launch_mask<double>(s, c->n, c->p + 1, c->r);
  apply_B(c, c->r, e);
  STATUS_TRY(check_launch("apply vcycle"));
  if (c->pc_start >= 0)
    CUDA_TRY(cudaMemcpyAsync(c->err_h + 2, c->err + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return cycle_wait_status(c);
}

hdgmg_status hdgmg_trace_vcycle(hdgmg_ctx* c, const double* r, double* e, int64_t* stamps,
                                int32_t cap, int32_t* count) {
  if (!c || !r || !e || !stamps || !count) return fail(HDGMG_EINVAL, "NULL argument");
  if (!c->setup_done) return fail(HDGMG_EINVAL, "hdgmg_setup has not succeeded");
  if (c->pc_start < 0) return fail(HDGMG_EINVAL, "this context does not run the persistent cycle");
  if (cap < 1 || cap > 4096) return fail(HDGMG_EINVAL, "cap must be in [1, 4096]");
  cudaStream_t s = c->stream;
  if (c->pc_trace_cap < cap) {
    if (c->pc_trace) cudaFree(c->pc_trace);
    c->pc_trace = nullptr;
    c->pc_trace_cap = 0;
    CUDA_TRY(cudaMalloc(&c->pc_trace, sizeof(unsigned long long) * 2 * (size_t)cap));
    c->pc_trace_cap = cap;
  }
  CUDA_TRY(cudaMemsetAsync(c->pc_trace, 0xff, sizeof(unsigned long long) * 2 * (size_t)cap, s));
  const int saved = c->pc_trace_cap;
  c->pc_trace_cap = cap;
  c->pc_trace_armed = true;
  const hdgmg_status st = hdgmg_apply_vcycle(c, r, e);
  c->pc_trace_armed = false;
  c->pc_trace_cap = saved;
  if (st != HDGMG_OK) return st;
  std::vector<unsigned long long> h(2 * (size_t)cap);
  CUDA_TRY(cudaMemcpy(h.data(), c->pc_trace, sizeof(unsigned long long) * h.size(),
                      cudaMemcpyDeviceToHost));
  int k = 0;
  while (k < cap && h[2 * k] != ~0ull) ++k;
  for (int i = 0; i < 2 * k; ++i) stamps[i] = (int64_t)h[i];
  *count = k;
  return HDGMG_OK;
}

hdgmg_status hdgmg_check_cycle_timeout(hdgmg_ctx* c, int32_t wait_us) {
  if (!c) return fail(HDGMG_EINVAL, "NULL argument");
  if (!c->setup_done) return fail(HDGMG_EINVAL, "hdgmg_setup has not succeeded");
  if (c->pc_start < 0) return fail(HDGMG_EINVAL, "this context does not run the persistent cycle");
  const int tail = c->opts.precision != HDGMG_PREC_FP64 ? c->pc32.tail : c->pc64.tail;
  if (tail == 0) return fail(HDGMG_EINVAL, "this context's cycle runs on one block (no grid barrier)");
  if (wait_us < 1 || wait_us > 1000000) return fail(HDGMG_EINVAL, "wait_us must be in [1, 1e6]");
  cudaStream_t s = c->stream;
  cudaError_t e;
  if (c->opts.precision != HDGMG_PREC_FP64) {
    PCycleParams<float> P = c->pc32;
    P.withhold = 1;
    P.wait_ns = (unsigned long long)wait_us * 1000ull;
    e = launch_pcycle<float>(s, P, c->pc_blocks);
  } else {
    PCycleParams<double> P = c->pc64;
    P.withhold = 1;
    P.wait_ns = (unsigned long long)wait_us * 1000ull;
    e = launch_pcycle<double>(s, P, c->pc_blocks);
  }
  if (e != cudaSuccess) return fail(HDGMG_ECUDA, std::string("persistent cycle: ") + cudaGetErrorString(e));
  CUDA_TRY(cudaMemcpyAsync(c->err_h + 2, c->err + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return cycle_wait_status(c);
}

hdgmg_status hdgmg_condensed_rhs(hdgmg_ctx* c, const double* f, const double* g_D, double* b) {
  if (!c || !f || !b) return fail(HDGMG_EINVAL, "NULL argument");
  if (!c->setup_done) return fail(HDGMG_EINVAL, "hdgmg_setup has not succeeded");
  STATUS_TRY(build_rhs(c, f, g_D));
  CUDA_TRY(cudaMemcpyAsync(b, c->b, sizeof(double) * c->fine_len(), cudaMemcpyDeviceToDevice, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return HDGMG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free variant of hdgmg_apply_operator.
//
// hdgmg_apply_operator takes its temporaries (the copy of x with the
// Dirichlet entries zeroed, and the FP32 accumulator on FP32 levels) from
// cudaMalloc on every call.  Some callers cannot allocate device memory at
// the point where they need the operator: integrations whose device memory
// is owned by another allocator (a cudaMalloc would fail or fragment it), and
// latency-critical loops that must not call cudaMalloc/cudaFree (both can
// synchronise the device).  For them the temporaries live in one fixed array
// that the library reserves in device memory when it is loaded.
// ---------------------------------------------------------------------------
namespace {

// 2^20 doubles (8 MiB) on every device that loads the library, held until
// the process exits.  Shared by all calls: calls whose work overlaps on the
// GPU (different streams, or different host threads) race on it.
constexpr size_t kNoAllocScratchDoubles = size_t(1) << 20;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array for the current device; resolved once
// per device (the host-side symbol is only a stand-in for it).
hdgmg_status noalloc_scratch(double** out) {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(HDGMG_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return HDGMG_OK;
}

}  // namespace

extern "C" hdgmg_status hdgmg_apply_operator_noalloc(hdgmg_ctx* c, int32_t level, const double* x,
                                                     double* y) {
  if (!c || !x || !y) return fail(HDGMG_EINVAL, "NULL argument");
  if (level < 0 || level >= (int)c->levels.size()) return fail(HDGMG_EINVAL, "level out of range");
  Level& L = c->levels[level];
  const int64_t len = (int64_t)L.nd * L.nEdge;
  if ((size_t)len > kNoAllocScratchDoubles) {
    char buf[160];
    snprintf(buf, sizeof(buf),
             "level %d has %lld trace values; the static scratch holds at most %zu",
             (int)level, (long long)len, kNoAllocScratchDoubles);
    return fail(HDGMG_EINVAL, buf);
  }
  if (!c->setup_done) return fail(HDGMG_EINVAL, "hdgmg_setup has not succeeded");
  double* scratch = nullptr;
  STATUS_TRY(noalloc_scratch(&scratch));
  cudaStream_t s = c->stream;
  if (level == 0 || c->opts.precision == HDGMG_PREC_FP64) {
    double* xm = scratch;                          // fully overwritten below
    CUDA_TRY(cudaMemcpyAsync(xm, x, sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
    launch_mask<double>(s, L.n, L.nd, xm);
    CUDA_TRY(cudaMemsetAsync(y, 0, sizeof(double) * len, s));
    launch_matvec<double>(s, L.n, L.nd, c->ns, L.d64.A, xm, y, 1.0);
  } else {
    float* xm = reinterpret_cast<float*>(scratch);  // len floats, fully overwritten
    float* ym = xm + len;                          // len floats, cleared below
    launch_convert<double, float>(s, len, x, xm);
    launch_mask<float>(s, L.n, L.nd, xm);
    CUDA_TRY(cudaMemsetAsync(ym, 0, sizeof(float) * len, s));
    launch_matvec<float>(s, L.n, L.nd, c->ns, L.d32.A, xm, ym, 1.0f);
    launch_convert<float, double>(s, len, ym, y);
  }
  STATUS_TRY(check_launch("apply operator (no allocation)"));
  CUDA_TRY(cudaStreamSynchronize(s));
  return HDGMG_OK;
}
