// Algorithm 1 (arXiv:1811.09909, Sec. 3.6) on the P1 tail of the hierarchy,
// run by ONE thread-block cluster.
//
// The coarse levels of the V-cycle are tiny and latency-bound: as separate
// kernels every smoothing sweep, local correction (eq. localCorrection) and
// transfer (eqs. n_1_Ik, n_1_Qk) costs a launch.  Here the levels with few
// macro-elements are processed by the CTAs of one cluster:
//   * every level vector (r, e, y) is split across the CTAs' shared memory
//     (distributed shared memory) by edge ranges;
//   * the level operators are split the same way by element / macro-element
//     ranges and staged into shared memory when they fit, otherwise read
//     from L2;
//   * each step is executed by the CTA that owns the item (edge, element,
//     macro-element), neighbour values are read and accumulated through
//     DSMEM, and the steps are separated by cluster barriers
//     (barrier.cluster with release/acquire semantics) instead of kernel
//     launches.
// The algebra of every step is the one of the single-kernel versions in
// k_mg.cu / k_edge.cuh.
#include <cooperative_groups.h>

#include "k_common.cuh"

namespace cg = cooperative_groups;

namespace hdgmg {

namespace {

// Array split over the CTAs of the cluster: CTA r holds items
// [r*chunk, (r+1)*chunk) as [stride][chunk] in its shared memory at the same
// offset in every CTA.  When not staged (loc == nullptr) the values are read
// from the global structure-of-arrays copy g[k][N].
template <typename T>
struct DArr {
  T* loc;
  const T* g;
  int chunk, N;
  __device__ __forceinline__ T* at(const cg::cluster_group& cl, int item, int k) const {
    const int r = item / chunk;
    T* b = cl.map_shared_rank(loc, (unsigned)r);
    return b + (size_t)k * chunk + (item - r * chunk);
  }
  __device__ __forceinline__ T get(const cg::cluster_group& cl, int item, int k) const {
    return loc ? *at(cl, item, k) : g[(size_t)k * N + item];
  }
};

template <typename T>
struct LevelView {
  int n, m, nE, ned, nc;
  DArr<T> r, e, y, A, D, AII, Y, Pi;
};

template <typename T>
__device__ __forceinline__ LevelView<T> view(const CTailParams<T>& P, int l, T* sm) {
  const CTailLevel<T>& L = P.lv[l];
  LevelView<T> v;
  v.n = L.n;
  v.m = L.m;
  v.nE = L.n * L.n;
  v.ned = L.nEdge;
  v.nc = L.n / 2;
  T* vb = sm + L.off_v;
  v.r = {vb, nullptr, L.edchunk, L.nEdge};
  v.e = {vb + 2 * L.edchunk, nullptr, L.edchunk, L.nEdge};
  v.y = {vb + 4 * L.edchunk, nullptr, L.edchunk, L.nEdge};
  const int nC = v.nE / 4;
  v.A = {L.off_A >= 0 ? sm + L.off_A : nullptr, L.A, L.echunk, v.nE};
  v.D = {L.off_D >= 0 ? sm + L.off_D : nullptr, L.Dinv, L.edchunk, L.nEdge};
  v.AII = {L.off_AII >= 0 ? sm + L.off_AII : nullptr, L.AIIinv, L.cchunk, nC};
  v.Y = {L.off_Y >= 0 ? sm + L.off_Y : nullptr, L.Y, L.cchunk, nC};
  v.Pi = {L.off_Pi >= 0 ? sm + L.off_Pi : nullptr, L.Pi, L.cchunk, nC};
  return v;
}

// loop over the items [0, N) owned by this CTA (chunk per CTA)
#define OWNED(item, N, chunk)                                                          \
  for (int li_ = threadIdx.x, item = (int)cl.block_rank() * (chunk) + threadIdx.x;    \
       li_ < (chunk) && item < (N); li_ += blockDim.x, item += blockDim.x)

template <typename T>
__device__ __forceinline__ void c_bj(const cg::cluster_group& cl, const LevelView<T>& v, T omega,
                                     bool first) {
  OWNED(edge, v.ned, v.r.chunk) {
    if (bnd_edge(v.n, edge)) continue;
    T* r0 = v.r.at(cl, edge, 0);
    T* r1 = v.r.at(cl, edge, 1);
    T* y0 = v.y.at(cl, edge, 0);
    T* y1 = v.y.at(cl, edge, 1);
    T* e0 = v.e.at(cl, edge, 0);
    T* e1 = v.e.at(cl, edge, 1);
    const T d0 = first ? *r0 : *r0 - *y0;
    const T d1 = first ? *r1 : *r1 - *y1;
    if (!first) {
      *y0 = T(0);
      *y1 = T(0);
    }
    const T a00 = v.D.get(cl, edge, 0), a10 = v.D.get(cl, edge, 1), a11 = v.D.get(cl, edge, 2);
    const T s0 = a00 * d0 + a10 * d1, s1 = a10 * d0 + a11 * d1;
    *e0 = first ? omega * s0 : *e0 + omega * s0;
    *e1 = first ? omega * s1 : *e1 + omega * s1;
  }
}

template <typename T>
__device__ __forceinline__ void c_matvec(const cg::cluster_group& cl, const LevelView<T>& v) {
  OWNED(el, v.nE, v.A.chunk) {
    int ed[4];
    elem_edges(v.n, el, ed);
    T xl[8], yl[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      xl[c] = *v.e.at(cl, ed[c >> 1], c & 1);
      yl[c] = T(0);
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
#pragma unroll
      for (int c = 0; c < r; ++c) {
        const T a = v.A.get(cl, el, pk(r, c));
        yl[r] += a * xl[c];
        yl[c] += a * xl[r];
      }
      yl[r] += v.A.get(cl, el, pk(r, r)) * xl[r];
    }
#pragma unroll
    for (int le = 0; le < 4; ++le) {
      if (bnd_edge(v.n, ed[le])) continue;
      atomicAdd(v.y.at(cl, ed[le], 0), yl[le * 2]);
      atomicAdd(v.y.at(cl, ed[le], 1), yl[le * 2 + 1]);
    }
  }
}

// e_I = A_II^-1 r_I + Y e_B per macro-element of the next coarser level
template <typename T>
__device__ __forceinline__ void c_local_correction(const cg::cluster_group& cl,
                                                   const LevelView<T>& v) {
  const int nc = v.nc;
  OWNED(C, nc * nc, v.AII.chunk) {
    const int J = C / nc, I = C - J * nc;
    T rI[8], eB[16];
#pragma unroll
    for (int ie = 0; ie < 4; ++ie) {
      const int ed = interior_edge(v.n, I, J, ie);
      rI[ie * 2] = *v.r.at(cl, ed, 0);
      rI[ie * 2 + 1] = *v.r.at(cl, ed, 1);
    }
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int ed = perimeter_edge(v.n, I, J, b >> 1, b & 1);
      eB[b * 2] = *v.e.at(cl, ed, 0);
      eB[b * 2 + 1] = *v.e.at(cl, ed, 1);
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      T s = T(0);
#pragma unroll
      for (int k = 0; k < 8; ++k) s += v.AII.get(cl, C, pk_any(a, k)) * rI[k];
#pragma unroll
      for (int b = 0; b < 16; ++b) s += v.Y.get(cl, C, a * 16 + b) * eB[b];
      *v.e.at(cl, interior_edge(v.n, I, J, a >> 1), a & 1) = s;
    }
  }
}

// r_c = J^T s_B + Pi^T s_I with s = r - y, per coarse edge
template <typename T>
__device__ __forceinline__ void c_restrict(const cg::cluster_group& cl, const LevelView<T>& v,
                                           const LevelView<T>& vc, const double (&Jc)[2][2][2]) {
  const int nc = v.nc, n = v.n, nvc = nc * (nc + 1);
  OWNED(E, vc.ned, vc.r.chunk) {
    T* rc0 = vc.r.at(cl, E, 0);
    T* rc1 = vc.r.at(cl, E, 1);
    if (bnd_edge(nc, E)) {
      *rc0 = T(0);
      *rc1 = T(0);
      continue;
    }
    int ch[2], Cs[2], mes[2];
    if (E < nvc) {
      const int J = E / (nc + 1), I = E % (nc + 1);
      ch[0] = fine_v(n, 2 * I, 2 * J);
      ch[1] = fine_v(n, 2 * I, 2 * J + 1);
      Cs[0] = J * nc + I - 1; mes[0] = 1;
      Cs[1] = J * nc + I;     mes[1] = 0;
    } else {
      const int J = (E - nvc) / nc, I = (E - nvc) % nc;
      ch[0] = fine_h(n, 2 * I, 2 * J);
      ch[1] = fine_h(n, 2 * I + 1, 2 * J);
      Cs[0] = (J - 1) * nc + I; mes[0] = 3;
      Cs[1] = J * nc + I;       mes[1] = 2;
    }
    T acc0 = T(0), acc1 = T(0);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const T s0 = *v.r.at(cl, ch[c], 0) - *v.y.at(cl, ch[c], 0);
      const T s1 = *v.r.at(cl, ch[c], 1) - *v.y.at(cl, ch[c], 1);
      acc0 += (T)Jc[c][0][0] * s0 + (T)Jc[c][1][0] * s1;
      acc1 += (T)Jc[c][0][1] * s0 + (T)Jc[c][1][1] * s1;
    }
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int C = Cs[side];
      const int J = C / nc, I = C - J * nc;
#pragma unroll
      for (int ie = 0; ie < 4; ++ie) {
        const int ed = interior_edge(n, I, J, ie);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const T s = *v.r.at(cl, ed, k) - *v.y.at(cl, ed, k);
          const int a = ie * 2 + k;
          acc0 += v.Pi.get(cl, C, a * 8 + mes[side] * 2) * s;
          acc1 += v.Pi.get(cl, C, a * 8 + mes[side] * 2 + 1) * s;
        }
      }
    }
    *rc0 = acc0;
    *rc1 = acc1;
  }
}

// e_I += Pi e_c(C) per macro-element, e_B += J e_c per coarse edge; y reset
template <typename T>
__device__ __forceinline__ void c_prolong(const cg::cluster_group& cl, const LevelView<T>& v,
                                          const LevelView<T>& vc, const double (&Jc)[2][2][2]) {
  const int nc = v.nc, n = v.n, nvc = nc * (nc + 1);
  OWNED(C, nc * nc, v.Pi.chunk) {
    const int J = C / nc, I = C - J * nc;
    const int ce[4] = {coarse_v(nc, I, J), coarse_v(nc, I + 1, J), coarse_h(nc, I, J),
                       coarse_h(nc, I, J + 1)};
    T xc[8];
#pragma unroll
    for (int me = 0; me < 4; ++me) {
      xc[me * 2] = *vc.e.at(cl, ce[me], 0);
      xc[me * 2 + 1] = *vc.e.at(cl, ce[me], 1);
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      T s = T(0);
#pragma unroll
      for (int b = 0; b < 8; ++b) s += v.Pi.get(cl, C, a * 8 + b) * xc[b];
      const int ed = interior_edge(n, I, J, a >> 1);
      T* ep = v.e.at(cl, ed, a & 1);
      *ep += s;
      *v.y.at(cl, ed, a & 1) = T(0);
    }
  }
  OWNED(E, vc.ned, vc.e.chunk) {
    int ch[2];
    if (E < nvc) {
      const int J = E / (nc + 1), I = E % (nc + 1);
      ch[0] = fine_v(n, 2 * I, 2 * J);
      ch[1] = fine_v(n, 2 * I, 2 * J + 1);
    } else {
      const int J = (E - nvc) / nc, I = (E - nvc) % nc;
      ch[0] = fine_h(n, 2 * I, 2 * J);
      ch[1] = fine_h(n, 2 * I + 1, 2 * J);
    }
    const T x0 = *vc.e.at(cl, E, 0), x1 = *vc.e.at(cl, E, 1);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
#pragma unroll
      for (int kf = 0; kf < 2; ++kf) {
        T* ep = v.e.at(cl, ch[c], kf);
        *ep += (T)Jc[c][kf][0] * x0 + (T)Jc[c][kf][1] * x1;
        *v.y.at(cl, ch[c], kf) = T(0);
      }
    }
  }
}

template <typename T, int NTHR>
__global__ void __launch_bounds__(NTHR) ctail_kernel(const CTailParams<T> P) {
  extern __shared__ __align__(16) unsigned char ctail_smem[];
  cg::cluster_group cl = cg::this_cluster();
  T* sm = reinterpret_cast<T*>(ctail_smem);
  const int rank = (int)cl.block_rank();
  // stage this CTA's partitions, clear the vectors
  for (int l = 0; l < P.nlev; ++l) {
    const CTailLevel<T>& L = P.lv[l];
    T* vb = sm + L.off_v;
    for (int i = threadIdx.x; i < 6 * L.edchunk; i += blockDim.x) vb[i] = T(0);
    if (l + 1 == P.nlev) continue;
    const int nE = L.n * L.n, nC = nE / 4;
    auto stage = [&](int off, const T* g, int chunk, int N, int stride) {
      if (off < 0) return;
      T* dst = sm + off;
      for (int t = threadIdx.x; t < stride * chunk; t += blockDim.x) {
        const int k = t / chunk, li = t - k * chunk, item = rank * chunk + li;
        dst[t] = item < N ? g[(size_t)k * N + item] : T(0);
      }
    };
    stage(L.off_A, L.A, L.echunk, nE, 36);
    stage(L.off_D, L.Dinv, L.edchunk, L.nEdge, 3);
    stage(L.off_AII, L.AIIinv, L.cchunk, nC, 36);
    stage(L.off_Y, L.Y, L.cchunk, nC, 128);
    stage(L.off_Pi, L.Pi, L.cchunk, nC, 64);
  }
  __syncthreads();
  {
    const CTailLevel<T>& L = P.lv[0];
    T* r = sm + L.off_v;
    for (int li = threadIdx.x; li < L.edchunk; li += blockDim.x) {
      const int edge = rank * L.edchunk + li;
      if (edge < L.nEdge) {
        r[li] = P.r_in[edge];
        r[L.edchunk + li] = P.r_in[(size_t)L.nEdge + edge];
      }
    }
  }
  cl.sync();
  // down sweep (steps 2-4)
  for (int l = 0; l + 1 < P.nlev; ++l) {
    const LevelView<T> v = view(P, l, sm);
    const LevelView<T> vc = view(P, l + 1, sm);
    c_bj(cl, v, P.omega, true);
    cl.sync();
    for (int it = 1; it < v.m; ++it) {
      c_matvec(cl, v);
      cl.sync();
      c_bj(cl, v, P.omega, false);
      cl.sync();
    }
    if (P.lc != HDGMG_LC_NONE) {
      c_local_correction(cl, v);
      cl.sync();
    }
    c_matvec(cl, v);
    cl.sync();
    c_restrict(cl, v, vc, P.Jc);
    cl.sync();
  }
  // B_1 = A_1^-1 on CTA 0 (dense FP64 inverse)
  if (rank == 0) {
    const LevelView<T> v = view(P, P.nlev - 1, sm);
    double* w = reinterpret_cast<double*>(ctail_smem + P.w_off);
    for (int ed = threadIdx.x; ed < v.ned; ed += blockDim.x) {
      const int f = P.fidx[ed];
      if (f >= 0) {
        w[f * 2] = (double)*v.r.at(cl, ed, 0);
        w[f * 2 + 1] = (double)*v.r.at(cl, ed, 1);
      } else {
        *v.e.at(cl, ed, 0) = T(0);
        *v.e.at(cl, ed, 1) = T(0);
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < P.nf; i += blockDim.x) {
      double s = 0.0;
      for (int j = 0; j < P.nf; ++j) s += P.Ainv[(size_t)i * P.nf + j] * w[j];
      *v.e.at(cl, P.fedge[i >> 1], i & 1) = (T)s;
    }
  }
  cl.sync();
  // up sweep (steps 4-6)
  for (int l = P.nlev - 2; l >= 0; --l) {
    const LevelView<T> v = view(P, l, sm);
    const LevelView<T> vc = view(P, l + 1, sm);
    c_prolong(cl, v, vc, P.Jc);
    cl.sync();
    if (P.lc == HDGMG_LC_BOTH) {
      c_local_correction(cl, v);
      cl.sync();
    }
    for (int it = 0; it < v.m; ++it) {
      c_matvec(cl, v);
      cl.sync();
      c_bj(cl, v, P.omega, false);
      cl.sync();
    }
  }
  {
    const CTailLevel<T>& L = P.lv[0];
    const T* e = sm + L.off_v + 2 * L.edchunk;
    for (int li = threadIdx.x; li < L.edchunk; li += blockDim.x) {
      const int edge = rank * L.edchunk + li;
      if (edge < L.nEdge) {
        P.e_out[edge] = e[li];
        P.e_out[(size_t)L.nEdge + edge] = e[L.edchunk + li];
      }
    }
  }
  // no CTA may exit while others still read its shared memory
  cl.sync();
}

#undef OWNED

template <typename T>
constexpr int ctail_threads() {
  return sizeof(T) == 8 ? 512 : 1024;
}

template <typename T>
void ctail_attributes() {
  static const bool done = [] {
    constexpr int NTHR = ctail_threads<T>();
    cudaFuncSetAttribute(ctail_kernel<T, NTHR>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(ctail_kernel<T, NTHR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kTailMaxSmem);
    return true;
  }();
  (void)done;
}

}  // namespace

template <typename T>
int ctail_max_clusters(int cluster, int smem_bytes) {
  constexpr int NTHR = ctail_threads<T>();
  ctail_attributes<T>();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster, 1, 1);
  cfg.blockDim = dim3(NTHR, 1, 1);
  cfg.dynamicSmemBytes = (size_t)smem_bytes;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, ctail_kernel<T, NTHR>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <typename T>
void launch_ctail(cudaStream_t s, const CTailParams<T>& P) {
  constexpr int NTHR = ctail_threads<T>();
  ctail_attributes<T>();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P.cl, 1, 1);
  cfg.blockDim = dim3(NTHR, 1, 1);
  cfg.dynamicSmemBytes = (size_t)P.smem_bytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = P.cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  note_launch();
  cudaLaunchKernelEx(&cfg, ctail_kernel<T, NTHR>, P);
}

template int ctail_max_clusters<float>(int, int);
template int ctail_max_clusters<double>(int, int);
template void launch_ctail<float>(cudaStream_t, const CTailParams<float>&);
template void launch_ctail<double>(cudaStream_t, const CTailParams<double>&);

}  // namespace hdgmg
