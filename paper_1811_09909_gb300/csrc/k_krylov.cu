// Flexible GMRES kernels (FP64): the Arnoldi step runs entirely on the
// device so that one restart cycle is one CUDA graph with a device-side
// while condition.  The current Arnoldi index j lives in device memory and
// every kernel reads it, so the same graph body serves every step.
//
// Right preconditioning with the V-cycle, z_j = B v_j, w = A z_j (Sec. 3.6;
// Sec. 4 solves with multigrid-preconditioned GMRES), classical Gram-Schmidt
// applied twice, Givens rotations on the Hessenberg column.
#include "k_common.cuh"

namespace hdgmg {

namespace {

constexpr int kGmBlocks = 304;     // 2 x 152 SMs, fixed: deterministic sums

__global__ void gm_select_kernel(int64_t len, const double* __restrict__ base,
                                 const int* __restrict__ jp, int shift, double* __restrict__ out) {
  const double* src = base + (int64_t)(*jp + shift) * len;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = src[i];
}

__global__ void gm_store_kernel(int64_t len, const double* __restrict__ in, double* __restrict__ base,
                                const int* __restrict__ jp, int shift) {
  double* dst = base + (int64_t)(*jp + shift) * len;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = in[i];
}

// partial[k][block] = sum_i V[k][i] w[i] for k <= j: the dot products of up to
// KC basis vectors per pass over the data (w read once per pass, the KC sums
// in registers, reduced by warp shuffles and across the block's warps)
constexpr int kMultidotChunk = 16;
__global__ void __launch_bounds__(256) gm_multidot_kernel(int64_t len, const double* __restrict__ V,
                                                          const int* __restrict__ jp,
                                                          const double* __restrict__ w,
                                                          double* __restrict__ partial) {
  constexpr int KC = kMultidotChunk;
  __shared__ double sh[KC][8];
  const int nk = *jp + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k0 = 0; k0 < nk; k0 += KC) {
    const int kc = nk - k0 < KC ? nk - k0 : KC;
    const double* vb = V + (int64_t)k0 * len;
    double s[KC];
#pragma unroll
    for (int q = 0; q < KC; ++q) s[q] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x) {
      const double wi = w[i];
#pragma unroll
      for (int q = 0; q < KC; ++q)
        if (q < kc) s[q] = fma(vb[(int64_t)q * len + i], wi, s[q]);
    }
#pragma unroll
    for (int q = 0; q < KC; ++q) {
      double t = s[q];
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      if (lane == 0) sh[q][warp] = t;
    }
    __syncthreads();
    if (threadIdx.x < kc) {
      double t = 0.0;
      for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) t += sh[threadIdx.x][wv];
      partial[(k0 + threadIdx.x) * gridDim.x + blockIdx.x] = t;
    }
    __syncthreads();
  }
}

// h[k] = sum_b partial[k][b]; H[:, j] (+)= h
__global__ void gm_multidot_final_kernel(const int* __restrict__ jp, const double* __restrict__ partial,
                                         int nblocks, int ldh, double* __restrict__ H,
                                         double* __restrict__ h, int accumulate) {
  const int nk = *jp + 1;
  const int k = blockIdx.x;
  if (k >= nk) return;
  __shared__ double sh[256];
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partial[k * nblocks + b];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    h[k] = sh[0];
    double* col = H + (int64_t)(*jp) * ldh;
    col[k] = accumulate ? col[k] + sh[0] : sh[0];
  }
}

// w -= sum_{k <= j} h[k] V[k]
__global__ void gm_subtract_kernel(int64_t len, const double* __restrict__ V,
                                   const int* __restrict__ jp, const double* __restrict__ h,
                                   double* __restrict__ w) {
  const int nk = *jp + 1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = w[i];
    for (int k = 0; k < nk; ++k) s -= h[k] * V[(int64_t)k * len + i];
    w[i] = s;
  }
}

// V[j+1] = w / sqrt(nrm2)  (zero if the norm vanished: happy breakdown)
__global__ void gm_normalize_kernel(int64_t len, const double* __restrict__ w,
                                    const double* __restrict__ nrm2, double* __restrict__ V,
                                    const int* __restrict__ jp) {
  const double nrm = sqrt(*nrm2);
  const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  double* dst = V + (int64_t)(*jp + 1) * len;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = w[i] * inv;
}

// Hessenberg column j: H[j+1][j] = ||w||, apply the previous rotations, form
// the new one, update the residual vector g, advance j and evaluate the test.
__global__ void gm_givens_kernel(double* __restrict__ H, int ldh, double* __restrict__ cs,
                                 double* __restrict__ sn, double* __restrict__ g,
                                 int* __restrict__ jp, int m, const double* __restrict__ tolp,
                                 const double* __restrict__ nrm2, cudaGraphConditionalHandle hdl,
                                 int* __restrict__ total, int max_total) {
  const double tol_abs = *tolp;
  const int j = *jp;
  double* col = H + (int64_t)j * ldh;
  col[j + 1] = sqrt(*nrm2);
  for (int i = 0; i < j; ++i) {
    const double t = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t;
  }
  const double a = col[j], b = col[j + 1];
  const double den = sqrt(a * a + b * b);
  const double c = den > 0.0 ? a / den : 1.0;
  const double s = den > 0.0 ? b / den : 0.0;
  cs[j] = c;
  sn[j] = s;
  col[j] = den;
  col[j + 1] = 0.0;
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
  *jp = j + 1;
  const int tot = ++(*total);
  const double res = fabs(g[j + 1]);
  if (!(res > tol_abs) || j + 1 >= m || tot >= max_total || !(*nrm2 > 0.0))
    cudaGraphSetConditional(hdl, 0);
}

// x += sum_{k < nk} y[k] Z[k]
__global__ void gm_update_kernel(int64_t len, const double* __restrict__ Z, int nk,
                                 const double* __restrict__ y, double* __restrict__ x) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = x[i];
    for (int k = 0; k < nk; ++k) s += y[k] * Z[(int64_t)k * len + i];
    x[i] = s;
  }
}

inline int vblocks(int64_t len) {
  int b = nblk(len, 256);
  return b > 2432 ? 2432 : b;
}

}  // namespace

int gm_partial_blocks() { return kGmBlocks; }

void launch_gm_select(cudaStream_t s, int64_t len, const double* base, const int* jp, int shift,
                      double* out) {
  note_launch();
  gm_select_kernel<<<vblocks(len), 256, 0, s>>>(len, base, jp, shift, out);
}

void launch_gm_store(cudaStream_t s, int64_t len, const double* in, double* base, const int* jp,
                     int shift) {
  note_launch();
  gm_store_kernel<<<vblocks(len), 256, 0, s>>>(len, in, base, jp, shift);
}

void launch_gm_orthogonalize(cudaStream_t s, int64_t len, const double* V, const int* jp,
                             double* w, double* partial, int ldh, double* H, double* h,
                             int max_k, int accumulate) {
  note_launch();
  gm_multidot_kernel<<<kGmBlocks, 256, 0, s>>>(len, V, jp, w, partial);
  note_launch();
  gm_multidot_final_kernel<<<max_k, 256, 0, s>>>(jp, partial, kGmBlocks, ldh, H, h, accumulate);
  note_launch();
  gm_subtract_kernel<<<vblocks(len), 256, 0, s>>>(len, V, jp, h, w);
}

void launch_gm_normalize(cudaStream_t s, int64_t len, const double* w, const double* nrm2, double* V,
                         const int* jp) {
  note_launch();
  gm_normalize_kernel<<<vblocks(len), 256, 0, s>>>(len, w, nrm2, V, jp);
}

void launch_gm_givens(cudaStream_t s, double* H, int ldh, double* cs, double* sn, double* g, int* jp,
                      int m, const double* tolp, const double* nrm2, cudaGraphConditionalHandle hdl,
                      int* total, int max_total) {
  note_launch();
  gm_givens_kernel<<<1, 1, 0, s>>>(H, ldh, cs, sn, g, jp, m, tolp, nrm2, hdl, total, max_total);
}

void launch_gm_update(cudaStream_t s, int64_t len, const double* Z, int nk, const double* y,
                      double* x) {
  note_launch();
  gm_update_kernel<<<vblocks(len), 256, 0, s>>>(len, Z, nk, y, x);
}

}  // namespace hdgmg
