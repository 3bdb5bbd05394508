// One (type, ND) instantiation of the edge/element kernels of k_edge.cuh;
// built once per pair with -DHDGMG_REAL=<double|float> -DHDGMG_ND=<2..9>, and
// once per ND with -DHDGMG_BF16 for the BF16-storage matvec alone (separate
// units so that the widest ones compile in parallel).
#include <cstring>

#include "k_edge.cuh"
#include "k_mf.cuh"

#ifndef HDGMG_REAL
#define HDGMG_REAL double
#endif
#ifndef HDGMG_ND
#define HDGMG_ND 2
#endif
#ifndef HDGMG_REAL_IS_DOUBLE
#define HDGMG_REAL_IS_DOUBLE 0
#endif

namespace hdgmg {
#ifndef HDGMG_BF16
#define HDGMG_INST(NS)                                                                          \
  template void launch_matvec_nd<HDGMG_REAL, HDGMG_ND, NS>(cudaStream_t, int, const HDGMG_REAL*, \
                                                           const HDGMG_REAL*, HDGMG_REAL*,      \
                                                           HDGMG_REAL, const HDGMG_REAL*, int); \
  template void launch_bj_blocks_nd<HDGMG_REAL, HDGMG_ND, NS>(cudaStream_t, int,                \
                                                              const HDGMG_REAL*, HDGMG_REAL*,  \
                                                              int*);                           \
  template void launch_bj_update_nd<HDGMG_REAL, HDGMG_ND, NS>(                                  \
      cudaStream_t, int, const HDGMG_REAL*, const HDGMG_REAL*, HDGMG_REAL*, HDGMG_REAL*,        \
      HDGMG_REAL, int, const HDGMG_REAL*, int);
HDGMG_INST(false)
HDGMG_INST(true)
#undef HDGMG_INST
#if !HDGMG_REAL_IS_DOUBLE && HDGMG_ND <= 7
template void launch_matvec_mf_nd<HDGMG_ND>(cudaStream_t, int, const float*, const double*,
                                            const float*, float*, float, const float*, int);
#endif
#if !HDGMG_REAL_IS_DOUBLE
template void launch_bj_update_dot_nd<HDGMG_ND>(cudaStream_t, int, const float*, const float*,
                                                float*, float*, float, const float*,
                                                const double*, double*, double*, unsigned*);
#endif
#if HDGMG_REAL_IS_DOUBLE
template void launch_cg_matvec_nd<HDGMG_ND>(cudaStream_t, int, const double*, const float*,
                                            const double*, const double*, double*, double*,
                                            double*, unsigned*);
#endif
#else
template void launch_matvec_bf16_nd<HDGMG_ND, false>(cudaStream_t, int, const __nv_bfloat16*,
                                                     const float*, float*, float, const float*, int);
template void launch_matvec_bf16_nd<HDGMG_ND, true>(cudaStream_t, int, const __nv_bfloat16*,
                                                    const float*, float*, float, const float*, int);
#endif
}  // namespace hdgmg
