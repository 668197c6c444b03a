// Register-resident Jacobi variants: (pairs NP, lanes per pair L, X rows per lane MR,
// W rows per lane WR, CTAs per cluster CS, vectors supported). A variant serves symbols
// with M <= MR*L rows and N <= 2*NP columns (with vectors also N <= WR*L), where
// X = A_k or A_k^* and N = r = min(c_out, c_in). Variants with CS > 1 spread one symbol
// over a thread-block cluster; vectors are instantiated only where they fit registers.
#pragma once
#include "jacobi.cuh"

// X(id, NP, L, MR, WR, CS, VEC_OK, MINB, PPT)  MINB: CTAs per SM the register allocation
// targets; PPT: teams per thread (2: a thread interleaves the rounds of two column pairs)
#define LFA_JACOBI_VARIANTS(X)        \
  X(0, 2, 4, 2, 1, 1, 1, 1, 1)        \
  X(1, 2, 8, 8, 1, 1, 1, 1, 1)        \
  X(2, 4, 4, 4, 2, 1, 1, 1, 1)        \
  X(3, 4, 8, 8, 1, 1, 1, 1, 1)        \
  X(4, 8, 4, 8, 4, 1, 1, 1, 1)        \
  X(5, 8, 8, 8, 2, 1, 1, 1, 1)        \
  X(6, 16, 8, 4, 4, 1, 1, 1, 1)       \
  X(7, 16, 8, 8, 4, 1, 1, 1, 1)       \
  X(8, 32, 8, 8, 8, 1, 1, 1, 1)       \
  X(9, 32, 4, 16, 16, 1, 1, 1, 1)     \
  X(10, 32, 16, 8, 4, 1, 1, 1, 1)     \
  X(11, 64, 16, 8, 8, 2, 1, 1, 1)     \
  X(12, 64, 16, 8, 8, 1, 0, 1, 1)     \
  X(13, 64, 32, 8, 4, 4, 1, 1, 1)     \
  X(14, 128, 32, 8, 8, 8, 1, 1, 1)    \
  X(15, 128, 32, 16, 8, 8, 0, 1, 1)   \
  X(16, 256, 32, 16, 16, 16, 0, 1, 1) \
  X(17, 32, 16, 4, 4, 1, 1, 2, 1)     \
  X(18, 16, 16, 4, 2, 1, 1, 2, 1)     \
  X(19, 128, 32, 8, 8, 8, 1, 1, 2)    \
  X(20, 256, 32, 16, 16, 16, 0, 1, 2)

namespace lfa {

template <int NP, int L, int MR, int WR, int CS, int MB, int PPT, bool VEC, bool FUSED, bool LOG = false>
cudaError_t jacobi_launch_t(const JacobiLaunch& P, int grid, cudaStream_t s) {
  using C = JCfg<NP, L, MR, WR, VEC, CS, MB, PPT>;
  if constexpr (CS == 1) {
    jacobi_kernel<C, FUSED, LOG><<<grid, C::BLOCK, C::SMEM, s>>>(P);
    return cudaGetLastError();
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3(C::BLOCK, 1, 1);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, jacobi_kernel<C, FUSED, LOG>, P);
  }
}

template <int NP, int L, int MR, int WR, int CS, int MB, int PPT, bool VEC, bool FUSED, bool LOG = false>
cudaError_t jacobi_prepare_t() {
  using C = JCfg<NP, L, MR, WR, VEC, CS, MB, PPT>;
  cudaError_t e = cudaFuncSetAttribute(jacobi_kernel<C, FUSED, LOG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)C::SMEM);
  if (e == cudaSuccess && CS > 8)
    e = cudaFuncSetAttribute(jacobi_kernel<C, FUSED, LOG>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

// Largest grid (in CTAs) that is fully co-resident: blocks per SM x SMs, or clusters x CS.
template <int NP, int L, int MR, int WR, int CS, int MB, int PPT, bool VEC, bool FUSED, bool LOG = false>
cudaError_t jacobi_grid_t(int sms, int* grid) {
  using C = JCfg<NP, L, MR, WR, VEC, CS, MB, PPT>;
  if constexpr (CS == 1) {
    int b = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, jacobi_kernel<C, FUSED, LOG>, C::BLOCK, C::SMEM);
    *grid = b * sms;
    return e;
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(CS * 64), 1, 1);
    cfg.blockDim = dim3(C::BLOCK, 1, 1);
    cfg.dynamicSmemBytes = C::SMEM;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&nc, jacobi_kernel<C, FUSED, LOG>, &cfg);
    *grid = nc * CS;
    return e;
  }
}

#define LFA_DEFINE_JACOBI_DISPATCH(NAME, VEC, FUSED)                                         \
  cudaError_t NAME##_launch(int id, const JacobiLaunch& P, int grid, cudaStream_t s) {     \
    switch (id) {                                                                           \
      LFA_JACOBI_VARIANTS(LFA_CASE_LAUNCH_##VEC##_##FUSED)                                  \
      default: return cudaErrorInvalidValue;                                                \
    }                                                                                       \
  }                                                                                         \
  cudaError_t NAME##_prepare(int id) {                                                      \
    switch (id) {                                                                           \
      LFA_JACOBI_VARIANTS(LFA_CASE_PREPARE_##VEC##_##FUSED)                                 \
      default: return cudaErrorInvalidValue;                                                \
    }                                                                                       \
  }                                                                                         \
  cudaError_t NAME##_grid(int id, int sms, int* g) {                                        \
    switch (id) {                                                                           \
      LFA_JACOBI_VARIANTS(LFA_CASE_GRID_##VEC##_##FUSED)                                    \
      default: return cudaErrorInvalidValue;                                                \
    }                                                                                       \
  }

// values-only instantiations exist for every variant; vector ones only where VEC_OK
#define LFA_CASE_LAUNCH_false_true(id, NP, L, MR, WR, CS, OK, MB, PPT) \
  case id: return jacobi_launch_t<NP, L, MR, WR, CS, MB, PPT, false, true>(P, grid, s);
#define LFA_CASE_LAUNCH_false_false(id, NP, L, MR, WR, CS, OK, MB, PPT) \
  case id: return jacobi_launch_t<NP, L, MR, WR, CS, MB, PPT, false, false>(P, grid, s);
#define LFA_CASE_LAUNCH_true_true(id, NP, L, MR, WR, CS, OK, MB, PPT)                              \
  case id:                                                                                 \
    if constexpr (OK) return jacobi_launch_t<NP, L, MR, WR, CS, MB, PPT, true, true>(P, grid, s); \
    else return cudaErrorInvalidValue;
#define LFA_CASE_PREPARE_false_true(id, NP, L, MR, WR, CS, OK, MB, PPT) \
  case id: return jacobi_prepare_t<NP, L, MR, WR, CS, MB, PPT, false, true>();
#define LFA_CASE_PREPARE_false_false(id, NP, L, MR, WR, CS, OK, MB, PPT) \
  case id: return jacobi_prepare_t<NP, L, MR, WR, CS, MB, PPT, false, false>();
#define LFA_CASE_PREPARE_true_true(id, NP, L, MR, WR, CS, OK, MB, PPT)                    \
  case id:                                                                        \
    if constexpr (OK) return jacobi_prepare_t<NP, L, MR, WR, CS, MB, PPT, true, true>();  \
    else return cudaErrorInvalidValue;
#define LFA_CASE_GRID_false_true(id, NP, L, MR, WR, CS, OK, MB, PPT) \
  case id: return jacobi_grid_t<NP, L, MR, WR, CS, MB, PPT, false, true>(sms, g);
#define LFA_CASE_GRID_false_false(id, NP, L, MR, WR, CS, OK, MB, PPT) \
  case id: return jacobi_grid_t<NP, L, MR, WR, CS, MB, PPT, false, false>(sms, g);
#define LFA_CASE_GRID_true_true(id, NP, L, MR, WR, CS, OK, MB, PPT)                           \
  case id:                                                                            \
    if constexpr (OK) return jacobi_grid_t<NP, L, MR, WR, CS, MB, PPT, true, true>(sms, g);   \
    else return cudaErrorInvalidValue;

// the rotation-logging forward exists for values-mode variants with one symbol per unit
#define LFA_CASE_LAUNCH_log_log(id, NP, L, MR, WR, CS, OK, MB, PPT)                                         \
  case id:                                                                                           \
    if constexpr (PPT == 1 && NP * L / CS >= 32) return jacobi_launch_t<NP, L, MR, WR, CS, MB, PPT, false, true, true>(P, grid, s); \
    else return cudaErrorInvalidValue;
#define LFA_CASE_PREPARE_log_log(id, NP, L, MR, WR, CS, OK, MB, PPT)                              \
  case id:                                                                                 \
    if constexpr (PPT == 1 && NP * L / CS >= 32) return jacobi_prepare_t<NP, L, MR, WR, CS, MB, PPT, false, true, true>(); \
    else return cudaErrorInvalidValue;
#define LFA_CASE_GRID_log_log(id, NP, L, MR, WR, CS, OK, MB, PPT)                                     \
  case id:                                                                                     \
    if constexpr (PPT == 1 && NP * L / CS >= 32) return jacobi_grid_t<NP, L, MR, WR, CS, MB, PPT, false, true, true>(sms, g); \
    else return cudaErrorInvalidValue;

cudaError_t jacobi_val_log_launch(int id, const JacobiLaunch& P, int grid, cudaStream_t s);
cudaError_t jacobi_val_log_prepare(int id);
cudaError_t jacobi_val_log_grid(int id, int sms, int* g);
cudaError_t jacobi_vec_fused_launch(int id, const JacobiLaunch& P, int grid, cudaStream_t s);
cudaError_t jacobi_vec_fused_prepare(int id);
cudaError_t jacobi_vec_fused_grid(int id, int sms, int* g);
cudaError_t jacobi_val_fused_launch(int id, const JacobiLaunch& P, int grid, cudaStream_t s);
cudaError_t jacobi_val_fused_prepare(int id);
cudaError_t jacobi_val_fused_grid(int id, int sms, int* g);
cudaError_t jacobi_val_plain_launch(int id, const JacobiLaunch& P, int grid, cudaStream_t s);
cudaError_t jacobi_val_plain_prepare(int id);
cudaError_t jacobi_val_plain_grid(int id, int sms, int* g);

}  // namespace lfa
