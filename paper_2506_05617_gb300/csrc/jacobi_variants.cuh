// Register-resident Jacobi variants: (pairs NP, lanes per pair L, X rows per lane MR,
// W rows per lane WR). A variant serves symbols with M <= MR*L rows and
// N <= min(2*NP, WR*L) columns (X = A_k or A_k^*, N = r = min(c_out, c_in)).
#pragma once
#include "jacobi.cuh"

// X(id, NP, L, MR, WR)
#define LFA_JACOBI_VARIANTS(X) \
  X(0, 2, 4, 2, 1)             \
  X(1, 2, 8, 8, 1)             \
  X(2, 4, 4, 4, 2)             \
  X(3, 4, 8, 8, 1)             \
  X(4, 8, 4, 8, 4)             \
  X(5, 8, 8, 8, 2)             \
  X(6, 16, 8, 4, 4)            \
  X(7, 16, 8, 8, 4)            \
  X(8, 32, 8, 8, 8)            \
  X(9, 32, 4, 16, 16)

namespace lfa {

template <int NP, int L, int MR, int WR, bool VEC, bool FUSED>
cudaError_t jacobi_launch_t(const JacobiLaunch& P, int grid, cudaStream_t s) {
  using C = JCfg<NP, L, MR, WR, VEC>;
  jacobi_kernel<C, FUSED><<<grid, C::BLOCK, C::SMEM, s>>>(P);
  return cudaGetLastError();
}

template <int NP, int L, int MR, int WR, bool VEC, bool FUSED>
cudaError_t jacobi_prepare_t() {
  using C = JCfg<NP, L, MR, WR, VEC>;
  return cudaFuncSetAttribute(jacobi_kernel<C, FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)C::SMEM);
}

template <int NP, int L, int MR, int WR, bool VEC, bool FUSED>
cudaError_t jacobi_occupancy_t(int* blocks) {
  using C = JCfg<NP, L, MR, WR, VEC>;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, jacobi_kernel<C, FUSED>, C::BLOCK,
                                                       C::SMEM);
}

// Per-translation-unit dispatch over the variant list for one (VEC, FUSED) pair.
#define LFA_DEFINE_JACOBI_DISPATCH(NAME, VEC, FUSED)                                        \
  cudaError_t NAME##_launch(int id, const JacobiLaunch& P, int grid, cudaStream_t s) {    \
    switch (id) {                                                                          \
      LFA_JACOBI_VARIANTS(LFA_CASE_LAUNCH_##VEC##_##FUSED)                                 \
      default: return cudaErrorInvalidValue;                                               \
    }                                                                                      \
  }                                                                                        \
  cudaError_t NAME##_prepare(int id) {                                                     \
    switch (id) {                                                                          \
      LFA_JACOBI_VARIANTS(LFA_CASE_PREPARE_##VEC##_##FUSED)                                \
      default: return cudaErrorInvalidValue;                                               \
    }                                                                                      \
  }                                                                                        \
  cudaError_t NAME##_occupancy(int id, int* b) {                                           \
    switch (id) {                                                                          \
      LFA_JACOBI_VARIANTS(LFA_CASE_OCC_##VEC##_##FUSED)                                    \
      default: return cudaErrorInvalidValue;                                               \
    }                                                                                      \
  }

#define LFA_CASE_LAUNCH_true_true(id, NP, L, MR, WR) case id: return jacobi_launch_t<NP, L, MR, WR, true, true>(P, grid, s);
#define LFA_CASE_LAUNCH_false_true(id, NP, L, MR, WR) case id: return jacobi_launch_t<NP, L, MR, WR, false, true>(P, grid, s);
#define LFA_CASE_LAUNCH_false_false(id, NP, L, MR, WR) case id: return jacobi_launch_t<NP, L, MR, WR, false, false>(P, grid, s);
#define LFA_CASE_PREPARE_true_true(id, NP, L, MR, WR) case id: return jacobi_prepare_t<NP, L, MR, WR, true, true>();
#define LFA_CASE_PREPARE_false_true(id, NP, L, MR, WR) case id: return jacobi_prepare_t<NP, L, MR, WR, false, true>();
#define LFA_CASE_PREPARE_false_false(id, NP, L, MR, WR) case id: return jacobi_prepare_t<NP, L, MR, WR, false, false>();
#define LFA_CASE_OCC_true_true(id, NP, L, MR, WR) case id: return jacobi_occupancy_t<NP, L, MR, WR, true, true>(b);
#define LFA_CASE_OCC_false_true(id, NP, L, MR, WR) case id: return jacobi_occupancy_t<NP, L, MR, WR, false, true>(b);
#define LFA_CASE_OCC_false_false(id, NP, L, MR, WR) case id: return jacobi_occupancy_t<NP, L, MR, WR, false, false>(b);

cudaError_t jacobi_vec_fused_launch(int id, const JacobiLaunch& P, int grid, cudaStream_t s);
cudaError_t jacobi_vec_fused_prepare(int id);
cudaError_t jacobi_vec_fused_occupancy(int id, int* b);
cudaError_t jacobi_val_fused_launch(int id, const JacobiLaunch& P, int grid, cudaStream_t s);
cudaError_t jacobi_val_fused_prepare(int id);
cudaError_t jacobi_val_fused_occupancy(int id, int* b);
cudaError_t jacobi_val_plain_launch(int id, const JacobiLaunch& P, int grid, cudaStream_t s);
cudaError_t jacobi_val_plain_prepare(int id);
cudaError_t jacobi_val_plain_occupancy(int id, int* b);

}  // namespace lfa
