// Instantiations of the register-resident Jacobi kernel: VEC=true, FUSED=true.
#include "jacobi_variants.cuh"

namespace lfa {
LFA_DEFINE_JACOBI_DISPATCH(jacobi_vec_fused, true, true)
}  // namespace lfa
