// Instantiations of the register-resident Jacobi kernel: VEC=false, FUSED=false.
#include "jacobi_variants.cuh"

namespace lfa {
LFA_DEFINE_JACOBI_DISPATCH(jacobi_val_plain, false, false)
}  // namespace lfa
