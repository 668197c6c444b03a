// Instantiations of the register-resident Jacobi kernel: VEC=false, FUSED=true.
#include "jacobi_variants.cuh"

namespace lfa {
LFA_DEFINE_JACOBI_DISPATCH(jacobi_val_fused, false, true)
}  // namespace lfa
