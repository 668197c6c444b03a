// Instantiations of the register-resident Jacobi kernel in values mode with the rotation log
// (cluster variants; the log is replayed onto W by replay.cu).
#include "jacobi_variants.cuh"

namespace lfa {
LFA_DEFINE_JACOBI_DISPATCH(jacobi_val_log, log, log)
}  // namespace lfa
