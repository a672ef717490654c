// Instantiations of the fused float32 kernels (one per supported embedding size).
#include "kernels.cuh"

namespace fh {
cudaError_t run_fused_any(int F, int which, const FusedArgs& a) {
    switch (F) {
        case 1: return run_fused<1>(which, a);
        case 2: return run_fused<2>(which, a);
        case 4: return run_fused<4>(which, a);
        case 8: return run_fused<8>(which, a);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace fh
