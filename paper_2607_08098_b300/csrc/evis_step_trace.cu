// Explicit instantiations of the synthesis kernel: debug-trace variants (with the statistics
// code), every tile shape.
#include "evis_step.cuh"

namespace evis {

template cudaError_t launch_shape<32, 8, true, true, 1, true>(const StepArgs &, int, int, cudaStream_t);
template cudaError_t launch_shape<32, 16, true, true, 1, true>(const StepArgs &, int, int, cudaStream_t);
template cudaError_t launch_shape<32, 32, true, true, 1, true>(const StepArgs &, int, int, cudaStream_t);
template cudaError_t launch_shape<64, 16, true, true, 1, true>(const StepArgs &, int, int, cudaStream_t);
template cudaError_t launch_shape<64, 32, true, true, 1, true>(const StepArgs &, int, int, cudaStream_t);
template cudaError_t launch_shape<128, 16, true, true, 1, true>(const StepArgs &, int, int, cudaStream_t);

}  // namespace evis
