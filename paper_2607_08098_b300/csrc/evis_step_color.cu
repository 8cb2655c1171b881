// Explicit instantiations of the synthesis kernel: colour events (three channels, with the
// statistics code), every tile shape.
#include "evis_step.cuh"

namespace evis {

template cudaError_t launch_shape<32, 8, false, true, 3, true>(const StepArgs &, int, int, cudaStream_t);
template cudaError_t launch_shape<32, 16, false, true, 3, true>(const StepArgs &, int, int, cudaStream_t);
template cudaError_t launch_shape<32, 32, false, true, 3, true>(const StepArgs &, int, int, cudaStream_t);
template cudaError_t launch_shape<64, 16, false, true, 3, true>(const StepArgs &, int, int, cudaStream_t);
template cudaError_t launch_shape<64, 32, false, true, 3, true>(const StepArgs &, int, int, cudaStream_t);
template cudaError_t launch_shape<128, 16, false, true, 3, true>(const StepArgs &, int, int, cudaStream_t);

}  // namespace evis
