// Explicit instantiations of the synthesis kernel: production variants without the statistics
// code, every tile shape, and the unpacked 64x16 variant of the allocation-free entry point.
#include "evis_step.cuh"

namespace evis {

template cudaError_t launch_shape<32, 8, false, true, 1, false>(const StepArgs &, int, int, cudaStream_t);
template cudaError_t launch_shape<32, 16, false, true, 1, false>(const StepArgs &, int, int, cudaStream_t);
template cudaError_t launch_shape<32, 32, false, true, 1, false>(const StepArgs &, int, int, cudaStream_t);
template cudaError_t launch_shape<64, 16, false, true, 1, false>(const StepArgs &, int, int, cudaStream_t);
template cudaError_t launch_shape<64, 32, false, true, 1, false>(const StepArgs &, int, int, cudaStream_t);
template cudaError_t launch_shape<128, 16, false, true, 1, false>(const StepArgs &, int, int, cudaStream_t);
template cudaError_t launch_shape<64, 16, false, false, 1, false>(const StepArgs &, int, int, cudaStream_t);

}  // namespace evis
