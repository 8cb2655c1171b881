// Device helpers shared by the event path and the soft-count surrogate of libevis.
#pragma once

#include <cuda_runtime.h>

namespace evis {

// A source splats iff its depth is finite and > 0.
__device__ __forceinline__ bool valid_depth(float z) { return z > 0.0f && z < INFINITY; }

// Depth of the other keyframe at the correspondence endpoint (Eq. 7): nearest pixel with
// halves rounded up, else the source's own depth (outside the image or invalid there).
__device__ __forceinline__ float other_depth(const float *__restrict__ Zo, int W, int H,
                                             float ux, float uy, float own) {
  const float nx = floorf(__fadd_rn(ux, 0.5f)), ny = floorf(__fadd_rn(uy, 0.5f));
  if (!(nx >= 0.0f && nx <= static_cast<float>(W - 1) && ny >= 0.0f &&
        ny <= static_cast<float>(H - 1)))
    return own;
  const float z = __ldg(Zo + static_cast<int>(ny) * W + static_cast<int>(nx));
  return valid_depth(z) ? z : own;
}

}  // namespace evis
