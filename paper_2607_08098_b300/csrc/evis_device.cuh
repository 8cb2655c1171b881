// Device helpers shared by the kernels of libevis (event path, preparation, surrogate).
#pragma once

#include <cfloat>

#include <cuda_runtime.h>

namespace evis {

constexpr unsigned kFull = 0xFFFFFFFFu;  // all lanes of a warp

// L = log(I + eps), Sec. 3.2; non-positive or NaN arguments clamp to the smallest normal.
__device__ __forceinline__ float log_intensity(float I, float eps) {
  float s = __fadd_rn(I, eps);
  if (!(s > 0.0f)) s = FLT_MIN;
  return logf(s);
}

// Rec. 709 luminance, Eq. 3: ((0.2126 R + 0.7152 G) + 0.0722 B), each product rounded.
__device__ __forceinline__ float rec709(float R, float G, float B) {
  return __fadd_rn(__fadd_rn(__fmul_rn(0.2126f, R), __fmul_rn(0.7152f, G)),
                   __fmul_rn(0.0722f, B));
}

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
