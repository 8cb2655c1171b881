// CUDA kernels of the EVIS event-synthesis path (sm_103a).
//
// Compiled with -fmad=false and written with explicit round-to-nearest intrinsics so that
// every floating-point step that decides a z-buffer winner or an event count is the same
// single IEEE-754 binary32 operation, in the same order, as in the method's definition:
// splat winners, event counts, pixels and polarities are then reproducible bit for bit on
// any IEEE host.
//
// Kernels here (the synthesis kernel itself is in evis_step.cuh)
//   prep_kernel  per keyframe: log-intensity (Sec. 3.2, Eq. 3), optional copies of the
//                motion/depth maps, per-environment max |mv| and per 32-pixel row segment
//                motion bounds (which sources can reach which tile).
//   defocus_kernel, log_kernel, init_ref_kernel: the per-keyframe stages around it.
#include <cuda_fp16.h>

#include <atomic>

#include "evis_device.cuh"
#include "evis_internal.h"

namespace evis {
namespace {

// One warp per 32-pixel row segment: log-intensity, optional copies, and the segment's
// motion bounds over the sources that can splat (valid depth, finite motion).
__global__ void __launch_bounds__(256, 8) prep_kernel(const PrepArgs a) {
  const int e = blockIdx.y;
  const DevEnv E = a.envs[e];
  const int nseg = E.segs_x * E.H;
  const int64_t o = E.pix_off;
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  float mx = 0.0f;
  unsigned bad = 0;  // this lane's sources that cannot splat (the statistics)
  for (int sg = blockIdx.x * wpb + (threadIdx.x >> 5); sg < nseg; sg += gridDim.x * wpb) {
    const int y = sg / E.segs_x;
    const int x = (sg - y * E.segs_x) * kSegW + lane;
    float lox = INFINITY, hix = -INFINITY, loy = INFINITY, hiy = -INFINITY;
    if (x < E.W) {
      const int64_t p = o + static_cast<int64_t>(y) * E.W + x;
      const float2 m = reinterpret_cast<const float2 *>(a.mv)[p];
      const float z = a.Z[p];
      if (valid_depth(z) && isfinite(m.x) && isfinite(m.y)) {
        lox = hix = m.x;
        loy = hiy = m.y;
        mx = fmaxf(mx, fmaxf(fabsf(m.x), fabsf(m.y)));
      } else {
        ++bad;
      }
      if (a.mv_out) reinterpret_cast<float2 *>(a.mv_out)[p] = m;
      if (a.Z_out) a.Z_out[p] = z;
      if (a.packA && a.ZA) {
        // the depth at the other endpoint of each source's correspondence (Eq. 7), once per
        // gap: B's sources look up A at p + m_B, A's sources look up B at p - m_A
        const float fx = static_cast<float>(x), fy = static_cast<float>(y);
        const float *ZAe = a.ZA + o, *ZBe = a.Z + o;
        const float zoB = other_depth(ZAe, E.W, E.H, __fadd_rn(fx, m.x), __fadd_rn(fy, m.y), z);
        a.packB[p] = make_float4(m.x, m.y, z, zoB);
        const float2 mA = reinterpret_cast<const float2 *>(a.mvA)[p];
        const float zA = a.ZA[p];
        const float zoA = other_depth(ZBe, E.W, E.H, __fsub_rn(fx, mA.x), __fsub_rn(fy, mA.y), zA);
        a.packA[p] = make_float4(mA.x, mA.y, zA, zoA);
      }
      if (a.L_out) {
        if (a.nc == 3) {  // colour: R, G, B planes
          for (int c = 0; c < 3; ++c) {
            float L;
            if (a.mode == EVIS_IN_LOG) L = a.frames[c * a.plane + p];
            else if (a.mode == EVIS_IN_LUM) L = log_intensity(a.frames[c * a.plane + p], a.eps);
            else L = log_intensity(a.frames[3 * p + c], a.eps);
            a.L_out[c * a.plane + p] = L;
          }
        } else {
          float L;
          if (a.mode == EVIS_IN_LOG) {
            L = a.frames[p];
          } else if (a.mode == EVIS_IN_LUM) {
            L = log_intensity(a.frames[p], a.eps);
          } else {
            const float *c = a.frames + 3 * p;
            L = log_intensity(rec709(c[0], c[1], c[2]), a.eps);
          }
          a.L_out[p] = L;
        }
      }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      lox = fminf(lox, __shfl_xor_sync(kFull, lox, d));
      hix = fmaxf(hix, __shfl_xor_sync(kFull, hix, d));
      loy = fminf(loy, __shfl_xor_sync(kFull, loy, d));
      hiy = fmaxf(hiy, __shfl_xor_sync(kFull, hiy, d));
    }
    if (lane == 0) a.seg[E.seg_off + sg] = make_float4(lox, hix, loy, hiy);
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, d));
  __shared__ float sm[32];
  __shared__ unsigned s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  if (lane == 0) sm[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (a.invalid) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) bad += __shfl_xor_sync(kFull, bad, d);
    if (lane == 0 && bad) atomicAdd(&s_bad, bad);
  }
  __syncthreads();
  if (a.invalid && threadIdx.x == 0 && s_bad) atomicAdd(a.invalid + e, static_cast<unsigned long long>(s_bad));
  if (threadIdx.x < 32) {
    mx = threadIdx.x < wpb ? sm[threadIdx.x] : 0.0f;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, d));
    // non-negative floats order like their bit patterns
    if (threadIdx.x == 0 && mx > 0.0f) atomicMax(reinterpret_cast<int *>(a.flow + e), __float_as_int(mx));
  }
}

// Defocus (Sec. 3.4): separable Gaussian on linear luminance.  One CTA per 64 x 32 output
// tile (blockIdx.x = tile, blockIdx.y = environment, blockIdx.z = channel): the tile and a
// halo of r pixels (edge pixels repeated) are loaded as luminance into shared memory, the
// horizontal pass writes (32 + 2r) x 64 sums, the vertical pass the 64 x 32 outputs.  Each
// sum runs over k = -r..r in order in binary32, as the definition states.  Radii 0..3
// (sigma up to 1.16 px) run unrolled with the weights in registers and a sliding window of
// taps per thread (4 outputs of a row, 8 of a column); larger radii take a plain loop.
constexpr int kBlurTX = 64, kBlurTY = 32, kBlurThreads = 256;

template <int R>
__device__ __forceinline__ void blur_passes(const float *A, float *B, const float *sw, int AW,
                                            float *out, int W, int H, int x0, int y0) {
  constexpr int AH = kBlurTY + 2 * R;
  float w[2 * R + 1];
#pragma unroll
  for (int k = 0; k <= 2 * R; ++k) w[k] = sw[k];
  // horizontal: thread -> one row, four adjacent columns
  for (int i = threadIdx.x; i < AH * (kBlurTX / 4); i += kBlurThreads) {
    const int ry = i / (kBlurTX / 4), c4 = (i % (kBlurTX / 4)) * 4;
    float v[4 + 2 * R];
#pragma unroll
    for (int j = 0; j < 4 + 2 * R; ++j) v[j] = A[ry * AW + c4 + j];
    float4 o4;
    float *o = &o4.x;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float acc = 0.0f;
#pragma unroll
      for (int k = 0; k <= 2 * R; ++k) acc = __fadd_rn(acc, __fmul_rn(w[k], v[q + k]));
      o[q] = acc;
    }
    *reinterpret_cast<float4 *>(B + ry * kBlurTX + c4) = o4;
  }
  __syncthreads();
  // vertical: thread -> one column, eight adjacent rows
  const int cx = threadIdx.x % kBlurTX, r8 = (threadIdx.x / kBlurTX) * 8;
  float v[8 + 2 * R];
#pragma unroll
  for (int j = 0; j < 8 + 2 * R; ++j) v[j] = B[(r8 + j) * kBlurTX + cx];
  const int x = x0 + cx;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k <= 2 * R; ++k) acc = __fadd_rn(acc, __fmul_rn(w[k], v[q + k]));
    const int y = y0 + r8 + q;
    if (x < W && y < H) out[y * W + x] = acc;
  }
}

__device__ __forceinline__ void blur_passes_any(const float *A, float *B, const float *sw, int r,
                                                int AW, float *out, int W, int H, int x0, int y0) {
  const int AH = kBlurTY + 2 * r;
  for (int i = threadIdx.x; i < AH * kBlurTX; i += kBlurThreads) {
    const int ry = i / kBlurTX, cx = i % kBlurTX;
    float acc = 0.0f;
    for (int k = 0; k <= 2 * r; ++k) acc = __fadd_rn(acc, __fmul_rn(sw[k], A[ry * AW + cx + k]));
    B[i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kBlurTY * kBlurTX; i += kBlurThreads) {
    const int row = i / kBlurTX, cx = i % kBlurTX;
    const int x = x0 + cx, y = y0 + row;
    if (x >= W || y >= H) continue;
    float acc = 0.0f;
    for (int k = 0; k <= 2 * r; ++k) acc = __fadd_rn(acc, __fmul_rn(sw[k], B[(row + k) * kBlurTX + cx]));
    out[y * W + x] = acc;
  }
}

__global__ void __launch_bounds__(kBlurThreads) defocus_kernel(const BlurArgs a) {
  extern __shared__ __align__(16) float blur_sm[];
  __shared__ float sw[2 * kMaxBlurR + 1];
  int W, H, r;
  int64_t o = 0;
  if (a.envs) {
    const DevEnv &E = a.envs[blockIdx.y];
    W = E.W;
    H = E.H;
    r = E.blur_r;
    o = E.pix_off;
    for (int i = threadIdx.x; i <= 2 * r; i += blockDim.x) sw[i] = a.wtab[E.blur_off + i];
  } else {
    W = a.W;
    H = a.H;
    r = a.r;
    for (int i = threadIdx.x; i <= 2 * r; i += blockDim.x) sw[i] = a.w[i];
  }
  const int tiles_x = (W + kBlurTX - 1) / kBlurTX;
  const int t = blockIdx.x;
  if (t >= tiles_x * ((H + kBlurTY - 1) / kBlurTY)) return;  // uniform over the CTA
  const int x0 = (t % tiles_x) * kBlurTX, y0 = (t / tiles_x) * kBlurTY;
  const int AW = kBlurTX + 2 * r, AH = kBlurTY + 2 * r;
  float *A = blur_sm;            // [AH][AW] luminance with halo
  float *B = blur_sm + ((AH * AW + 3) & ~3);  // [AH][64] horizontal sums (16-byte aligned)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = kBlurThreads / 32;
  const int ch = a.nc == 3 ? static_cast<int>(blockIdx.z) : 0;
  const float *in = a.in + (a.nc == 3 || a.mode == EVIS_IN_RGB ? 3 * o : o);  // this environment
  const int stride = (a.nc == 3 || a.mode == EVIS_IN_RGB) ? 3 : 1;
  const bool lum = a.nc != 3 && a.mode == EVIS_IN_RGB;
  // loads in batches of two rows per warp, every column chunk of a row issued before the
  // first shared-memory store (AW <= 64 + 2 kMaxBlurR <= 128: four chunks)
  static_assert(kBlurTX + 2 * kMaxBlurR <= 4 * 32, "four column chunks cover a halo row");
  for (int ry0 = warp; ry0 < AH; ry0 += 2 * NW) {
    float v[2][4];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int ry = ry0 + q * NW;
      const int row = min(max(y0 - r + ry, 0), H - 1) * W;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int rx = lane + 32 * m;
        v[q][m] = 0.0f;
        if (ry < AH && rx < AW) {
          const int p = (row + min(max(x0 - r + rx, 0), W - 1)) * stride;
          v[q][m] = lum ? rec709(__ldg(in + p), __ldg(in + p + 1), __ldg(in + p + 2)) : __ldg(in + p + ch);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int ry = ry0 + q * NW;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int rx = lane + 32 * m;
        if (ry < AH && rx < AW) A[ry * AW + rx] = v[q][m];
      }
    }
  }
  __syncthreads();
  float *out = a.out + static_cast<int64_t>(blockIdx.z) * a.plane + o;
  switch (r) {
    case 0: blur_passes<0>(A, B, sw, AW, out, W, H, x0, y0); break;
    case 1: blur_passes<1>(A, B, sw, AW, out, W, H, x0, y0); break;
    case 2: blur_passes<2>(A, B, sw, AW, out, W, H, x0, y0); break;
    case 3: blur_passes<3>(A, B, sw, AW, out, W, H, x0, y0); break;
    default: blur_passes_any(A, B, sw, r, AW, out, W, H, x0, y0);
  }
}

__global__ void init_ref_kernel(const float *__restrict__ L, float *__restrict__ Lref, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    Lref[i] = L[i];
}

__global__ void log_kernel(const float *__restrict__ in, int64_t n, uint32_t mode, float eps,
                           float *__restrict__ out) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    out[i] = mode == EVIS_IN_RGB ? log_intensity(rec709(in[3 * i], in[3 * i + 1], in[3 * i + 2]), eps)
                                 : log_intensity(in[i], eps);
  }
}

int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 148 * 64) b = 148 * 64;
  return static_cast<int>(b);
}

}  // namespace

cudaError_t launch_prep(const PrepArgs &a, int n_envs, cudaStream_t s) {
  const int threads = 256;
  int bx = (a.max_segs + 4 * (threads / 32) - 1) / (4 * (threads / 32));
  if (bx < 1) bx = 1;
  prep_kernel<<<dim3(bx, n_envs), threads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_defocus(const BlurArgs &a, int n_envs, int max_tiles, cudaStream_t s) {
  if (a.max_r < 0 || a.max_r > kMaxBlurR || n_envs < 1 || max_tiles < 1) return cudaErrorInvalidValue;
  const int R = a.max_r;
  const size_t smem = sizeof(float) * (static_cast<size_t>(kBlurTY + 2 * R) * (kBlurTX + 2 * R + kBlurTX) + 4);
  // up to 56 KB of shared memory at the largest radius, allowed once per device (the
  // attribute belongs to the device's context)
  constexpr int kMaxDevices = 64;
  static std::atomic<bool> attr[kMaxDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (!attr[dev].load(std::memory_order_relaxed)) {
    e = cudaFuncSetAttribute(defocus_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(sizeof(float) * ((kBlurTY + 2 * kMaxBlurR) *
                                              (2 * kBlurTX + 2 * kMaxBlurR) + 4)));
    if (e != cudaSuccess) return e;
    attr[dev].store(true, std::memory_order_relaxed);
  }
  defocus_kernel<<<dim3(max_tiles, n_envs, a.nc == 3 ? 3 : 1), kBlurThreads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_init_ref(const float *L, float *Lref, int64_t n, cudaStream_t s) {
  init_ref_kernel<<<grid_for(n, 256), 256, 0, s>>>(L, Lref, n);
  return cudaGetLastError();
}

cudaError_t launch_log(const float *in, int64_t n, uint32_t mode, float eps, float *out,
                       cudaStream_t s) {
  if (n > 0) log_kernel<<<grid_for(n, 256), 256, 0, s>>>(in, n, mode, eps, out);
  return cudaGetLastError();
}

bool tile_shape_supported(int tw, int th) {
  return (tw == 32 && (th == 8 || th == 16 || th == 32)) || (tw == 64 && (th == 16 || th == 32)) ||
         (tw == 128 && th == 16);
}

cudaError_t launch_step(const StepArgs &a, int tile_w, int tile_h, bool trace, int grid_cap,
                        cudaStream_t s) {
  const int n_tiles = a.n_tiles;
  if (n_tiles <= 0) return cudaSuccess;
  if (!a.packA) {  // unpacked sources: 64x16 tiles only
    if (tile_w != 64 || tile_h != 16 || trace) return cudaErrorInvalidValue;
    if (a.nc == 3) return cudaErrorInvalidValue;
    return launch_shape<64, 16, false, false, 1, false>(a, n_tiles, grid_cap, s);
  }
  // the trace and colour variants always carry the statistics code; the mono production one
  // only when asked
#define EVIS_SHAPE(TX, TY)                                                                      \
  if (tile_w == TX && tile_h == TY)                                                             \
    return a.nc == 3 ? (trace ? launch_shape<TX, TY, true, true, 3, true>(a, n_tiles, grid_cap, s)  \
                              : launch_shape<TX, TY, false, true, 3, true>(a, n_tiles, grid_cap, s)) \
                     : (trace ? launch_shape<TX, TY, true, true, 1, true>(a, n_tiles, grid_cap, s)   \
                              : (a.stats ? launch_shape<TX, TY, false, true, 1, true>(a, n_tiles, grid_cap, s) \
                                         : launch_shape<TX, TY, false, true, 1, false>(a, n_tiles, grid_cap, s)));
  EVIS_SHAPE(32, 8)
  EVIS_SHAPE(32, 16)
  EVIS_SHAPE(32, 32)
  EVIS_SHAPE(64, 16)
  EVIS_SHAPE(64, 32)
  EVIS_SHAPE(128, 16)
#undef EVIS_SHAPE
  return cudaErrorInvalidValue;
}

}  // namespace evis
