// Event voxel grid: per environment, polarity and time bin, the events of a segment linearly
// interpolated along time, each bin divided by its largest value (the input of the paper's
// speed regression, appendix).  Weights are 16-bit fixed point so that the sums are exact
// integers, independent of the order in which atomics land.
//
//   voxel_scatter    grid-stride over the event records (count read on the device); each
//                    event adds w_b and w_next to two uint32 accumulators (global atomics).
//   voxel_normalize  one CTA per (environment, polarity, bin) plane: the plane's maximum by
//                    a block reduction, then the normalised floats (the second read of the
//                    plane comes from L2).
#include <algorithm>
#include <string>
#include <vector>

#include "evis_device.cuh"
#include "evis_internal.h"

namespace {

struct VoxelEnvDev {
  int32_t W, H;
  int64_t t0, t1;
  int64_t off;   // first voxel of the environment
};

constexpr int kVoxThreads = 256;
constexpr int kNormUnroll = 8;  // independent loads per thread per pass of voxel_normalize

// q = floor(n / d) and n - q d for n < 2^48 and 0 < d < 2^32 whose quotient is below 2^20,
// without a 64-bit division: a binary32 estimate of the quotient (relative error below
// 2^-22, so off by at most one) corrected with exact integer arithmetic.
__device__ __forceinline__ uint64_t div_small(uint64_t n, uint64_t d, uint64_t *rem) {
  const float qf = floorf(__fdiv_rn(__ull2float_rn(n), __ull2float_rn(d)));
  int64_t q = static_cast<int64_t>(qf);
  int64_t r = static_cast<int64_t>(n) - q * static_cast<int64_t>(d);
  if (r < 0) {
    --q;
    r += static_cast<int64_t>(d);
  }
  if (r < 0) {
    --q;
    r += static_cast<int64_t>(d);
  }
  if (r >= static_cast<int64_t>(d)) {
    ++q;
    r -= static_cast<int64_t>(d);
  }
  if (r >= static_cast<int64_t>(d)) {
    ++q;
    r -= static_cast<int64_t>(d);
  }
  *rem = static_cast<uint64_t>(r);
  return static_cast<uint64_t>(q);
}

__global__ void __launch_bounds__(kVoxThreads) voxel_scatter(const ulonglong2 *__restrict__ ev,
                                                             const uint64_t *count, int64_t max_events,
                                                             const VoxelEnvDev *__restrict__ envs,
                                                             int n_envs, int bins,
                                                             unsigned *__restrict__ acc) {
  int64_t n = max_events;
  if (count) n = min(n, static_cast<int64_t>(min(*count, static_cast<uint64_t>(max_events))));
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < n;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const ulonglong2 r = __ldg(ev + k);
    const int64_t t = static_cast<int64_t>(r.x);
    const int x = static_cast<int>(r.y & 0xFFFFu), y = static_cast<int>((r.y >> 16) & 0xFFFFu);
    const int e = static_cast<int>((r.y >> 32) & 0xFFFFu);
    const int p = static_cast<int16_t>(static_cast<uint16_t>(r.y >> 48));
    if (e >= n_envs || p == 0) continue;
    const VoxelEnvDev E = envs[e];
    if (x >= E.W || y >= E.H || t < E.t0 || t > E.t1) continue;
    const uint64_t D = static_cast<uint64_t>(E.t1 - E.t0);
    const uint64_t N = static_cast<uint64_t>(bins - 1) * static_cast<uint64_t>(t - E.t0);
    uint64_t rem = 0, unused = 0;
    const uint64_t b = div_small(N, D, &rem);                           // b <= bins - 1
    const unsigned w_next = static_cast<unsigned>(div_small(rem << 16, D, &unused));  // < 2^16
    const int64_t plane = static_cast<int64_t>(E.W) * E.H;
    const int64_t base = E.off + (static_cast<int64_t>(p > 0 ? 0 : 1) * bins + static_cast<int64_t>(b)) * plane +
                         static_cast<int64_t>(y) * E.W + x;
    atomicAdd(acc + base, 65536u - w_next);
    if (w_next > 0 && static_cast<int64_t>(b) + 1 < bins) atomicAdd(acc + base + plane, w_next);
  }
}

__global__ void __launch_bounds__(kVoxThreads) voxel_normalize(const VoxelEnvDev *__restrict__ envs,
                                                               int bins,
                                                               const unsigned *__restrict__ acc,
                                                               float *__restrict__ out) {
  const int64_t q = blockIdx.x;              // plane: environment q / (2 bins), slot q % (2 bins)
  const int e = static_cast<int>(q / (2 * bins));
  const VoxelEnvDev E = envs[e];
  const int64_t plane = static_cast<int64_t>(E.W) * E.H;
  const int64_t start = E.off + (q - static_cast<int64_t>(e) * 2 * bins) * plane;
  const unsigned *a = acc + start;
  unsigned mx = 0;
  for (int64_t base = threadIdx.x; base < plane; base += kVoxThreads * kNormUnroll) {
    unsigned v[kNormUnroll];
#pragma unroll
    for (int u = 0; u < kNormUnroll; ++u) {
      const int64_t i = base + u * kVoxThreads;
      v[u] = i < plane ? __ldg(a + i) : 0u;
    }
#pragma unroll
    for (int u = 0; u < kNormUnroll; ++u) mx = max(mx, v[u]);
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) mx = max(mx, __shfl_xor_sync(evis::kFull, mx, d));
  __shared__ unsigned s_mx[kVoxThreads / 32];
  if ((threadIdx.x & 31) == 0) s_mx[threadIdx.x >> 5] = mx;
  __syncthreads();
  mx = 0;
  for (int w = 0; w < kVoxThreads / 32; ++w) mx = max(mx, s_mx[w]);
  float *o = out + start;
  const float fm = __uint2float_rn(mx);
  for (int64_t base = threadIdx.x; base < plane; base += kVoxThreads * kNormUnroll) {
    unsigned v[kNormUnroll];
#pragma unroll
    for (int u = 0; u < kNormUnroll; ++u) {
      const int64_t i = base + u * kVoxThreads;
      v[u] = i < plane ? a[i] : 0u;   // the plane was just read: mostly L2 hits
    }
#pragma unroll
    for (int u = 0; u < kNormUnroll; ++u) {
      const int64_t i = base + u * kVoxThreads;
      if (i < plane) o[i] = mx ? __fdiv_rn(__uint2float_rn(v[u]), fm) : 0.0f;
    }
  }
}

constexpr size_t kTableAlign = 256;

std::string check(const evis_voxel_env *envs, int32_t n_envs, int32_t bins, int64_t *voxels) {
  if (!envs) return "envs is null";
  if (n_envs < 1 || n_envs > 65535) return "n_envs must be in 1..65535";
  if (bins < 1 || bins > 1024) return "bins must be in 1..1024";
  int64_t v = 0;
  for (int i = 0; i < n_envs; ++i) {
    const evis_voxel_env &d = envs[i];
    if (d.width < 1 || d.height < 1 || d.width > 65535 || d.height > 65535 ||
        int64_t(d.width) * d.height > (int64_t(1) << 24))
      return "sensor sizes must be in 1..65535 with width*height <= 2^24";
    if (!(d.t1_ns > d.t0_ns) || d.t1_ns - d.t0_ns >= (int64_t(1) << 32))
      return "each segment needs 0 < t1_ns - t0_ns < 2^32";
    v += 2LL * bins * d.width * d.height;
  }
  *voxels = v;
  return "";
}

size_t table_bytes(int32_t n_envs) {
  return (sizeof(VoxelEnvDev) * n_envs + kTableAlign - 1) / kTableAlign * kTableAlign;
}

}  // namespace

extern "C" evis_status evis_voxel_workspace_size(const evis_voxel_env *envs, int32_t n_envs,
                                                 int32_t bins, int64_t *bytes) {
  int64_t voxels = 0;
  if (!bytes || !check(envs, n_envs, bins, &voxels).empty()) return EVIS_ERR_INVALID_ARG;
  *bytes = static_cast<int64_t>(table_bytes(n_envs)) + voxels * static_cast<int64_t>(sizeof(unsigned));
  return EVIS_OK;
}

extern "C" evis_status evis_voxel_grid(const evis_event *events, const uint64_t *count,
                                       int64_t max_events, const evis_voxel_env *envs,
                                       int32_t n_envs, int32_t bins, void *workspace,
                                       int64_t workspace_bytes, float *grid,
                                       evis_stream_t stream) {
  auto reject = [](const std::string &why) {
    evis::set_detached_error("evis_voxel_grid: " + why);
    return EVIS_ERR_INVALID_ARG;
  };
  int64_t voxels = 0;
  const std::string why = check(envs, n_envs, bins, &voxels);
  if (!why.empty()) return reject(why);
  if (max_events < 0 || (max_events > 0 && !events)) return reject("events is null");
  if (!workspace || !grid) return reject("null workspace or grid");
  const int64_t need = static_cast<int64_t>(table_bytes(n_envs)) + voxels * static_cast<int64_t>(sizeof(unsigned));
  if (workspace_bytes < need) return reject("workspace smaller than evis_voxel_workspace_size");
  std::vector<VoxelEnvDev> tab(n_envs);
  int64_t off = 0;
  for (int i = 0; i < n_envs; ++i) {
    tab[i] = VoxelEnvDev{envs[i].width, envs[i].height, envs[i].t0_ns, envs[i].t1_ns, off};
    off += 2LL * bins * envs[i].width * envs[i].height;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned char *ws = static_cast<unsigned char *>(workspace);
  VoxelEnvDev *d_tab = reinterpret_cast<VoxelEnvDev *>(ws);
  unsigned *acc = reinterpret_cast<unsigned *>(ws + table_bytes(n_envs));
  cudaError_t e;
  // pageable source: the copy is staged before the call returns, so tab may go away
  if ((e = cudaMemcpyAsync(d_tab, tab.data(), sizeof(VoxelEnvDev) * n_envs, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemsetAsync(acc, 0, sizeof(unsigned) * voxels, s)))
    goto fail;
  if (max_events > 0) {
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
      goto fail;
    const int64_t want = (max_events + kVoxThreads - 1) / kVoxThreads;
    const int blocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(want, 16LL * sms)));
    voxel_scatter<<<blocks, kVoxThreads, 0, s>>>(reinterpret_cast<const ulonglong2 *>(events), count,
                                                 max_events, d_tab, n_envs, bins, acc);
    if ((e = cudaGetLastError()) != cudaSuccess) goto fail;
  }
  voxel_normalize<<<static_cast<unsigned>(2LL * bins * n_envs), kVoxThreads, 0, s>>>(d_tab, bins, acc, grid);
  if ((e = cudaGetLastError()) != cudaSuccess) goto fail;
  return EVIS_OK;
fail:
  evis::set_detached_error(std::string("evis_voxel_grid: ") + cudaGetErrorString(e));
  return EVIS_ERR_CUDA;
}
