// Event voxel grid: per environment, polarity and time bin, the events of a segment linearly
// interpolated along time, each bin divided by its largest value (the input of the paper's
// speed regression, appendix).  Weights are 16-bit fixed point so that the sums are exact
// integers, independent of the order in which atomics land.
//
//   voxel_scatter    grid-stride over the event records (count read on the device) with
//                    three blocks per SM, so that the events in flight touch a part of the
//                    accumulator that L2 holds, and evict-first loads of the records; each
//                    event adds w_b and w_next to two uint32 accumulators (global atomics).
//                    (8 x 640x480, 128 bins, 130 M events: the whole grid in 3.88 ms with
//                    sixteen blocks per SM, 3.14 ms with three.)
//   voxel_plane_max  chunks of 8192 voxels of every (environment, polarity, bin) plane: a
//                    block reduction, then one atomicMax into the plane's maximum.
//   voxel_divide     the same chunks: each voxel divided by its plane's maximum.
// Both stream the accumulator at full occupancy; one CTA per plane doing both passes had up
// to 1,200 planes in flight, so its second read missed L2.
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
    const ulonglong2 r = __ldcs(ev + k);  // evict-first: the accumulator keeps L2
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

constexpr int kChunk = 8192;    // voxels per CTA and pass: 32 independent loads per thread

// Chunk i of the passes: plane i / cpp (chunks per plane), voxels [k, k + kChunk) of it with
// k = (i % cpp) kChunk (empty for chunks past a smaller plane's end).
struct PlaneChunk {
  int64_t start;   // first voxel of the plane
  int k, n;        // first voxel of the chunk in the plane, voxels in the chunk (<= 0: none)
  int64_t q;       // plane
};

__device__ __forceinline__ PlaneChunk plane_chunk(const VoxelEnvDev *envs, int bins, int cpp,
                                                  int64_t i) {
  PlaneChunk c;
  c.q = i / cpp;
  const int e = static_cast<int>(c.q / (2 * bins));
  const VoxelEnvDev E = envs[e];
  const int plane = E.W * E.H;   // below 2^24
  c.start = E.off + (c.q - static_cast<int64_t>(e) * 2 * bins) * plane;
  c.k = static_cast<int>(i % cpp) * kChunk;
  c.n = min(plane - c.k, kChunk);
  return c;
}

__global__ void __launch_bounds__(kVoxThreads) voxel_plane_max(const VoxelEnvDev *__restrict__ envs,
                                                               int bins, int cpp, int64_t chunks,
                                                               const unsigned *__restrict__ acc,
                                                               unsigned *__restrict__ pmax) {
  __shared__ unsigned s_mx[kVoxThreads / 32];
  for (int64_t ci = blockIdx.x; ci < chunks; ci += gridDim.x) {
    const PlaneChunk c = plane_chunk(envs, bins, cpp, ci);
    if (c.n <= 0) continue;  // uniform over the block
    const unsigned *a = acc + c.start + c.k + threadIdx.x;
    const int n = c.n - static_cast<int>(threadIdx.x);
    unsigned mx = 0;
#pragma unroll
    for (int u = 0; u < kChunk / kVoxThreads; ++u)
      mx = max(mx, u * kVoxThreads < n ? __ldg(a + u * kVoxThreads) : 0u);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) mx = max(mx, __shfl_xor_sync(evis::kFull, mx, d));
    if ((threadIdx.x & 31) == 0) s_mx[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < kVoxThreads / 32; ++w) mx = max(mx, s_mx[w]);
      if (mx) atomicMax(pmax + c.q, mx);
    }
    __syncthreads();  // s_mx is reused by the next chunk
  }
}

__global__ void __launch_bounds__(kVoxThreads) voxel_divide(const VoxelEnvDev *__restrict__ envs,
                                                            int bins, int cpp, int64_t chunks,
                                                            const unsigned *__restrict__ acc,
                                                            const unsigned *__restrict__ pmax,
                                                            float *__restrict__ out) {
  constexpr int kHalf = kChunk / kVoxThreads / 2;  // two rounds of independent loads
  for (int64_t ci = blockIdx.x; ci < chunks; ci += gridDim.x) {
    const PlaneChunk c = plane_chunk(envs, bins, cpp, ci);
    if (c.n <= 0) continue;
    const unsigned mx = pmax[c.q];
    const float fm = __uint2float_rn(mx);
    const int64_t first = c.start + c.k;
    if (c.n == kChunk && (first & 3) == 0) {  // a whole chunk on a 16-byte boundary: vectors
      constexpr int kVec = kChunk / 4 / kVoxThreads;
      const uint4 *a4 = reinterpret_cast<const uint4 *>(acc + first) + threadIdx.x;
      float4 *o4 = reinterpret_cast<float4 *>(out + first) + threadIdx.x;
      uint4 v[kVec];
#pragma unroll
      for (int u = 0; u < kVec; ++u) v[u] = __ldg(a4 + u * kVoxThreads);
#pragma unroll
      for (int u = 0; u < kVec; ++u) {
        float4 r;
        r.x = mx ? __fdiv_rn(__uint2float_rn(v[u].x), fm) : 0.0f;
        r.y = mx ? __fdiv_rn(__uint2float_rn(v[u].y), fm) : 0.0f;
        r.z = mx ? __fdiv_rn(__uint2float_rn(v[u].z), fm) : 0.0f;
        r.w = mx ? __fdiv_rn(__uint2float_rn(v[u].w), fm) : 0.0f;
        o4[u * kVoxThreads] = r;
      }
      continue;
    }
    const unsigned *a = acc + c.start + c.k + threadIdx.x;
    float *o = out + c.start + c.k + threadIdx.x;
    const int n = c.n - static_cast<int>(threadIdx.x);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      unsigned v[kHalf];
#pragma unroll
      for (int u = 0; u < kHalf; ++u) {
        const int j = (h * kHalf + u) * kVoxThreads;
        v[u] = j < n ? __ldg(a + j) : 0u;
      }
#pragma unroll
      for (int u = 0; u < kHalf; ++u) {
        const int j = (h * kHalf + u) * kVoxThreads;
        if (j < n) o[j] = mx ? __fdiv_rn(__uint2float_rn(v[u]), fm) : 0.0f;
      }
    }
  }
}

constexpr size_t kTableAlign = 256;

std::string check(const evis_voxel_env *envs, int32_t n_envs, int32_t bins, int64_t *voxels,
                  int64_t *max_plane = nullptr) {
  if (!envs) return "envs is null";
  if (n_envs < 1 || n_envs > 65535) return "n_envs must be in 1..65535";
  if (bins < 1 || bins > 1024) return "bins must be in 1..1024";
  int64_t v = 0, mp = 0;
  for (int i = 0; i < n_envs; ++i) {
    const evis_voxel_env &d = envs[i];
    if (d.width < 1 || d.height < 1 || d.width > 65535 || d.height > 65535 ||
        int64_t(d.width) * d.height > (int64_t(1) << 24))
      return "sensor sizes must be in 1..65535 with width*height <= 2^24";
    if (!(d.t1_ns > d.t0_ns) || d.t1_ns - d.t0_ns >= (int64_t(1) << 32))
      return "each segment needs 0 < t1_ns - t0_ns < 2^32";
    v += 2LL * bins * d.width * d.height;
    mp = std::max<int64_t>(mp, int64_t(d.width) * d.height);
  }
  *voxels = v;
  if (max_plane) *max_plane = mp;
  return "";
}

size_t table_bytes(int32_t n_envs, int32_t bins) {
  const size_t tab = (sizeof(VoxelEnvDev) * n_envs + kTableAlign - 1) / kTableAlign * kTableAlign;
  const size_t pm = (sizeof(unsigned) * 2 * bins * n_envs + kTableAlign - 1) / kTableAlign * kTableAlign;
  return tab + pm;   // the descriptor table, then the plane maxima
}

}  // namespace

extern "C" evis_status evis_voxel_workspace_size(const evis_voxel_env *envs, int32_t n_envs,
                                                 int32_t bins, int64_t *bytes) {
  int64_t voxels = 0;
  if (!bytes || !check(envs, n_envs, bins, &voxels).empty()) return EVIS_ERR_INVALID_ARG;
  *bytes = static_cast<int64_t>(table_bytes(n_envs, bins)) + voxels * static_cast<int64_t>(sizeof(unsigned));
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
  int64_t voxels = 0, max_plane = 0;
  const std::string why = check(envs, n_envs, bins, &voxels, &max_plane);
  if (!why.empty()) return reject(why);
  if (max_events < 0 || (max_events > 0 && !events)) return reject("events is null");
  if (!workspace || !grid) return reject("null workspace or grid");
  const int64_t need = static_cast<int64_t>(table_bytes(n_envs, bins)) + voxels * static_cast<int64_t>(sizeof(unsigned));
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
  unsigned *pmax = reinterpret_cast<unsigned *>(
      ws + (sizeof(VoxelEnvDev) * n_envs + kTableAlign - 1) / kTableAlign * kTableAlign);
  unsigned *acc = reinterpret_cast<unsigned *>(ws + table_bytes(n_envs, bins));
  const int cpp = static_cast<int>((max_plane + kChunk - 1) / kChunk);   // chunks per plane
  const int64_t planes = 2LL * bins * n_envs;
  cudaError_t e;
  // pageable source: the copy is staged before the call returns, so tab may go away
  if ((e = cudaMemcpyAsync(d_tab, tab.data(), sizeof(VoxelEnvDev) * n_envs, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemsetAsync(pmax, 0, sizeof(unsigned) * planes, s)) ||
      (e = cudaMemsetAsync(acc, 0, sizeof(unsigned) * voxels, s)))
    goto fail;
  if (max_events > 0) {
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
      goto fail;
    const int64_t want = (max_events + kVoxThreads - 1) / kVoxThreads;
    const int blocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(want, 3LL * sms)));
    voxel_scatter<<<blocks, kVoxThreads, 0, s>>>(reinterpret_cast<const ulonglong2 *>(events), count,
                                                 max_events, d_tab, n_envs, bins, acc);
    if ((e = cudaGetLastError()) != cudaSuccess) goto fail;
  }
  {
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
      goto fail;
    const int64_t chunks = planes * cpp;
    const int blocks = static_cast<int>(std::min<int64_t>(chunks, 64LL * sms));
    voxel_plane_max<<<blocks, kVoxThreads, 0, s>>>(d_tab, bins, cpp, chunks, acc, pmax);
    if ((e = cudaGetLastError()) != cudaSuccess) goto fail;
    voxel_divide<<<blocks, kVoxThreads, 0, s>>>(d_tab, bins, cpp, chunks, acc, pmax, grid);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) goto fail;
  return EVIS_OK;
fail:
  evis::set_detached_error(std::string("evis_voxel_grid: ") + cudaGetErrorString(e));
  return EVIS_ERR_CUDA;
}
