// Event voxel grid: per environment, polarity and time bin, the events of a segment linearly
// interpolated along time, each bin divided by its largest value (the input of the paper's
// speed regression, appendix).  Weights are 16-bit fixed point so that the sums are exact
// integers, independent of the order in which they are added.
//
// The grid is built region by region in shared memory, so that its accumulator never goes
// to HBM.  A region is one environment's row segment of kSeg pixels across a group of kGroup
// planes (plane = polarity * bins + bin):
//
//   voxel_count       one pass over the event records (count read on the device): per
//                     region, how many entries its events make (warp-aggregated atomics).
//   voxel_scan_*      exclusive prefix sum of the counts: each region's range of entries.
//   voxel_bucket      a second pass over the records: each event becomes one 32-bit entry
//                     (pixel in the segment, plane in the group, weight) in its region's
//                     range, two where its bins straddle a group boundary.
//   voxel_region<0>   per region: the entries summed in shared memory, the row's maximum of
//                     each plane merged into the plane maxima (atomicMax).
//   voxel_region<1>   per region: the same sums again, divided by the plane maxima and
//                     written to the grid (one 128-byte row per plane and warp).
//
// HBM traffic is two reads of the records, the entries written once and read twice, and the
// grid written once; a dense accumulator also clears, read-modify-writes and twice reads 4
// bytes per voxel.
#include <algorithm>
#include <string>
#include <vector>

#include "evis_device.cuh"
#include "evis_internal.h"

namespace {

constexpr int kSeg = 32;       // pixels of a region's row segment (one warp's row of a plane)
constexpr int kGroup = 256;    // planes of a region
constexpr int kVoxThreads = 256;

struct VoxelEnvDev {
  int32_t W, H;
  int64_t t0, t1;
  uint64_t D;         // t1 - t0
  uint64_t inv;       // floor((2^64 - 1) / D)
  int64_t vox_off;    // first voxel of the environment in the grid
  int32_t reg_off;    // first region of the environment (fewer than 2^31 regions)
  int32_t nseg;       // row segments per row
  int32_t plane_off;  // first plane of the environment in the plane maxima
};
static_assert(sizeof(VoxelEnvDev) % 16 == 0, "descriptors are copied as 16-byte words");

// An entry: bits 0-15 w_next, 16-20 the pixel in the segment, 21-28 the plane in the group,
// 29-30 the kind: kFirst adds 2^16 - w_next to the plane, kPair also w_next to the next plane,
// kSecond adds w_next to the plane.
enum : unsigned { kFirst = 0, kPair = 1, kSecond = 2 };

__device__ __forceinline__ unsigned entry(unsigned kind, int pl, int px, unsigned w) {
  return (kind << 29) | (static_cast<unsigned>(pl) << 21) | (static_cast<unsigned>(px) << 16) | w;
}

// The entries of one record: region and word of the first, and of a second where the two
// bins fall in different plane groups (r2 < 0: none).  r1 < 0: the record is skipped.
struct RecordEntries {
  int r1, r2;
  unsigned e1, e2;
};

// FULL = false: only r1, for calls whose planes form one group (bins <= 128), where the
// region does not depend on the time bin.
template <bool FULL>
__device__ __forceinline__ RecordEntries record_entries(const ulonglong2 rec,
                                                        const VoxelEnvDev *__restrict__ envs,
                                                        int n_envs, int bins) {
  RecordEntries o{-1, -1, 0u, 0u};
  const int64_t t = static_cast<int64_t>(rec.x);
  const int x = static_cast<int>(rec.y & 0xFFFFu), y = static_cast<int>((rec.y >> 16) & 0xFFFFu);
  const int e = static_cast<int>((rec.y >> 32) & 0xFFFFu);
  const int p = static_cast<int16_t>(static_cast<uint16_t>(rec.y >> 48));
  if (e >= n_envs || p == 0) return o;
  const VoxelEnvDev E = envs[e];
  if (x >= E.W || y >= E.H || t < E.t0 || t > E.t1) return o;
  if (!FULL) {
    o.r1 = E.reg_off + y * E.nseg + x / kSeg;
    return o;
  }
  // Q = floor(N 2^16 / D) with N = (bins - 1)(t - t0) < 2^42: b = Q >> 16 and
  // w_next = Q mod 2^16 (= floor((N mod D) 2^16 / D)).  A 64-bit reciprocal gives Q or
  // Q - 1 (its error times X < 2^58 stays below 2^-5); one remainder test corrects it.
  const uint64_t X = (static_cast<uint64_t>(bins - 1) * static_cast<uint64_t>(t - E.t0)) << 16;
  uint64_t Q = __umul64hi(X, E.inv);
  if (X - Q * E.D >= E.D) ++Q;
  const int b = static_cast<int>(Q >> 16);
  const unsigned w = static_cast<unsigned>(Q & 0xFFFFu);
  const int plane = (p > 0 ? 0 : bins) + b;
  const int g = plane / kGroup, pl = plane - g * kGroup;
  const int px = x % kSeg;
  o.r1 = E.reg_off + (g * E.H + y) * E.nseg + x / kSeg;
  const bool next = w > 0 && b + 1 < bins;
  if (!next) {
    o.e1 = entry(kFirst, pl, px, w);
  } else if (pl + 1 < kGroup) {
    o.e1 = entry(kPair, pl, px, w);
  } else {   // the next bin opens the next group
    o.e1 = entry(kFirst, pl, px, w);
    o.r2 = o.r1 + E.H * E.nseg;
    o.e2 = entry(kSecond, 0, px, w);
  }
  return o;
}

__device__ __forceinline__ int64_t records_in(const uint64_t *count, int64_t max_events) {
  int64_t n = max_events;
  if (count) n = min(n, static_cast<int64_t>(min(*count, static_cast<uint64_t>(max_events))));
  return n;
}

// Counts one entry of region r for every lane with `active` set, one atomic per distinct
// region of the warp; with want_slot, returns this lane's slot (the counter's old value plus
// the lane's rank among the lanes of the same region).  Collective over the whole warp.
// Used for the rare second entries; the first entries go through the unrolled form below.
__device__ __forceinline__ unsigned long long warp_claim(unsigned long long *ctr, int r,
                                                         bool active, bool want_slot) {
  const unsigned act = __ballot_sync(evis::kFull, active);
  if (!active) return 0ull;
  const unsigned same = __match_any_sync(act, r);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(same) - 1;
  unsigned long long base = 0ull;
  if (lane == leader) base = atomicAdd(ctr + r, static_cast<unsigned long long>(__popc(same)));
  if (!want_slot) return 0ull;
  base = __shfl_sync(same, base, leader);
  return base + __popc(same & ((1u << lane) - 1u));
}

constexpr int kRecU = 4;   // batches of 32 records per warp and iteration (independent loads)

// Both record passes: each warp takes kRecU x 32 consecutive records per iteration (loads
// first, then the decoding, then one atomic per distinct region and batch, all in flight
// together).  BUCKET = false counts entries per region; BUCKET = true writes them into the
// regions' ranges (ctr then holds each range's next free slot).  FULL as for record_entries.
template <bool BUCKET, bool FULL>
__device__ __forceinline__ void record_pass(const ulonglong2 *__restrict__ ev, int64_t n,
                                            const VoxelEnvDev *__restrict__ envs, int n_envs,
                                            int bins, unsigned long long *__restrict__ ctr,
                                            unsigned long long cap,
                                            unsigned *__restrict__ entries) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  // whole warps step together (the claims are collective): the loop bound is per warp
  for (int64_t c = gw; c * 32 * kRecU < n; c += nw) {
    const int64_t k0 = c * 32 * kRecU + lane;
    ulonglong2 rec[kRecU];
#pragma unroll
    for (int u = 0; u < kRecU; ++u)
      rec[u] = k0 + 32 * u < n ? __ldcs(ev + k0 + 32 * u) : make_ulonglong2(0ull, 0ull);
    RecordEntries re[kRecU];
    unsigned same[kRecU];
    bool second = false;
#pragma unroll
    for (int u = 0; u < kRecU; ++u) {
      re[u] = record_entries<FULL>(rec[u], envs, n_envs, bins);   // an all-zero record has p = 0
      const unsigned act = __ballot_sync(evis::kFull, re[u].r1 >= 0);
      same[u] = re[u].r1 >= 0 ? __match_any_sync(act, re[u].r1) : 0u;
      second |= re[u].r2 >= 0;
    }
    unsigned long long base[kRecU];
#pragma unroll
    for (int u = 0; u < kRecU; ++u) {
      base[u] = 0ull;
      if (same[u] && lane == __ffs(same[u]) - 1) {
        if (BUCKET)
          base[u] = atomicAdd(ctr + re[u].r1, static_cast<unsigned long long>(__popc(same[u])));
        else
          atomicAdd(ctr + re[u].r1, static_cast<unsigned long long>(__popc(same[u])));
      }
    }
    if (BUCKET) {
#pragma unroll
      for (int u = 0; u < kRecU; ++u) {
        if (!same[u]) continue;
        const unsigned long long s1 = __shfl_sync(same[u], base[u], __ffs(same[u]) - 1) +
                                      __popc(same[u] & ((1u << lane) - 1u));
        // the counts came from the same records, so every slot lies in its region's range;
        // the test only keeps a damaged count from writing past the entries
        if (s1 < cap) entries[s1] = re[u].e1;
      }
    }
    if (FULL && __any_sync(evis::kFull, second)) {
#pragma unroll
      for (int u = 0; u < kRecU; ++u) {
        const unsigned long long s2 = warp_claim(ctr, re[u].r2, re[u].r2 >= 0, BUCKET);
        if (BUCKET && re[u].r2 >= 0 && s2 < cap) entries[s2] = re[u].e2;
      }
    }
  }
}

constexpr int kSmemEnvs = 64;   // environment tables up to this size go to shared memory

// Copies the first n descriptors into shared memory (whole block).
__device__ __forceinline__ void stage_envs(VoxelEnvDev *s_env, const VoxelEnvDev *envs, int n) {
  const uint4 *src = reinterpret_cast<const uint4 *>(envs);
  uint4 *dst = reinterpret_cast<uint4 *>(s_env);
  for (int i = threadIdx.x; i < n * static_cast<int>(sizeof(VoxelEnvDev) / 16); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

// Pass 1: entries per region.  n_used receives the number of records read, so that the
// bucketing pass reads exactly the same records.
__global__ void __launch_bounds__(kVoxThreads) voxel_count(const ulonglong2 *__restrict__ ev,
                                                           const uint64_t *count, int64_t max_events,
                                                           const VoxelEnvDev *__restrict__ envs,
                                                           int n_envs, int bins,
                                                           unsigned long long *__restrict__ ctr,
                                                           int64_t *n_used) {
  __shared__ __align__(16) VoxelEnvDev s_env[kSmemEnvs];
  const int64_t n = records_in(count, max_events);
  if (blockIdx.x == 0 && threadIdx.x == 0) *n_used = n;
  const bool multi = 2 * bins > kGroup;
  if (n_envs <= kSmemEnvs) {
    stage_envs(s_env, envs, n_envs);
    if (multi) record_pass<false, true>(ev, n, s_env, n_envs, bins, ctr, 0ull, nullptr);
    else record_pass<false, false>(ev, n, s_env, n_envs, bins, ctr, 0ull, nullptr);
  } else {
    if (multi) record_pass<false, true>(ev, n, envs, n_envs, bins, ctr, 0ull, nullptr);
    else record_pass<false, false>(ev, n, envs, n_envs, bins, ctr, 0ull, nullptr);
  }
}

// Pass 3: entries into their regions' ranges (cur starts at each range's first slot; cap is
// the length of the entries array).
__global__ void __launch_bounds__(kVoxThreads) voxel_bucket(const ulonglong2 *__restrict__ ev,
                                                            const int64_t *n_used,
                                                            const VoxelEnvDev *__restrict__ envs,
                                                            int n_envs, int bins,
                                                            unsigned long long *__restrict__ cur,
                                                            unsigned long long cap,
                                                            unsigned *__restrict__ entries) {
  __shared__ __align__(16) VoxelEnvDev s_env[kSmemEnvs];
  if (n_envs <= kSmemEnvs) {
    stage_envs(s_env, envs, n_envs);
    record_pass<true, true>(ev, *n_used, s_env, n_envs, bins, cur, cap, entries);
  } else {
    record_pass<true, true>(ev, *n_used, envs, n_envs, bins, cur, cap, entries);
  }
}

// Exclusive prefix sum of R counts, in blocks of kScanItems: block sums, their scan in one
// block, then each block's items with its base.
constexpr int kScanThreads = 1024, kScanPer = 8, kScanItems = kScanThreads * kScanPer;

// Block-wide exclusive scan of one value per thread; *total receives the block's sum.
__device__ __forceinline__ unsigned long long block_exclusive(unsigned long long v,
                                                              unsigned long long *total) {
  __shared__ unsigned long long s_w[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned long long u = __shfl_up_sync(evis::kFull, inc, d);
    if (lane >= d) inc += u;
  }
  if (lane == 31) s_w[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    unsigned long long w = s_w[lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long u = __shfl_up_sync(evis::kFull, w, d);
      if (lane >= d) w += u;
    }
    s_w[lane] = w;   // inclusive over warps
  }
  __syncthreads();
  const unsigned long long wbase = warp ? s_w[warp - 1] : 0ull;
  *total = s_w[kScanThreads / 32 - 1];
  __syncthreads();   // s_w is reused by the next call
  return wbase + inc - v;
}

__global__ void __launch_bounds__(kScanThreads) voxel_scan_sums(const unsigned long long *__restrict__ cnt,
                                                                int64_t R, unsigned long long *__restrict__ bsum) {
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * kScanItems + threadIdx.x * kScanPer;
  unsigned long long s = 0ull;
#pragma unroll
  for (int j = 0; j < kScanPer; ++j)
    if (i0 + j < R) s += cnt[i0 + j];
  unsigned long long total = 0ull;
  block_exclusive(s, &total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) voxel_scan_top(unsigned long long *__restrict__ bsum,
                                                               int64_t nb) {
  unsigned long long carry = 0ull;
  for (int64_t c = 0; c < nb; c += kScanThreads) {
    const int64_t i = c + threadIdx.x;
    const unsigned long long v = i < nb ? bsum[i] : 0ull;
    unsigned long long total = 0ull;
    const unsigned long long ex = block_exclusive(v, &total);
    if (i < nb) bsum[i] = carry + ex;
    carry += total;
  }
}

// off[i] = exclusive prefix of cnt; cur[i] = off[i] (cnt and cur may be the same array);
// off[R] = the total.
__global__ void __launch_bounds__(kScanThreads) voxel_scan_out(unsigned long long *cnt, int64_t R,
                                                               const unsigned long long *__restrict__ bsum,
                                                               unsigned long long *__restrict__ off) {
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * kScanItems + threadIdx.x * kScanPer;
  unsigned long long v[kScanPer], s = 0ull;
#pragma unroll
  for (int j = 0; j < kScanPer; ++j) {
    v[j] = i0 + j < R ? cnt[i0 + j] : 0ull;
    s += v[j];
  }
  unsigned long long total = 0ull;
  unsigned long long run = bsum[blockIdx.x] + block_exclusive(s, &total);
#pragma unroll
  for (int j = 0; j < kScanPer; ++j) {
    if (i0 + j < R) {
      off[i0 + j] = run;
      cnt[i0 + j] = run;
    }
    run += v[j];
    if (i0 + j == R - 1) off[R] = run;
  }
}

// The region of block r: its environment (binary search of the region offsets), plane group,
// row and segment.
struct Region {
  int64_t base;       // grid index of the region's first pixel in its group's first plane
  int64_t plane_px;   // voxels per plane of the environment
  int plane0;         // the group's first plane in the plane maxima
  int nx, np;         // pixels of the segment, planes of the group
};

__device__ __forceinline__ Region region_of(const VoxelEnvDev *__restrict__ envs, int n_envs,
                                            int bins, int r) {
  int lo = 0, hi = n_envs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (envs[mid].reg_off <= r) lo = mid; else hi = mid - 1;
  }
  const VoxelEnvDev &E = envs[lo];
  Region q;
  const int local = r - E.reg_off;
  const int seg = local % E.nseg, gy = local / E.nseg;
  const int y = gy % E.H, g = gy / E.H;
  const int x0 = seg * kSeg;
  q.nx = min(kSeg, E.W - x0);
  q.np = min(kGroup, 2 * bins - g * kGroup);
  q.plane_px = static_cast<int64_t>(E.W) * E.H;
  q.plane0 = E.plane_off + g * kGroup;
  q.base = E.vox_off + static_cast<int64_t>(g) * kGroup * q.plane_px + static_cast<int64_t>(y) * E.W + x0;
  return q;
}

// a / m correctly rounded for 0 <= a <= m < 2^32 (m > 0) with y = RN(1/m): the product a y,
// then two residual corrections q + (a - q m) y with exact fused residuals.  After the first
// q is within one unit in the last place of a / m, and the second then rounds correctly
// (Markstein, IBM J. Res. Dev. 34(1), 1990: a faithful quotient corrected with the
// correctly rounded reciprocal).
__device__ __forceinline__ float quotient(float a, float m, float y) {
  float q = __fmul_rn(a, y);
  q = __fmaf_rn(__fmaf_rn(-q, m, a), y, q);
  return __fmaf_rn(__fmaf_rn(-q, m, a), y, q);
}

constexpr int kRegionsPerBlock = 8;   // consecutive regions: mostly one row of one group
constexpr int kPrefetch = 8;          // entries per thread loaded one region ahead
constexpr int kRow = kSeg + 4;        // words per plane row of the sums: 16-byte rows whose
                                      // 128-bit reads by eight consecutive planes hit
                                      // distinct banks

// Adds one entry to the sums and its blocks of eight planes to the touch mask.
__device__ __forceinline__ void add_entry(unsigned *s_acc, unsigned v, unsigned &touch) {
  const unsigned w = v & 0xFFFFu, kind = v >> 29;
  const int px = (v >> 16) & 31, pl = (v >> 21) & 255;
  unsigned *a = s_acc + pl * kRow + px;
  touch |= 1u << (pl >> 3);
  if (kind == kSecond) {
    atomicAdd(a, w);
  } else {
    atomicAdd(a, 65536u - w);
    if (kind == kPair) {
      atomicAdd(a + kRow, w);
      touch |= 1u << ((pl + 1) >> 3);
    }
  }
}

// OUT = 0: the plane maxima; OUT = 1: the normalised grid.  Each block takes kRegionsPerBlock
// consecutive regions in turn; their descriptors and entry ranges are read once at the start,
// and each region's first kPrefetch entries per thread are loaded while the region before it
// is finished.  Per-plane state lives in shared memory for as long as the regions stay in
// one (environment, group): OUT = 0 keeps the running maxima (thread pl owns plane pl) and
// merges them into the global maxima once; OUT = 1 loads the group's maxima and their
// reciprocals once.  The sums are cleared once per block; after that only planes in the
// blocks of eight that a region's entries touched (bit j of the touch mask: planes 8j ..
// 8j + 7) are read, and zeroed as they are read.
template <int OUT>
__global__ void __launch_bounds__(kVoxThreads) voxel_region(const VoxelEnvDev *__restrict__ envs,
                                                            int n_envs, int bins, int R,
                                                            const unsigned long long *__restrict__ off,
                                                            const unsigned *__restrict__ entries,
                                                            unsigned *__restrict__ pmax,
                                                            float *__restrict__ grid) {
  static_assert(kGroup == kVoxThreads, "one thread per plane of the group");
  __shared__ __align__(16) unsigned s_acc[kGroup * kRow];
  __shared__ unsigned s_max[kGroup];
  __shared__ float s_m[kGroup], s_y[kGroup];
  __shared__ unsigned s_touch;
  __shared__ Region s_reg[kRegionsPerBlock];
  __shared__ unsigned long long s_off[kRegionsPerBlock + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r0 = blockIdx.x * kRegionsPerBlock, nr = min(R - r0, kRegionsPerBlock);
  {
    uint4 *s4 = reinterpret_cast<uint4 *>(s_acc);
    for (int i = tid; i < kGroup * kRow / 4; i += kVoxThreads) s4[i] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) s_touch = 0u;
    if (tid < nr) s_reg[tid] = region_of(envs, n_envs, bins, r0 + tid);
    if (tid >= 32 && tid - 32 <= nr) s_off[tid - 32] = off[r0 + tid - 32];
  }
  __syncthreads();
  unsigned pre[kPrefetch];
  auto prefetch = [&](int k) {
    const unsigned long long b = s_off[k], n = s_off[k + 1] - b;
#pragma unroll
    for (int u = 0; u < kPrefetch; ++u) {
      const unsigned long long i = tid + static_cast<unsigned long long>(u) * kVoxThreads;
      pre[u] = i < n ? (OUT ? __ldcs(entries + b + i) : __ldg(entries + b + i)) : 0xFFFFFFFFu;
    }
  };
  prefetch(0);
  int cur0 = -1, cur_np = 0;   // the plane group whose state is loaded (first plane, planes)
  for (int k = 0; k < nr; ++k) {
    const Region q = s_reg[k];
    const int plane0 = q.plane0;
    if (plane0 != cur0) {   // uniform over the block; thread i reads and resets entry i
      if (OUT == 0) {
        if (tid < cur_np && s_max[tid]) atomicMax(pmax + cur0 + tid, s_max[tid]);
        s_max[tid] = 0u;
      } else if (tid < q.np) {
        const unsigned m = pmax[plane0 + tid];
        const float fm = __uint2float_rn(m);
        s_m[tid] = fm;
        s_y[tid] = m ? __frcp_rn(fm) : 0.0f;
      }
      cur0 = plane0;
      cur_np = q.np;
    }
    __syncthreads();   // state loaded, sums and touch mask clear
    unsigned touch = 0u;
#pragma unroll
    for (int u = 0; u < kPrefetch; ++u)
      if (pre[u] != 0xFFFFFFFFu) add_entry(s_acc, pre[u], touch);   // no entry has all bits set
    {
      // entries past the prefetched ones, four loads in flight per thread
      const unsigned long long b = s_off[k], n = s_off[k + 1] - b;
      for (unsigned long long i = tid + static_cast<unsigned long long>(kPrefetch) * kVoxThreads; i < n;
           i += 4 * kVoxThreads) {
        unsigned v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const unsigned long long j = i + u * kVoxThreads;
          v[u] = j < n ? (OUT ? __ldcs(entries + b + j) : __ldg(entries + b + j)) : 0xFFFFFFFFu;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (v[u] != 0xFFFFFFFFu) add_entry(s_acc, v[u], touch);
      }
    }
    if (k + 1 < nr) prefetch(k + 1);
    touch = __reduce_or_sync(evis::kFull, touch);
    if (lane == 0 && touch) atomicOr(&s_touch, touch);
    __syncthreads();
    touch = s_touch;
    if (OUT == 0) {
      // thread tid takes plane tid: eight 128-bit reads of its row, zeroed behind it
      if (tid < q.np && ((touch >> (tid >> 3)) & 1u)) {
        uint4 *a = reinterpret_cast<uint4 *>(s_acc + tid * kRow);
        unsigned m = s_max[tid];
#pragma unroll
        for (int c = 0; c < kSeg / 4; ++c) {
          const uint4 v = a[c];
          m = max(m, max(max(v.x, v.y), max(v.z, v.w)));
          a[c] = make_uint4(0u, 0u, 0u, 0u);
        }
        s_max[tid] = m;
      }
    } else {
      const int64_t plane_px = q.plane_px, base = q.base;
      // 16-byte stores need every plane's row start on a 16-byte boundary (the grid itself
      // need only be 4-byte aligned)
      if (q.nx == kSeg && (reinterpret_cast<uintptr_t>(grid + base) & 15) == 0 && (plane_px & 3) == 0) {
        // four pixels per thread: eight threads per plane row, 32 planes per pass of the block
        const int px = (tid & 7) * 4;
        for (int pl = tid >> 3; pl < q.np; pl += kVoxThreads / 8) {
          float4 val = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          if ((touch >> (pl >> 3)) & 1u) {   // uniform over each warp's four planes
            uint4 *a = reinterpret_cast<uint4 *>(s_acc + pl * kRow + px);
            const uint4 v = *a;
            *a = make_uint4(0u, 0u, 0u, 0u);
            const float fy = s_y[pl], fm = s_m[pl];
            if (fy != 0.0f) {
              val.x = quotient(__uint2float_rn(v.x), fm, fy);
              val.y = quotient(__uint2float_rn(v.y), fm, fy);
              val.z = quotient(__uint2float_rn(v.z), fm, fy);
              val.w = quotient(__uint2float_rn(v.w), fm, fy);
            }
          }
          __stcs(reinterpret_cast<float4 *>(grid + base + pl * plane_px + px), val);
        }
      } else {
        // one pixel per lane, one plane row per warp
        float *o = grid + base + warp * plane_px + lane;
        for (int j = 0, pl = warp; pl < q.np; ++j, pl += kVoxThreads / 32, o += (kVoxThreads / 32) * plane_px) {
          float val = 0.0f;
          if ((touch >> j) & 1u) {
            unsigned *a = s_acc + pl * kRow + lane;
            const unsigned v = *a;
            *a = 0u;
            const float fy = s_y[pl];
            if (fy != 0.0f) val = quotient(__uint2float_rn(v), s_m[pl], fy);
          }
          if (lane < q.nx) __stcs(o, val);
        }
      }
    }
    __syncthreads();   // every read of the sums, the mask and the per-plane state is done
    if (tid == 0) s_touch = 0u;
  }
  if (OUT == 0 && cur0 >= 0 && tid < cur_np && s_max[tid]) atomicMax(pmax + cur0 + tid, s_max[tid]);
}

constexpr size_t kAlign = 256;

size_t up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

std::string check(const evis_voxel_env *envs, int32_t n_envs, int32_t bins, int64_t max_events,
                  int64_t *regions) {
  if (!envs) return "envs is null";
  if (n_envs < 1 || n_envs > 65535) return "n_envs must be in 1..65535";
  if (bins < 1 || bins > 1024) return "bins must be in 1..1024";
  if (max_events < 0) return "max_events must be >= 0";
  const int ngroups = (2 * bins + kGroup - 1) / kGroup;
  int64_t R = 0;
  for (int i = 0; i < n_envs; ++i) {
    const evis_voxel_env &d = envs[i];
    if (d.width < 1 || d.height < 1 || d.width > 65535 || d.height > 65535 ||
        int64_t(d.width) * d.height > (int64_t(1) << 24))
      return "sensor sizes must be in 1..65535 with width*height <= 2^24";
    if (!(d.t1_ns > d.t0_ns) || d.t1_ns - d.t0_ns >= (int64_t(1) << 32))
      return "each segment needs 0 < t1_ns - t0_ns < 2^32";
    R += int64_t(ngroups) * d.height * ((d.width + kSeg - 1) / kSeg);
  }
  if (R > int64_t(INT32_MAX)) return "too many regions (one block each)";
  *regions = R;
  return "";
}

// Workspace: descriptor table, plane maxima (uint32), records read (int64), region counters
// and cursors (uint64 each), region offsets (R + 1), scan block sums, entries (uint32).
struct Layout {
  size_t tab, pmax, nused, cur, off, bsum, ent, total;
  int64_t R, nb, cap;
};

Layout layout(int32_t n_envs, int32_t bins, int64_t R, int64_t max_events) {
  Layout L;
  L.R = R;
  L.nb = (R + kScanItems - 1) / kScanItems;
  L.cap = max_events * (2 * bins > kGroup ? 2 : 1);
  L.tab = 0;
  L.pmax = L.tab + up(sizeof(VoxelEnvDev) * n_envs);
  L.nused = L.pmax + up(sizeof(unsigned) * 2 * bins * n_envs);
  L.cur = L.nused + up(sizeof(int64_t));
  L.off = L.cur + up(sizeof(unsigned long long) * R);
  L.bsum = L.off + up(sizeof(unsigned long long) * (R + 1));
  L.ent = L.bsum + up(sizeof(unsigned long long) * L.nb);
  L.total = L.ent + up(sizeof(unsigned) * L.cap);
  return L;
}

}  // namespace

extern "C" evis_status evis_voxel_workspace_size(const evis_voxel_env *envs, int32_t n_envs,
                                                 int32_t bins, int64_t max_events, int64_t *bytes) {
  int64_t R = 0;
  if (!bytes || !check(envs, n_envs, bins, max_events, &R).empty()) return EVIS_ERR_INVALID_ARG;
  *bytes = static_cast<int64_t>(layout(n_envs, bins, R, max_events).total);
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
  int64_t R = 0;
  const std::string why = check(envs, n_envs, bins, max_events, &R);
  if (!why.empty()) return reject(why);
  if (max_events > 0 && !events) return reject("events is null");
  if (!workspace || !grid) return reject("null workspace or grid");
  if (reinterpret_cast<uintptr_t>(events) % 16 || reinterpret_cast<uintptr_t>(workspace) % 16 ||
      reinterpret_cast<uintptr_t>(grid) % 4 || reinterpret_cast<uintptr_t>(count) % 8)
    return reject("events and workspace need 16-byte alignment, count 8-byte, grid 4-byte");
  const Layout L = layout(n_envs, bins, R, max_events);
  if (workspace_bytes < static_cast<int64_t>(L.total))
    return reject("workspace smaller than evis_voxel_workspace_size");
  const int ngroups = (2 * bins + kGroup - 1) / kGroup;
  std::vector<VoxelEnvDev> tab(n_envs);
  int64_t vox = 0, reg = 0;
  for (int i = 0; i < n_envs; ++i) {
    VoxelEnvDev &d = tab[i];
    d.W = envs[i].width;
    d.H = envs[i].height;
    d.t0 = envs[i].t0_ns;
    d.t1 = envs[i].t1_ns;
    d.D = static_cast<uint64_t>(d.t1 - d.t0);
    d.inv = ~0ull / d.D;
    d.vox_off = vox;
    d.reg_off = static_cast<int32_t>(reg);
    d.nseg = (d.W + kSeg - 1) / kSeg;
    d.plane_off = 2 * bins * i;
    vox += 2LL * bins * d.W * d.H;
    reg += int64_t(ngroups) * d.H * d.nseg;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned char *ws = static_cast<unsigned char *>(workspace);
  VoxelEnvDev *d_tab = reinterpret_cast<VoxelEnvDev *>(ws + L.tab);
  unsigned *pmax = reinterpret_cast<unsigned *>(ws + L.pmax);
  int64_t *n_used = reinterpret_cast<int64_t *>(ws + L.nused);
  unsigned long long *cur = reinterpret_cast<unsigned long long *>(ws + L.cur);
  unsigned long long *off = reinterpret_cast<unsigned long long *>(ws + L.off);
  unsigned long long *bsum = reinterpret_cast<unsigned long long *>(ws + L.bsum);
  unsigned *ent = reinterpret_cast<unsigned *>(ws + L.ent);
  const ulonglong2 *ev = reinterpret_cast<const ulonglong2 *>(events);
  cudaError_t e;
  int dev = 0, sms = 0;
  // pageable source: the copy is staged before the call returns, so tab may go away
  if ((e = cudaMemcpyAsync(d_tab, tab.data(), sizeof(VoxelEnvDev) * n_envs, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemsetAsync(pmax, 0, sizeof(unsigned) * 2 * bins * n_envs, s)) ||
      (e = cudaMemsetAsync(cur, 0, sizeof(unsigned long long) * R, s)) ||
      (e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
    goto fail;
  {
    // the record passes: one resident wave of blocks in a grid-stride loop
    int occ_c = 0, occ_b = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_c, voxel_count, kVoxThreads, 0)) ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_b, voxel_bucket, kVoxThreads, 0)))
      goto fail;
    const int64_t want = (max_events + 32 * kRecU * (kVoxThreads / 32) - 1) / (32 * kRecU * (kVoxThreads / 32));
    const int blocks_c = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(std::max(occ_c, 1)) * sms)));
    const int blocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(std::max(occ_b, 1)) * sms)));
    voxel_count<<<blocks_c, kVoxThreads, 0, s>>>(ev, count, max_events, d_tab, n_envs, bins, cur, n_used);
    if ((e = cudaGetLastError()) != cudaSuccess) goto fail;
    voxel_scan_sums<<<static_cast<unsigned>(L.nb), kScanThreads, 0, s>>>(cur, R, bsum);
    voxel_scan_top<<<1, kScanThreads, 0, s>>>(bsum, L.nb);
    voxel_scan_out<<<static_cast<unsigned>(L.nb), kScanThreads, 0, s>>>(cur, R, bsum, off);
    if ((e = cudaGetLastError()) != cudaSuccess) goto fail;
    voxel_bucket<<<blocks, kVoxThreads, 0, s>>>(ev, n_used, d_tab, n_envs, bins, cur,
                                                static_cast<unsigned long long>(L.cap), ent);
    if ((e = cudaGetLastError()) != cudaSuccess) goto fail;
    const unsigned rb = static_cast<unsigned>((R + kRegionsPerBlock - 1) / kRegionsPerBlock);
    const int Ri = static_cast<int>(R);
    voxel_region<0><<<rb, kVoxThreads, 0, s>>>(d_tab, n_envs, bins, Ri, off, ent, pmax, grid);
    voxel_region<1><<<rb, kVoxThreads, 0, s>>>(d_tab, n_envs, bins, Ri, off, ent, pmax, grid);
    if ((e = cudaGetLastError()) != cudaSuccess) goto fail;
  }
  return EVIS_OK;
fail:
  evis::set_detached_error(std::string("evis_voxel_grid: ") + cudaGetErrorString(e));
  return EVIS_ERR_CUDA;
}
