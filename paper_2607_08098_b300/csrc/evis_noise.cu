// Sensor noise of Sec. 3.4 (leak events, shot noise, hot pixels), one keyframe gap at a time
// and apart from the synthesis kernel: noise events neither read nor change the per-pixel
// event state, so they need only the gap's two prepared keyframes.
//
// noise_kernel: one thread per sensor pixel and channel of one environment (grid.y) for all
// K sub-frames.  The block first puts each sub-frame's constants (f, the sources' rates times
// its duration, its start and duration) in shared memory.  Each pixel-sub-frame draws one
// 32-bit word, four consecutive sub-frames sharing one Philox4x32-10 call; the word picks at
// most one of the competing sources by cumulative thresholds (leak, then shot, then hot), and
// a source that fires takes its time (and the shot polarity) from a second call.  A block
// stages its events in shared memory and reserves their range of the event buffer with one
// atomic at the end.
#include "evis_device.cuh"
#include "evis_internal.h"

namespace evis {
namespace {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
// SC 2011): ten rounds, each two 32 x 32 -> 64-bit products of the counter's even words
// mixed into the odd words with the round key; the key advances by the Weyl increments.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, unsigned k0, unsigned k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// The 24-bit value of a uniform word against a probability q, both in binary32 units of
// 2^-24: a Bernoulli draw with probability q fires when it holds.
__device__ __forceinline__ bool below(float x24, float q) { return x24 < __fmul_rn(q, 16777216.0f); }

// t0 + floor(u d / 2^32) for d < 2^41: the product split at bit 32 of d.
__device__ __forceinline__ int64_t noise_time(unsigned u, int64_t t0, int64_t d) {
  const unsigned long long du = static_cast<unsigned long long>(d);
  const unsigned long long lo = (static_cast<unsigned long long>(u) * (du & 0xFFFFFFFFull)) >> 32;
  return t0 + static_cast<int64_t>(static_cast<unsigned long long>(u) * (du >> 32) + lo);
}

__device__ __forceinline__ ulonglong2 make_event(int64_t t, int x, int y, int env, int p) {
  ulonglong2 r;
  r.x = static_cast<unsigned long long>(t);
  r.y = static_cast<unsigned long long>(x & 0xFFFF) |
        (static_cast<unsigned long long>(y & 0xFFFF) << 16) |
        (static_cast<unsigned long long>(env & 0xFFFF) << 32) |
        (static_cast<unsigned long long>(static_cast<uint16_t>(static_cast<int16_t>(p))) << 48);
  return r;
}

constexpr int kNoiseThreads = 256;
constexpr int kNoiseStage = 1024;   // events staged per block; more go out one atomic each
constexpr int kSubChunk = 256;      // sub-frames whose constants a block holds at once (4 | it)

__global__ void __launch_bounds__(kNoiseThreads) noise_kernel(const StepArgs a) {
  __shared__ ulonglong2 s_ev[kNoiseStage];
  __shared__ float4 s_sf[kSubChunk];     // per sub-frame: f, leak dts, shot dts, hot dts
  __shared__ longlong2 s_t[kSubChunk];   // per sub-frame: t_{i-1}, d = t_i - t_{i-1}
  __shared__ unsigned s_n, s_on, s_off;
  __shared__ unsigned long long s_base;
  const int env = blockIdx.y, c = blockIdx.z;
  const DevEnv &E = a.envs[env];
  if (!E.noise) return;   // uniform over the block
  const int m = E.margin, SW = E.W - 2 * m, SH = E.H - 2 * m;
  if (static_cast<int64_t>(blockIdx.x) * kNoiseThreads >= static_cast<int64_t>(SW) * SH) return;
  if (threadIdx.x == 0) s_n = s_on = s_off = 0u;
  const int sp = blockIdx.x * kNoiseThreads + threadIdx.x;   // sensor pixel index sy * SW + sx
  const bool valid = sp < SW * SH;
  const int sy = valid ? sp / SW : 0, sx = valid ? sp - sy * SW : 0;
  const int64_t pix = E.pix_off + static_cast<int64_t>(sy + m) * E.W + (sx + m);
  const float la = valid ? __ldg(a.LA + c * a.plane + pix) : 0.0f;
  const float lb = valid ? __ldg(a.LB + c * a.plane + pix) : 0.0f;
  const unsigned npix = static_cast<unsigned>(sp), cw = 4u * static_cast<unsigned>(c);
  const unsigned gap = a.gap_in[env];
  const int K = E.K;
  const int64_t T0 = a.clock_in[env];
  const unsigned k0 = E.key0, k1 = E.key1;
  // the hot subset: fixed per pixel and channel, the same in every gap
  const bool hot = valid && E.hot_hz > 0.0f &&
                   below(__uint2float_rn(philox4x32_10(make_uint4(npix, 0xFFFFFFFFu, 0u, 2u + cw), k0, k1).x >> 8),
                         E.hot_fraction);
  const float lo = E.noise_lo, inv_range = __frcp_rn(__fsub_rn(E.noise_hi, E.noise_lo));
  // t_i = T0 + floor(i dt / K) = T0 + i q + floor(i r / K) with dt = q K + r (no overflow)
  const int64_t dq = a.dt / K;
  const int64_t dr = a.dt % K;
  const unsigned lanes_below = (1u << (threadIdx.x & 31)) - 1u;
  for (int c0 = 0; c0 < K; c0 += kSubChunk) {   // sub-frames c0 + 1 .. c0 + nk
    const int nk = min(kSubChunk, K - c0);
    __syncthreads();   // the previous chunk's constants are no longer read
    for (int k = threadIdx.x; k < nk; k += kNoiseThreads) {
      const int i = c0 + k + 1;
      const int64_t tim1 = T0 + (i - 1) * dq + ((i - 1) * dr) / K;
      const int64_t d = T0 + i * dq + (i * dr) / K - tim1;
      const float dts = __fmul_rn(__ll2float_rn(d), 1e-9f);
      s_sf[k] = make_float4(__fdiv_rn(static_cast<float>(i), static_cast<float>(K)), __fmul_rn(E.leak_hz, dts),
                            __fmul_rn(E.shot_hz, dts), __fmul_rn(E.hot_hz, dts));
      s_t[k] = make_longlong2(tim1, d);
    }
    __syncthreads();
    for (int k4 = 0; k4 < nk; k4 += 4) {   // one Philox call per four sub-frames
      const uint4 r = philox4x32_10(make_uint4(npix, gap, static_cast<unsigned>(c0 + k4) >> 2, cw), k0, k1);
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const int k = k4 + w;
        if (k >= nk) break;   // uniform over the block
        const unsigned u = w == 0 ? r.x : (w == 1 ? r.y : (w == 2 ? r.z : r.w));
        const float4 q = s_sf[k];   // f, leak dts, shot dts, hot dts
        const float L = __fadd_rn(__fmul_rn(__fsub_rn(1.0f, q.x), la), __fmul_rn(q.x, lb));
        float ib = __fmul_rn(__fsub_rn(L, lo), inv_range);
        ib = ib < 0.0f ? 0.0f : (ib > 1.0f ? 1.0f : ib);
        const float s1 = q.y;
        const float s2 = __fadd_rn(s1, __fmul_rn(q.z, __fsub_rn(1.0f, ib)));
        const float s3 = hot ? __fadd_rn(s2, q.w) : s2;
        const float x24 = __uint2float_rn(u >> 8);
        const bool fire = valid && below(x24, s3);
        const unsigned mf = __ballot_sync(kFull, fire);
        if (mf == 0) continue;   // by far the common case
        ulonglong2 rec = make_ulonglong2(0ull, 0ull);
        if (fire) {
          const int i = c0 + k + 1;
          const bool leak = below(x24, s1), shot = !leak && below(x24, s2);
          const uint4 rt = philox4x32_10(make_uint4(npix, gap, static_cast<unsigned>(i), 1u + cw), k0, k1);
          const int p = (shot && !(rt.w & 1u)) ? -(1 + c) : 1 + c;
          const longlong2 tt = s_t[k];
          rec = make_event(noise_time(rt.x, tt.x, tt.y), sx, sy, env, p);
        }
        unsigned base = 0;
        if ((threadIdx.x & 31) == 0) base = atomicAdd(&s_n, static_cast<unsigned>(__popc(mf)));
        base = __shfl_sync(kFull, base, 0);
        if (fire) {
          const unsigned idx = base + static_cast<unsigned>(__popc(mf & lanes_below));
          if (idx < static_cast<unsigned>(kNoiseStage)) {
            s_ev[idx] = rec;
          } else {   // the stage is full: straight to the buffer
            const unsigned long long gi = atomicAdd(a.ev_count, 1ull);
            if (gi < a.capacity) a.events[gi] = rec;
          }
          if (a.stats) atomicAdd(static_cast<long long>(rec.y) < 0 ? &s_off : &s_on, 1u);
        }
      }
    }
  }
  __syncthreads();
  const unsigned n = min(s_n, static_cast<unsigned>(kNoiseStage));
  if (threadIdx.x == 0) {
    s_base = n ? atomicAdd(a.ev_count, static_cast<unsigned long long>(n)) : 0ull;
    if (a.stats && a.env_stats && (s_on | s_off)) {
      unsigned long long *st = a.env_stats + static_cast<int64_t>(env) * kStatWords;
      atomicAdd(st + kStatNoise, static_cast<unsigned long long>(s_on + s_off));
      if (s_on) atomicAdd(st + kStatEventsOn, static_cast<unsigned long long>(s_on));
      if (s_off) atomicAdd(st + kStatEventsOff, static_cast<unsigned long long>(s_off));
    }
  }
  __syncthreads();
  for (unsigned k = threadIdx.x; k < n; k += kNoiseThreads) {
    const unsigned long long gi = s_base + k;
    if (gi < a.capacity) a.events[gi] = s_ev[k];
  }
}

}  // namespace

cudaError_t launch_noise(const StepArgs &a, int n_envs, int max_px, cudaStream_t s) {
  if (!a.noise || n_envs <= 0 || max_px <= 0) return cudaSuccess;
  if (!a.gap_in || !a.clock_in) return cudaErrorInvalidValue;
  const dim3 grid((max_px + kNoiseThreads - 1) / kNoiseThreads, n_envs, a.nc == 3 ? 3 : 1);
  noise_kernel<<<grid, kNoiseThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace evis
