// The synthesis kernel of the EVIS event path (sm_103a), as templates: the translation
// units evis_step_*.cu instantiate its variants (tile shapes, trace, colour, statistics), so
// that they compile in parallel.  Sensor noise has its own kernel (evis_noise.cu).
//
// Compiled with -fmad=false and written with explicit round-to-nearest intrinsics so that
// every floating-point step that decides a z-buffer winner or an event count is the same
// single IEEE-754 binary32 operation, in the same order, as in the method's definition:
// splat winners, event counts, pixels and polarities are then reproducible bit for bit on
// any IEEE host.
//
// step_kernel: per keyframe gap, one CTA owns a TX x TY target tile of one environment and
//   keeps, for all K sub-frames, its pixels' event state in registers.  Once per gap it
//   lists the row segments whose motion bounds let them reach the tile.  Per sub-frame:
//   phase 1 re-tests the listed segments and lists the sources that may land in the tile
//   (whole segments, and lane intervals of the others); phase 2 gives every thread one
//   listed source and splats A forward and B backward into two shared-memory z-buffers with
//   64-bit atomicMin on (depth, weight, source) keys (Eqs. 5-7); phase 3 resolves the
//   winners, blends in time with hole filling, runs the event model (Eq. 4, Eq. 8,
//   refractory period) and compacts the events: a warp-wide reservation per chunk of
//   crossings in a shared staging buffer, one global atomic per CTA per sub-frame, and a
//   coalesced 16-byte-per-thread flush during the next sub-frame.
#pragma once

#include <cuda_fp16.h>

#include <atomic>

#include "evis_device.cuh"
#include "evis_internal.h"

namespace evis {
namespace {

// floor(v) of |v| < 2^22 without a conversion instruction: adding 1.5 * 2^23 with rounding
// toward -infinity lands on the integer grid (ulp 1), whose low significand bits hold the
// integer.  *fv receives floor(v) as a float (exact).
__device__ __forceinline__ int floor_small(float v, float *fv) {
  const float t = __fadd_rd(v, 12582912.0f);
  *fv = __fsub_rn(t, 12582912.0f);
  return __float_as_int(t) - 0x4B400000;
}

// (float)i for 0 <= i < 2^23 without a conversion instruction.
__device__ __forceinline__ float small_int_to_float(int i) {
  return __fsub_rn(__int_as_float(0x4B000000 + i), 8388608.0f);
}

// The target tile clipped to the image: pixels [x0, x0 + nx) x [y0, y0 + ny).
struct TileBox {
  int x0, y0, nx, ny;
  float qxl, qxh, qyl, qyh;  // x0 - 1, x0 + nx, y0 - 1, y0 + ny as floats
};

// Splat of one source at one sub-frame into the tile's z-buffer of that sub-frame
// (Sec. 3.3).  Direction 0 moves a source of A forward to q = p - f m_A with depth
// (1-f) Z_A(p) + f Z_B(p - m_A); direction 1 moves a source of B backward to
// q = p + (1-f) m_B with depth (1-f) Z_A(p + m_B) + f Z_B(p) (Eqs. 5, 7): zs is the source's
// own depth, zo the other keyframe's at the correspondence endpoint.  Every integer pixel of
// the bilinear footprint of q with weight > 0, inside the image and inside the tile, keeps
// the minimum key [depth bits | quantised (1 - w) | source index] (Eq. 6).
template <int TX, int TY>
__device__ __forceinline__ void splat_at(unsigned long long *zb, int dir, int p, float fx,
                                         float fy, float mx, float my, float zs, float zo,
                                         float f, float g, TileBox bx, bool tie_index) {
  float qx, qy;
  if (dir == 0) {
    qx = __fsub_rn(fx, __fmul_rn(f, mx));
    qy = __fsub_rn(fy, __fmul_rn(f, my));
  } else {
    qx = __fadd_rn(fx, __fmul_rn(g, mx));
    qy = __fadd_rn(fy, __fmul_rn(g, my));
  }
  // A footprint pixel lies in the box only if x0 - 1 < q_x < x0 + nx (floor(q_x) + 1 needs
  // a positive weight) and likewise in y.  The box lies inside the image, so this also
  // rejects targets that leave it, and NaN.
  if (!(qx > bx.qxl && qx < bx.qxh && qy > bx.qyl && qy < bx.qyh)) return;
  float fx0, fy0;
  const int lx0 = floor_small(qx, &fx0) - bx.x0, ly0 = floor_small(qy, &fy0) - bx.y0;  // >= -1
  const float zt = dir == 0 ? __fadd_rn(__fmul_rn(g, zs), __fmul_rn(f, zo))
                            : __fadd_rn(__fmul_rn(g, zo), __fmul_rn(f, zs));
  const float ax = __fsub_rn(qx, fx0), ay = __fsub_rn(qy, fy0);
  const float wx[2] = {__fsub_rn(1.0f, ax), ax};
  const float wy[2] = {__fsub_rn(1.0f, ay), ay};
  const bool in_x[2] = {lx0 >= 0, lx0 + 1 < bx.nx};
  const bool in_y[2] = {ly0 >= 0, ly0 + 1 < bx.ny};
  const unsigned long long hi = static_cast<unsigned long long>(__float_as_uint(zt)) << 32;
  const int c00 = ly0 * TX + lx0;
  // Straight-line code: every cell's key is formed, only the atomic is predicated.
#pragma unroll
  for (int dy = 0; dy < 2; ++dy) {
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
      const float w = __fmul_rn(wx[dx], wy[dy]);
      // Inside the box the pixel floor(q) has q >= 0, so a = q - floor(q) < 1 is exact and
      // 1 - a >= 2^-24: its weight is at least 2^-48.  The others may round to 0.
      const bool ok = in_x[dx] && in_y[dy] && ((dx | dy) == 0 || w > 0.0f);
      // (1 - w) 256 in [0, 256], rounded once (256 w is exact), clamped below 256 and
      // truncated by a rounding-down add onto the integer grid of 1.5 x 2^23: the low byte
      // of the sum's bits is the integer min(floor((1 - w) 256), 255)
      const float t = fminf(__fmaf_rn(-256.0f, w, 256.0f), 255.5f);
      const unsigned low = static_cast<unsigned>(p) +
                           (tie_index ? 0u : __float_as_uint(__fadd_rd(t, 12582912.0f)) << 24);
      if (ok) atomicMin(&zb[c00 + dy * TX + dx], hi | low);
    }
  }
}

// One source of direction dir splat at the first ns sub-frames of a pass (fractions fs,
// 1 - fs) into their z-buffers.  PACKED reads (mx, my, Z, Z at the other endpoint) prepared
// once per keyframe gap; otherwise the motion and depth maps are read and the other
// endpoint's depth is gathered.  Only sources with a valid depth splat.
template <int TX, int TY, int NP, bool PACKED>
__device__ __forceinline__ void splat_source(unsigned long long (&zb)[NP][2][TX * TY], int dir,
                                             int sx, int sy, float fx, float fy, int W, int H,
                                             TileBox bx, const float *fs,
                                             const float *gs, int ns, const StepArgs &a,
                                             int64_t o) {
  const int p = sy * W + sx;
  float mx, my, zs, zo;
  if (PACKED) {
    const float4 v = __ldg((dir ? a.packB : a.packA) + o + p);
    mx = v.x;
    my = v.y;
    zs = v.z;
    zo = v.w;
    if (!valid_depth(zs)) return;
  } else {
    zs = __ldg((dir ? a.ZB : a.ZA) + o + p);
    if (!valid_depth(zs)) return;
    const float2 m = __ldg(reinterpret_cast<const float2 *>(dir ? a.mvB : a.mvA) + o + p);
    mx = m.x;
    my = m.y;
    zo = dir == 0 ? other_depth(a.ZB + o, W, H, __fsub_rn(fx, mx), __fsub_rn(fy, my), zs)
                  : other_depth(a.ZA + o, W, H, __fadd_rn(fx, mx), __fadd_rn(fy, my), zs);
  }
  const bool tie_index = (a.flags & EVIS_TIE_INDEX) != 0;
#pragma unroll
  for (int u = 0; u < NP; ++u)
    if (u < ns) splat_at<TX, TY>(zb[u][dir], dir, p, fx, fy, mx, my, zs, zo, fs[u], gs[u], bx, tie_index);
}

// True when no source of a row segment [xs, xs+31] x {ys}, displaced by an amount in
// [dxl, dxh] x [dyl, dyh], can put a footprint pixel into the TX x TY tile at (x0, y0).  A
// source lands a footprint pixel in the tile only if its target q has x0 - 1 < q_x <
// x0 + TX (the pixel floor(q) + 1 needs a positive weight) and likewise in y.  The bounds
// enclose the rounded displacements and rounding is monotone, so fl(xs + 31 + dxh) bounds
// every q_x of the segment from above and fl(xs + dxl) from below: fl(that + 1) < x0 or
// fl(xs + dxl) >= x0 + TX excludes the tile exactly.  NaN bounds never count as a miss.
template <int TX, int TY>
__device__ __forceinline__ bool seg_misses(float xs, float ys, float dxl, float dxh, float dyl,
                                           float dyh, int x0, int y0) {
  return (xs + 31.0f + dxh + 1.0f < static_cast<float>(x0)) ||
         (xs + dxl >= static_cast<float>(x0 + TX)) ||
         (ys + dyh + 1.0f < static_cast<float>(y0)) ||
         (ys + dyl >= static_cast<float>(y0 + TY));
}

// t_prev + llrint(fr * (t_i - t_prev)) with the product taken in binary64 and rounded half to
// even.  When t_i - t_prev < 2^29 the binary64 product of the binary32 fraction (24-bit
// significand) and the interval is exact, so the same integer is obtained with a 64-bit
// integer multiply, a shift and a round-half-even on the discarded bits.  Longer intervals
// take the binary64 route.
__device__ __forceinline__ int64_t interp_time(float fr, int64_t tprev, int64_t ti) {
  const int64_t d = ti - tprev;
  if (d < (int64_t(1) << 29)) {
    const unsigned b = __float_as_uint(fr);          // fr in [0, 1]
    const unsigned ex = b >> 23;
    const unsigned m = ex ? ((b & 0x7FFFFFu) | 0x800000u) : (b & 0x7FFFFFu);
    const int sh = ex ? 150 - static_cast<int>(ex) : 149;   // fr = m * 2^-sh, sh >= 23
    const unsigned long long P = static_cast<unsigned long long>(m) *
                                 static_cast<unsigned>(d);   // 24 x 29 bits: < 2^53
    if (sh >= 64) return tprev;                      // fr * d < 2^-11
    // round half to even: adding 2^(sh-1) - 1 and the parity of the truncated quotient
    // carries into bit sh exactly when the discarded part exceeds the half, or equals it
    // with an odd quotient (the sum stays below 2^63)
    const unsigned long long q =
        (P + ((1ull << (sh - 1)) - 1ull) + ((P >> sh) & 1ull)) >> sh;
    return tprev + static_cast<int64_t>(q);
  }
  return tprev + __double2ll_rn(__dmul_rn(static_cast<double>(fr), static_cast<double>(d)));
}

// Time of the k-th crossing of a pixel in this sub-frame: the level Lref + p k theta,
// interpolated linearly between the previous sample (tprev, Lprev) and this one (ti, L).
__device__ __forceinline__ int64_t crossing_time(float Lref, float pk, float th, float Lprev,
                                                 float L, int64_t tprev, int64_t ti) {
  const float lev = __fadd_rn(Lref, __fmul_rn(pk, th));
  const float num = __fsub_rn(lev, Lprev);
  const float den = __fsub_rn(L, Lprev);
  float fr = den == 0.0f ? 1.0f : __fdiv_rn(num, den);
  if (!(fr > 0.0f)) fr = 0.0f;
  else if (fr > 1.0f) fr = 1.0f;
  return interp_time(fr, tprev, ti);
}

// Sub-frames per pass of the step kernel for a tile shape: each pass lists the sources
// once, reads each listed source once and has two barriers, and holds a pair of z-buffers
// per sub-frame in shared memory.  More where the extra pairs still leave the shape's
// resident CTAs their shared memory: four for 64 x 16 tiles (with a smaller event stage),
// three for 32 x 32 and for 32 x 16 (with a 512-event stage, keeping four CTAs per SM).
// 96 environments of 640 x 480, K = 32, 64 x 16 tiles: 28.99 ms per gap one sub-frame at a
// time, 23.87 ms in pairs, 22.12 ms in threes; with the later emission and timestamp
// changes 20.91 ms in threes and 19.82 ms in fours.  64 environments of 346 x 260, K = 16,
// 32 x 16 tiles: 2.87 ms in pairs, 2.81 ms in threes.  Colour
// (three channels' state in registers) runs one sub-frame per pass: 64 environments of
// 346 x 260, 64 x 16 tiles, 8.20 ms per gap against 8.88 in pairs and 9.13 in threes.
template <int TX, int TY, int NC>
__host__ __device__ constexpr int step_pass() {
  return NC == 3 ? 1 : ((TX == 64 && TY == 16) ? 4 : ((TX == 32 && (TY == 32 || TY == 16)) ? 3 : 2));
}

// Threads of one step CTA for a tile shape: one target per thread for 32 x 16 and 64 x 16,
// two for 32 x 32 (measured on 64 environments of 346 x 260: 3.59 ms per gap for 32 x 16 at
// 512 threads and four CTAs per SM, against 3.75 ms at 256 threads and six), 256 threads
// for the other shapes.
template <int TX, int TY>
__host__ __device__ constexpr int step_threads() {
  return (TX == 32 && (TY == 16 || TY == 32)) ? 512 : ((TX == 64 && TY == 16) ? 1024 : kThreads);
}

// Events staged in shared memory per CTA and pass (more go to global memory one warp
// reservation at a time): two per target up to 2048, 1024 for the largest tiles and for
// passes of four sub-frames, 512 for 32 x 16 tiles in passes of three, whose shared memory
// would otherwise cost resident CTAs.  On 32 x 346x260 environments (K=16,
// 0.72 events per pixel-substep) 1 % of the emission chunks of 32 x 16 tiles then overflow
// the stage, against 16 % with 512 events.
template <int TX, int TY, int NP>
__host__ __device__ constexpr int step_stage() {
  return (TX == 32 && TY == 16 && NP == 3) ? 512 : ((TX * TY >= 2048 || NP >= 4) ? 1024 : (2 * TX * TY < kEventStage ? kEventStage : 2 * TX * TY));
}

// Dynamic shared memory of one step CTA with passes of NP sub-frames.
template <int TX, int TY, int NP>
struct StepSmem {
  unsigned long long zb[NP][2][TX * TY];   // per sub-frame of a pass: A forward, B backward
  ulonglong2 stage[step_stage<TX, TY, NP>()];  // events of this pass before the flush
  uint2 cand_b[2][kCandidates];            // candidate segments' motion bounds, as half2 pairs
                                           // (min dx, max dx), (min dy, max dy) rounded outward
  unsigned cand_xy[2][kCandidates];        // candidate segments (row << 16 | column)
  unsigned short full[2 * kCandidates];    // segments splat whole this sub-frame (candidate)
  unsigned short items[kSplatItems];       // other sources to splat: candidate | lane << 10
  unsigned ovf[kSplatOverflow];            // candidates beyond the item list: c | lo << 16 | hi << 24
  int64_t rt[step_threads<TX, TY>() / 32][32];           // per warp: crossing times of one chunk
  unsigned char rkeep[step_threads<TX, TY>() / 32][32];  // per warp: refractory decisions of one chunk
};

// Resident CTAs per SM each tile shape is compiled for (bounded by its shared memory); it
// sets the register budget.  Targets per thread NT decide the resident threads: 2048 (64
// warps, 32 registers) for one target per thread in CTAs of 512 or more threads, 1536 (48
// warps, 40 registers) for one or two otherwise, 1024 for four, 768 for more.  Colour
// (NC = 3) triples the per-pixel state held in registers; it too runs best with more
// resident threads and some spills than with fewer and none (measured on 64 environments of
// 346 x 260: 64 x 16 tiles at 2048 threads 8.15 ms per gap, 32 x 16 at 1536 threads 8.63 ms;
// before the CTA size followed the tile, six CTAs of 32 x 8 beat four, five tied).
template <int TX, int TY, int NC>
__host__ __device__ constexpr int step_min_blocks() {
  constexpr int nth = step_threads<TX, TY>(), nt = TX * TY / nth;
  return (nt == 1 && nth >= 512 ? 2048
                                : (NC == 1 ? (nt <= 2 ? 1536 : (nt <= 4 ? 1024 : 768))
                                           : (nt <= 1 ? 1536 : (nt <= 2 ? 1024 : 768)))) / nth;
}

// Statistics of one tile in shared memory (the environment's kStat* words).  Warps add
// their counts of a sub-frame to 32-bit words with one atomic each (every count of a
// sub-frame stays below 2^16); the warp that closes the sub-frame folds them into the tile's
// 64-bit totals, which go to the environment's words once per tile.
struct TileStats {
  unsigned holes_ab;     // target-sub-frames without a source of A | without one of B << 16
  unsigned holes_both;   // ... without either
  unsigned pol;          // staged events copied out since the last fold: ON | OFF << 16
  unsigned long long tot[kStatOverLimit];
};

// Folds the per-sub-frame words into the totals (one thread; no warp is between its
// staging or flush and the end of the sub-frame).
__device__ __forceinline__ void fold_stats(TileStats &st) {
  st.tot[kStatHolesA] += st.holes_ab & 0xFFFFu;
  st.tot[kStatHolesB] += st.holes_ab >> 16;
  st.tot[kStatHolesBoth] += st.holes_both;
  st.tot[kStatEventsOn] += st.pol & 0xFFFFu;
  st.tot[kStatEventsOff] += st.pol >> 16;
  st.holes_ab = st.holes_both = st.pol = 0;
}

// A record written to global memory without the stage (the stage was full) counts at once.
__device__ __forceinline__ void count_polarity(TileStats &st, const ulonglong2 &rec) {
  atomicAdd(&st.tot[static_cast<long long>(rec.y) < 0 ? kStatEventsOff : kStatEventsOn], 1ull);
}

// Copies staged records [0, n) to the event buffer from position gbs; with statistics on,
// counts them by polarity (one shared atomic per warp; every lane of a warp then runs the
// same iterations).
template <int TX, int TY, int NP>
__device__ __forceinline__ void flush_stage(const StepSmem<TX, TY, NP> &S, unsigned n,
                                            unsigned long long gbs, const StepArgs &a,
                                            TileStats &st, bool stats, int tid, int nth) {
  if (!stats) {
    for (unsigned r = tid; r < n; r += nth) {
      const unsigned long long gi = gbs + r;
      if (gi < a.capacity) a.events[gi] = S.stage[r];
    }
    return;
  }
  for (unsigned r0 = tid & ~31u; r0 < n; r0 += nth) {
    const unsigned r = r0 + (tid & 31);
    bool off = false;
    if (r < n) {
      const ulonglong2 rec = S.stage[r];
      const unsigned long long gi = gbs + r;
      if (gi < a.capacity) a.events[gi] = rec;
      off = static_cast<long long>(rec.y) < 0;
    }
    const unsigned moff = __ballot_sync(kFull, off);
    if ((tid & 31) == 0) {
      const unsigned k = min(32u, n - r0), koff = static_cast<unsigned>(__popc(moff));
      atomicAdd(&st.pol, (k - koff) | (koff << 16));
    }
  }
}

// Stages the records of the warp's lanes that have emit set (the warp is converged): one
// shared-memory reservation per warp; past the stage's capacity, one global reservation.
template <int TX, int TY, int NP>
__device__ __forceinline__ void stage_warp(StepSmem<TX, TY, NP> &S, unsigned *s_n,
                                           TileStats &st, bool stats, const StepArgs &a,
                                           bool emit, const ulonglong2 &rec, unsigned lanes_below,
                                           int lane) {
  const unsigned m = __ballot_sync(kFull, emit);
  if (m == 0) return;
  const unsigned cnt = static_cast<unsigned>(__popc(m));
  unsigned base = 0;
  unsigned long long gb = 0;
  if (lane == 0) {
    base = atomicAdd(s_n, cnt);
    if (base + cnt > static_cast<unsigned>(step_stage<TX, TY, NP>()))
      gb = atomicAdd(a.ev_count, static_cast<unsigned long long>(
                                     base + cnt - max(base, static_cast<unsigned>(step_stage<TX, TY, NP>()))));
  }
  base = __shfl_sync(kFull, base, 0);
  gb = __shfl_sync(kFull, gb, 0);
  if (emit) {
    const unsigned idx = base + static_cast<unsigned>(__popc(m & lanes_below));
    if (idx < static_cast<unsigned>(step_stage<TX, TY, NP>())) {
      S.stage[idx] = rec;
    } else {
      const unsigned long long gi = gb + (idx - max(base, static_cast<unsigned>(step_stage<TX, TY, NP>())));
      if (gi < a.capacity) a.events[gi] = rec;
      if (stats) count_polarity(st, rec);
    }
  }
}

// All K sub-frames of one target tile (the body of step_kernel).  NC = 3 runs the event
// model on the R, G and B planes (Sec. 3.2), NC = 1 on the one log-intensity plane.
template <int TX, int TY, bool TRACE, bool PACKED, int NC, bool STATS>
__device__ __forceinline__ void run_tile(const StepArgs &a, const Tile tl) {
  constexpr int NTH = step_threads<TX, TY>();
  constexpr int NT = TX * TY / NTH;        // targets per thread
  constexpr int NW = NTH / 32;
  constexpr int ROWS = NTH / TX;           // tile rows covered by one pass of the block
  constexpr int NP = step_pass<TX, TY, NC>();  // sub-frames per pass
  constexpr unsigned NSTAGE = step_stage<TX, TY, NP>();
  static_assert(TX % 32 == 0 && NTH % TX == 0 && NT * NTH == TX * TY, "tile shape");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  StepSmem<TX, TY, NP> &S = *reinterpret_cast<StepSmem<TX, TY, NP> *>(smem_raw);
  __shared__ unsigned s_n, s_flush, s_nitems[2], s_novf[2], s_nfull[2], s_p1[2], s_arrive;
  __shared__ unsigned long long s_base;
  __shared__ TileStats tstat;  // this tile's statistics
  __shared__ float s_fs[2][NP], s_gs[2][NP];  // the pass's fractions f and 1 - f
  __shared__ int s_nc[2], s_over, s_ovf_full[2];

  const DevEnv E = a.envs[tl.env];
  const int W = E.W, H = E.H, K = E.K;
  const int64_t o = E.pix_off;
  const float *__restrict__ LA = a.LA + o;
  const float *__restrict__ LB = a.LB + o;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned lanes_below = (1u << lane) - 1u;
  const bool b_primary = (a.flags & EVIS_MODE_B_PRIMARY) != 0;
  const bool joint = (a.flags & EVIS_MODE_JOINT) != 0;
  const bool stats = STATS && a.stats;  // the plain variant compiles no statistics code
  const int64_t T0 = a.clock_in[tl.env];
  const int64_t refr = E.refractory_ns;
  const int tx = tl.x0 + tid % TX;
  const int ty0 = tl.y0 + tid / TX;
  const int64_t HW = static_cast<int64_t>(W) * H;
  TileBox box = {tl.x0, tl.y0, min(TX, W - tl.x0), min(TY, H - tl.y0), 0.0f, 0.0f, 0.0f, 0.0f};
  box.qxl = static_cast<float>(box.x0 - 1);
  box.qxh = static_cast<float>(box.x0 + box.nx);
  box.qyl = static_cast<float>(box.y0 - 1);
  box.qyh = static_cast<float>(box.y0 + box.ny);

  // per-pixel event state of this thread's targets (rows ty0 + ROWS j), in registers for
  // the whole keyframe gap
  float Lref[NT][NC], Lprev[NT][NC];  // thresholds are read at use (constants or the maps)
  int64_t tprev[NT], tlast[NT][NC];
  bool act[NT];
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    const int ty = ty0 + ROWS * j;
    const int pix = ty * W + tx;
    act[j] = tx < W - E.margin && ty < H - E.margin;  // tiles start inside the margin
    tprev[j] = T0;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      tlast[j][c] = kNoEvent;
      Lref[j][c] = 0.0f;
      Lprev[j][c] = 0.0f;
      if (act[j]) {
        Lref[j][c] = a.Lref[c * a.plane + o + pix];
        Lprev[j][c] = LA[c * a.plane + pix];
        if (a.tlast) tlast[j][c] = a.tlast[c * a.plane + o + pix];
      }
    }
  }

  // Sources that can reach the tile lie within the largest |mv| (+ footprint) of it.
  const float mf = fmaxf(a.flowA[tl.env], a.flowB[tl.env]);
  const int h = mf < 65536.0f ? static_cast<int>(ceilf(mf)) + 2 : 65536;
  const int sx0 = max(0, tl.x0 - h), sx1 = min(W, tl.x0 + TX + h);
  const int sy0 = max(0, tl.y0 - h), sy1 = min(H, tl.y0 + TY + h);
  if (tid == 0) {
    s_n = 0;
    s_flush = 0;
    s_base = 0;
    s_nitems[0] = s_nitems[1] = 0;
    s_novf[0] = s_novf[1] = 0;
    s_nfull[0] = s_nfull[1] = 0;
    s_p1[0] = s_p1[1] = 0;
    s_ovf_full[0] = s_ovf_full[1] = 0;
    s_arrive = 0;
    s_nc[0] = s_nc[1] = 0;
    s_over = 0;
  }
  if (tid < kStatOverLimit) tstat.tot[tid] = 0;
  if (tid == 0) tstat.holes_ab = tstat.holes_both = tstat.pol = 0;
  // z-buffers start empty; afterwards each thread clears its own slots once it has read them
#pragma unroll
  for (int j = 0; j < NT; ++j) {
#pragma unroll
    for (int u = 0; u < NP; ++u) {
      S.zb[u][0][tid + NTH * j] = kEmptyKey;
      S.zb[u][1][tid + NTH * j] = kEmptyKey;
    }
  }
  __syncthreads();

  // Candidate row segments for this keyframe gap: those whose motion bounds let them reach
  // the tile at some f in [0, 1].  A full list falls back to scanning the whole region.
  {
    const int cx_lo = sx0 / kSegW, cx_hi = (sx1 - 1) / kSegW;
    const int ncx = cx_hi - cx_lo + 1;
    const int nreg = ncx * (sy1 - sy0);
    for (int r = tid; r < 2 * nreg; r += NTH) {
      const int dir = r >= nreg ? 1 : 0;
      const int rr = r - dir * nreg;
      const int row = rr / ncx;
      const int cy = sy0 + row, cx = cx_lo + (rr - row * ncx);
      const float4 b = (dir ? a.segB : a.segA)[E.seg_off + static_cast<int64_t>(cy) * E.segs_x + cx];
      if (!(b.x <= b.y)) continue;  // no source of this segment can splat
      float dxl, dxh, dyl, dyh;     // displacement range over f in [0, 1]
      if (dir == 0) {
        dxl = fminf(0.0f, -b.y); dxh = fmaxf(0.0f, -b.x);
        dyl = fminf(0.0f, -b.w); dyh = fmaxf(0.0f, -b.z);
      } else {
        dxl = fminf(0.0f, b.x); dxh = fmaxf(0.0f, b.y);
        dyl = fminf(0.0f, b.z); dyh = fmaxf(0.0f, b.w);
      }
      if (seg_misses<TX, TY>(static_cast<float>(cx * kSegW), static_cast<float>(cy), dxl, dxh,
                             dyl, dyh, tl.x0, tl.y0))
        continue;
      const int pos = atomicAdd(&s_nc[dir], 1);
      if (pos < kCandidates) {
        S.cand_xy[dir][pos] = (static_cast<unsigned>(cy) << 16) | static_cast<unsigned>(cx);
        // outward rounding keeps the bounds conservative (overflow goes to +-inf)
        const __half2 bx = __halves2half2(__float2half_rd(b.x), __float2half_ru(b.y));
        const __half2 by = __halves2half2(__float2half_rd(b.z), __float2half_ru(b.w));
        S.cand_b[dir][pos] = make_uint2(*reinterpret_cast<const unsigned *>(&bx),
                                        *reinterpret_cast<const unsigned *>(&by));
      } else {
        s_over = 1;
      }
    }
  }
  __syncthreads();
  const bool over = s_over != 0;
  const int nA = min(s_nc[0], kCandidates);
  const int nAB = nA + min(s_nc[1], kCandidates);
  // t_i = T0 + floor(i dt / K), stepped with a quotient and a remainder
  const int64_t dq = a.dt / K;
  const int dr = static_cast<int>(a.dt % K);  // remainders stay below K <= 4096
  int64_t tq = 0;
  int trem = 0;

  // Sub-frames are processed in passes of NP (i0 .. i0 + ns - 1; the last pass may hold
  // fewer): one source list serves them all, each listed source is read once and splat at
  // every f of the pass into that sub-frame's pair of z-buffers, and the pass has two
  // barriers.
  for (int i0 = 1; i0 <= K; i0 += NP) {
    const int ns = min(NP, K - i0 + 1);
    // The pass's fractions f and 1 - f (past ns: the last sub-frame's again, which extends
    // no bound), in shared memory (double-buffered by pass parity) for phase 3 of every
    // pass, which then divides no more (2.76 -> 2.74 ms on 64 x 346x260).  The splat reads
    // them there for passes of up to three, which frees registers through it (64 x 346x260,
    // 32 x 16 tiles: 2.82 -> 2.76 ms), and from registers for passes of four (96 x 640x480,
    // 64 x 16: 19.80 against 19.96).
    const int par = ((i0 - 1) / NP) & 1;
    constexpr bool kSharedF = NP <= 3;
    float fs[NP], gs[NP];
#pragma unroll
    for (int u = 0; u < NP; ++u) {
      fs[u] = __fdiv_rn(static_cast<float>(min(i0 + u, K)), static_cast<float>(K));
      gs[u] = __fsub_rn(1.0f, fs[u]);
    }
    if (tid < NP) {
#pragma unroll
      for (int u = 0; u < NP; ++u)
        if (u == tid) {
          s_fs[par][u] = fs[u];
          s_gs[par][u] = gs[u];
        }
    }
    const float f1 = fs[0], g1 = gs[0], f2 = fs[NP - 1], g2 = gs[NP - 1];
    const float *pfs = kSharedF ? s_fs[par] : fs;
    const float *pgs = kSharedF ? s_gs[par] : gs;

    // Phase 1 (list reaching candidates) may overlap other warps' phase 3 of the previous
    // pass; the hit list is double-buffered by parity.
    // ---- phase 1: list the sources that can reach the tile at some f of the pass (f1 to f2):
    // for each candidate segment whose motion bounds reach the tile, the interval of its lanes
    // (sources) whose displaced position can put a footprint pixel into the tile; the
    // sources go into one flat list so that every lane of phase 2 splats a source that may
    // land ----
    if (!over) {
      // warps take chunks of 32 candidates from a counter: those that finish the previous
      // sub-frame's emission first do more of this phase
      for (;;) {
        unsigned cb = 0;
        if (lane == 0) cb = atomicAdd(&s_p1[par], 32u);
        cb = __shfl_sync(kFull, cb, 0);
        if (cb >= static_cast<unsigned>(nAB)) break;
        const int c = static_cast<int>(cb) + lane;
        int lo = 0, cnt = 0;
        if (c < nAB) {
          const int dir = c >= nA ? 1 : 0;
          const int idx = c - dir * nA;
          const uint2 hb = S.cand_b[dir][idx];
          const float2 bx = __half22float2(*reinterpret_cast<const __half2 *>(&hb.x));
          const float2 by = __half22float2(*reinterpret_cast<const __half2 *>(&hb.y));
          const float4 b = make_float4(bx.x, bx.y, by.x, by.y);
          const unsigned xy = S.cand_xy[dir][idx];
          // displacement bounds at the pass's first and last f (the products are monotone in
          // f and in the motion, so the corners enclose every rounded displacement; an
          // infinite bound times g = 0 is NaN and leaves the other corner, itself infinite)
          float dxl, dxh, dyl, dyh;
          if (dir == 0) {
            dxl = fminf(-f1 * b.y, -f2 * b.y); dxh = fmaxf(-f1 * b.x, -f2 * b.x);
            dyl = fminf(-f1 * b.w, -f2 * b.w); dyh = fmaxf(-f1 * b.z, -f2 * b.z);
          } else {
            dxl = fminf(g1 * b.x, g2 * b.x); dxh = fmaxf(g1 * b.y, g2 * b.y);
            dyl = fminf(g1 * b.z, g2 * b.z); dyh = fmaxf(g1 * b.w, g2 * b.w);
          }
          const int xs = static_cast<int>(xy & 0xFFFFu) * kSegW;
          const float xsf = small_int_to_float(xs);
          if (!seg_misses<TX, TY>(xsf, small_int_to_float(static_cast<int>(xy >> 16)), dxl, dxh,
                                  dyl, dyh, tl.x0, tl.y0)) {
            // a source x can reach only if x + dxh > x0 - 1 and x + dxl < x0 + TX (its
            // footprint spans floor(q) and floor(q) + 1); a quarter pixel more on each side
            // covers the rounding of these sums.  NaN bounds keep every lane.
            const float flo = ceilf(static_cast<float>(tl.x0) - 1.25f - dxh - xsf);
            const float fhi = ceilf(static_cast<float>(tl.x0 + TX) + 0.25f - dxl - xsf);
            lo = flo > 0.0f ? (flo < 32.0f ? static_cast<int>(flo) : 32) : 0;
            int hi = fhi < 32.0f ? (fhi > 0.0f ? static_cast<int>(fhi) : 0) : 32;
            hi = min(hi, W - xs);
            cnt = max(0, hi - lo);
          }
        }
        // a segment whose 32 sources all may land goes to the list of whole segments (32
        // consecutive slots of phase 2's flat index); the sources of the others are listed
        // one by one
        const bool whole = cnt == 32;
        {
          const unsigned wm = __ballot_sync(kFull, whole);
          if (wm) {
            unsigned fb = 0;
            if (lane == 0) fb = atomicAdd(&s_nfull[par], static_cast<unsigned>(__popc(wm)));
            fb = __shfl_sync(kFull, fb, 0);
            if (whole) S.full[fb + __popc(wm & lanes_below)] = static_cast<unsigned short>(c);
          }
        }
        if (whole) cnt = 0;
        // allocate the warp's items (a scan of the counts, one atomic) and write them
        // cooperatively; what does not fit goes to the overflow list, one entry per segment
        int incl = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int v = __shfl_up_sync(kFull, incl, d);
          if (lane >= d) incl += v;
        }
        const int wtot = __shfl_sync(kFull, incl, 31);
        if (wtot == 0) continue;
        unsigned wbase = 0;
        if (lane == 0) wbase = atomicAdd(&s_nitems[par], static_cast<unsigned>(wtot));
        wbase = __shfl_sync(kFull, wbase, 0);
        const int excl = incl - cnt;
        // items that fit in the list (uniform over the warp: every lane shuffles)
        const int lim = wbase >= static_cast<unsigned>(kSplatItems)
                            ? 0 : min(wtot, kSplatItems - static_cast<int>(wbase));
        for (int j0 = 0; j0 < lim; j0 += 32) {
          const int j = j0 + lane;
          int own = 0;  // the lane whose interval holds item j
#pragma unroll
          for (int st = 16; st > 0; st >>= 1) {
            const int v = __shfl_sync(kFull, incl, own + st - 1);
            if (v <= j) own += st;
          }
          own = min(own, 31);
          const int oc = __shfl_sync(kFull, c, own);
          const int olo = __shfl_sync(kFull, lo, own);
          const int oex = __shfl_sync(kFull, excl, own);
          if (j < lim) S.items[wbase + j] = static_cast<unsigned short>(oc | ((olo + j - oex) << 10));
        }
        const unsigned my_start = wbase + static_cast<unsigned>(excl);
        if (cnt > 0 && my_start + cnt > static_cast<unsigned>(kSplatItems)) {
          const int skip = my_start < static_cast<unsigned>(kSplatItems)
                               ? static_cast<int>(kSplatItems - my_start) : 0;
          const unsigned pos = atomicAdd(&s_novf[par], 1u);
          if (pos < static_cast<unsigned>(kSplatOverflow))
            S.ovf[pos] = static_cast<unsigned>(c) | (static_cast<unsigned>(lo + skip) << 16) |
                         (static_cast<unsigned>(lo + cnt) << 24);
          else
            s_ovf_full[par] = 1;
        }
      }
    }
    __syncthreads();

    // ---- phase 2: flush the previous pass's staged events (reserved by the last warp to
    // finish it), then splat both directions at every sub-frame of the pass (Eq. 5 targets,
    // Eq. 7 depth, Eq. 6 z-test) ----
    if (tid == 0) {
      s_nitems[par ^ 1] = 0;
      s_novf[par ^ 1] = 0;
      s_nfull[par ^ 1] = 0;
      s_p1[par ^ 1] = 0;
      s_ovf_full[par ^ 1] = 0;
    }
    flush_stage(S, s_flush, s_base, a, tstat, stats, tid, NTH);
    if (!over && !s_ovf_full[par]) {
      // one flat index space, one source per thread: the whole segments' sources first
      // (item it -> segment it / 32, lane it % 32), then the listed sources
      const unsigned nwh = s_nfull[par] * 32u;
      const unsigned ni = nwh + min(s_nitems[par], static_cast<unsigned>(kSplatItems));
      for (unsigned it = tid; it < ni; it += NTH) {
        int c, l;
        if (it < nwh) {
          c = static_cast<int>(S.full[it >> 5]);
          l = static_cast<int>(it & 31u);
        } else {
          const unsigned v = S.items[it - nwh];
          c = static_cast<int>(v & 1023u);
          l = static_cast<int>(v >> 10);
        }
        const int dir = c >= nA ? 1 : 0;
        const unsigned xy = S.cand_xy[dir][c - dir * nA];
        const int sx = static_cast<int>(xy & 0xFFFFu) * kSegW + l, sy = static_cast<int>(xy >> 16);
        splat_source<TX, TY, NP, PACKED>(S.zb, dir, sx, sy, small_int_to_float(sx),
                                         small_int_to_float(sy), W, H, box, pfs, pgs, ns, a, o);
      }
      const unsigned no = min(s_novf[par], static_cast<unsigned>(kSplatOverflow));
      for (unsigned e = warp; e < no; e += NW) {  // overflow: one warp per segment
        const unsigned v = S.ovf[e];
        const int c = static_cast<int>(v & 0xFFFFu);
        const int lo = static_cast<int>((v >> 16) & 0xFFu), hi = static_cast<int>(v >> 24);
        const int dir = c >= nA ? 1 : 0;
        const unsigned xy = S.cand_xy[dir][c - dir * nA];
        const int sx = static_cast<int>(xy & 0xFFFFu) * kSegW + lane, sy = static_cast<int>(xy >> 16);
        if (lane >= lo && lane < hi)
          splat_source<TX, TY, NP, PACKED>(S.zb, dir, sx, sy, small_int_to_float(sx),
                                           small_int_to_float(sy), W, H, box, pfs, pgs, ns, a, o);
      }
    } else {  // the candidate or overflow lists were full: every source of the region
      for (int sy = sy0 + warp; sy < sy1; sy += NW) {
        const float fy = small_int_to_float(sy);
        for (int sx = sx0 + lane; sx < sx1; sx += 32) {
          const float fx = small_int_to_float(sx);
          splat_source<TX, TY, NP, PACKED>(S.zb, 0, sx, sy, fx, fy, W, H, box, pfs, pgs, ns, a, o);
          splat_source<TX, TY, NP, PACKED>(S.zb, 1, sx, sy, fx, fy, W, H, box, pfs, pgs, ns, a, o);
        }
      }
    }
    __syncthreads();

    // ---- phase 3, per sub-frame of the pass: resolve, blend, threshold crossings, emission
    // (per channel: the winners depend on motion and depth only, so one resolve serves all
    // NC channels) ----
#pragma unroll 1
    for (int u = 0; u < ns; ++u) {
    const int i = i0 + u;
    const float f = s_fs[par][u], g = s_gs[par][u];   // i / K and 1 - i / K
    tq += dq;
    trem += dr;
    if (trem >= K) {
      trem -= K;
      ++tq;
    }
    const int64_t ti = T0 + tq;
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const int ty = ty0 + ROWS * j;
      const int pix = ty * W + tx;
      // sensor (x | y << 16) of the warp's first target; its lanes add their index
      const unsigned ev_xy = static_cast<unsigned>(tl.x0 - E.margin + (warp * 32) % TX) |
                             (static_cast<unsigned>(ty - E.margin) << 16);
      unsigned long long kA = kEmptyKey, kB = kEmptyKey;  // read at channel 0
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        bool has = false;
        float L = 0.0f, th = E.c_on, nf = 0.0f;
        int n = 0, pol = 1;
        if (act[j]) {
          if (c == 0) {
            kA = S.zb[u][0][tid + NTH * j];
            kB = S.zb[u][1][tid + NTH * j];
            S.zb[u][0][tid + NTH * j] = kEmptyKey;  // ready for the next pass
            S.zb[u][1][tid + NTH * j] = kEmptyKey;
          }
          const bool hasA = kA != kEmptyKey, hasB = kB != kEmptyKey;
          const float la = hasA ? __ldg(LA + c * a.plane + (kA & 0xFFFFFFull)) : 0.0f;
          const float lb = hasB ? __ldg(LB + c * a.plane + (kB & 0xFFFFFFull)) : 0.0f;
          if (joint) {  // Eq. 6: the nearer winner; equal depths go to B
            L = (hasA && hasB) ? ((kA >> 32) < (kB >> 32) ? la : lb)
                               : (hasA ? la : (hasB ? lb : __int_as_float(0x7fc00000)));
          } else if (b_primary) {
            L = hasB ? lb : (hasA ? la : __int_as_float(0x7fc00000));
          } else {
            L = (hasA && hasB) ? __fadd_rn(__fmul_rn(g, la), __fmul_rn(f, lb))
                               : (hasA ? la : (hasB ? lb : __int_as_float(0x7fc00000)));
          }
          if (TRACE) {
            if (c == 0) {
              const int64_t kb = a.tr_koff[tl.env] + static_cast<int64_t>(i - 1) * 2 * HW + pix;
              a.tr_keys[kb] = kA;
              a.tr_keys[kb + HW] = kB;
            }
            a.tr_L[a.tr_loff[tl.env] + (static_cast<int64_t>(i - 1) * NC + c) * HW + pix] = L;
          }
          has = hasA || hasB;  // no sample: the pixel holds its state this sub-frame
          if (has) {
            const float d = __fsub_rn(L, Lref[j][c]);
            pol = d > 0.0f ? 1 : -1;
            // Eq. 8 thresholds: the environment's, or its per-pixel maps (read through L1)
            th = E.con_map ? __ldg((pol > 0 ? E.con_map : E.coff_map) + pix)
                           : (pol > 0 ? E.c_on : E.c_off);
            const float q = __fdiv_rn(fabsf(d), th);
            if (q >= 1.0f) {
              if (q < static_cast<float>(kMaxCrossings + 1)) {
                n = floor_small(q, &nf);
              } else {  // n of Eq. 4 above the emission limit: none emitted, counted
                nf = floorf(q);
                atomicAdd(a.ev_count + 1, 1ull);
                if (a.env_stats)
                  atomicAdd(a.env_stats + static_cast<int64_t>(tl.env) * kStatWords + kStatOverLimit, 1ull);
              }
            }
          }
        }
        if (c == 0 && stats) {  // holes per warp direction (statistics)
          const unsigned ha = __ballot_sync(kFull, act[j] && kA == kEmptyKey);
          const unsigned hb = __ballot_sync(kFull, act[j] && kB == kEmptyKey);
          if (lane == 0 && (ha | hb)) {
            atomicAdd(&tstat.holes_ab, static_cast<unsigned>(__popc(ha)) |
                                        (static_cast<unsigned>(__popc(hb)) << 16));
            if (ha & hb) atomicAdd(&tstat.holes_both, static_cast<unsigned>(__popc(ha & hb)));
          }
        }
        // ---- crossings k = 1..n of the warp's 32 pixels ----
        // When no pixel of the warp has more than one crossing, each lane emits its own
        // (measured on 640x480, K = 32: 22.1 -> 21.1 ms per gap of 96 environments; letting
        // lanes walk two or three crossings each is slower than spreading them).
        const int maxn = __reduce_max_sync(kFull, n);
        if (maxn <= 1) {
          if (maxn == 1) {
            bool emit = n == 1;
            int64_t t = 0;
            if (emit) {
              t = crossing_time(Lref[j][c], pol > 0 ? 1.0f : -1.0f, th, Lprev[j][c], L, tprev[j], ti);
              if (a.tlast) {  // refractory filter against the pixel's last kept time
                emit = refr <= 0 || tlast[j][c] == kNoEvent || t - tlast[j][c] >= refr;
                if (emit) tlast[j][c] = t;
              }
            }
            ulonglong2 rec;
            rec.x = static_cast<unsigned long long>(t);
            rec.y = static_cast<unsigned long long>(ev_xy + static_cast<unsigned>(lane)) |
                    (static_cast<unsigned long long>(
                         (static_cast<unsigned>(tl.env) & 0xFFFFu) |
                         (static_cast<unsigned>(static_cast<uint16_t>(static_cast<int16_t>(pol * (1 + c)))) << 16))
                     << 32);
            stage_warp<TX, TY, NP>(S, &s_n, tstat, stats, a, emit, rec, lanes_below, lane);
          }
        } else {
        // Otherwise item c of the warp (pixels in lane order, k ascending) is computed by lane
        // c % 32.
        int incl = n;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int v = __shfl_up_sync(kFull, incl, d);
          if (lane >= d) incl += v;
        }
        const int total = __shfl_sync(kFull, incl, 31);
        const int excl = incl - n;
        for (int c0 = 0; c0 < total; c0 += 32) {
          const int it = c0 + lane;
          // owner = number of lanes whose items all lie before it
          int own = 0;
#pragma unroll
          for (int st = 16; st > 0; st >>= 1) {
            const int v = __shfl_sync(kFull, incl, own + st - 1);
            if (v <= it) own += st;
          }
          own = min(own, 31);
          const int k = it - __shfl_sync(kFull, excl, own) + 1;
          const float oL = __shfl_sync(kFull, L, own);
          const float oLref = __shfl_sync(kFull, Lref[j][c], own);
          const float oLprev = __shfl_sync(kFull, Lprev[j][c], own);
          const float oth = __shfl_sync(kFull, th, own);
          const int opol = __shfl_sync(kFull, pol, own);
          const int64_t otprev = __shfl_sync(kFull, tprev[j], own);
          int64_t t = 0;
          if (it < total) {
            const float kf = small_int_to_float(k);
            t = crossing_time(oLref, opol > 0 ? kf : -kf, oth, oLprev, oL, otprev, ti);
          }
          bool emit = it < total;
          if (a.tlast) {
            // refractory filter (Sec. 3.4): greedy along each pixel's crossings, t_last
            // carried over chunks.  Fast path: if every item clears the last kept time of
            // its pixel under the assumption that its predecessors in the chunk were kept
            // (a pixel's first item here against t_last, the others against the item just
            // before them), then by induction the greedy filter keeps them all.
            const int64_t t_before = __shfl_up_sync(kFull, t, 1);
            const int64_t otl = __shfl_sync(kFull, tlast[j][c], own);
            const bool first = k == 1 || lane == 0;  // no earlier item of its pixel in the chunk
            const bool ok = it >= total || refr <= 0 || (first && otl == kNoEvent) ||
                            t - (first ? otl : t_before) >= refr;
            if (__all_sync(kFull, ok)) {
              // all kept: each pixel's t_last is its last item's time in this chunk
              const int last = min(incl, c0 + 32) - 1 - c0;
              const int64_t tl_new = __shfl_sync(kFull, t, min(max(last, 0), 31));
              if (n > 0 && incl > c0 && excl < c0 + 32) tlast[j][c] = tl_new;
            } else {
              // each owner walks its items of this chunk in order
              S.rt[warp][lane] = t;
              __syncwarp();
              const int lo = max(excl, c0), hi = min(incl, c0 + 32);
              for (int cc = lo; cc < hi; ++cc) {
                const int64_t tt = S.rt[warp][cc - c0];
                const bool keep = refr <= 0 || tlast[j][c] == kNoEvent || tt - tlast[j][c] >= refr;
                if (keep) tlast[j][c] = tt;
                S.rkeep[warp][cc - c0] = keep ? 1 : 0;
              }
              __syncwarp();
              emit = emit && S.rkeep[warp][lane] != 0;
            }
          }
          const unsigned m = __ballot_sync(kFull, emit);
          if (m == 0) continue;
          const unsigned cnt = static_cast<unsigned>(__popc(m));
          unsigned base = 0;
          if (lane == 0) base = atomicAdd(&s_n, cnt);
          base = __shfl_sync(kFull, base, 0);
          const unsigned idx = base + static_cast<unsigned>(__popc(m & lanes_below));
          // the warp's 32 targets are consecutive pixels of one row: the owner's sensor x
          // is the warp's first x plus its lane (below 2^16, so the add stays in its field)
          ulonglong2 rec;
          rec.x = static_cast<unsigned long long>(t);
          rec.y = static_cast<unsigned long long>(ev_xy + static_cast<unsigned>(own)) |
                  (static_cast<unsigned long long>(
                       (static_cast<unsigned>(tl.env) & 0xFFFFu) |
                       (static_cast<unsigned>(static_cast<uint16_t>(static_cast<int16_t>(opol * (1 + c)))) << 16))
                   << 32);
          if (base + cnt <= NSTAGE) {  // (uniform) the chunk fits in the stage
            if (emit) S.stage[idx] = rec;
          } else {  // staging full: what does not fit goes to global memory directly
            unsigned long long gb = 0;
            if (lane == 0)
              gb = atomicAdd(a.ev_count, static_cast<unsigned long long>(base + cnt - max(base, NSTAGE)));
            gb = __shfl_sync(kFull, gb, 0);
            if (emit) {
              if (idx < NSTAGE) {
                S.stage[idx] = rec;
              } else {
                const unsigned long long gi = gb + (idx - max(base, NSTAGE));
                if (gi < a.capacity) a.events[gi] = rec;
                if (stats) count_polarity(tstat, rec);
              }
            }
          }
          __syncwarp();  // the next chunk reuses this warp's refractory scratch
        }
        }  // crossings spread over the lanes
        if (has) {
          if (nf > 0.0f) Lref[j][c] = __fadd_rn(Lref[j][c], __fmul_rn(pol > 0 ? nf : -nf, th));
          Lprev[j][c] = L;
          if (c == NC - 1) tprev[j] = ti;  // after every channel's crossings used it
        }
      }
    }
    }  // sub-frames of the pass
    // ---- end of phase 3: the last warp to finish reserves the global range of this
    // pass's staged events (one atomic per CTA); they are copied out in phase 2 of the next
    // pass, or after the loop ----
    __syncwarp();
    if (lane == 0) {
      __threadfence_block();
      if (atomicAdd(&s_arrive, 1u) == static_cast<unsigned>(NW - 1)) {
        const unsigned nn = min(s_n, NSTAGE);
        s_flush = nn;
        s_base = nn ? atomicAdd(a.ev_count, static_cast<unsigned long long>(nn)) : 0ull;
        s_n = 0;
        s_arrive = 0;
        if (stats) fold_stats(tstat);
      }
    }
  }
  __syncthreads();
  flush_stage(S, s_flush, s_base, a, tstat, stats, tid, NTH);
  __syncthreads();  // the statistics words are complete

#pragma unroll
  for (int j = 0; j < NT; ++j) {
    if (!act[j]) continue;
    const int pix = (ty0 + ROWS * j) * W + tx;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      a.Lref[c * a.plane + o + pix] = Lref[j][c];
      if (a.tlast) a.tlast[c * a.plane + o + pix] = tlast[j][c];
    }
  }
  if (tid == 0 && stats) {
    fold_stats(tstat);  // the last stage's copy
    for (int w = 0; w < kStatOverLimit; ++w)
      if (tstat.tot[w])
        atomicAdd(a.env_stats + static_cast<int64_t>(tl.env) * kStatWords + w, tstat.tot[w]);
  }
  if (tid == 0 && tl.x0 == E.margin && tl.y0 == E.margin) {  // the environment's first tile
    a.clock_out[tl.env] = T0 + a.dt;
    if (a.gap_out) a.gap_out[tl.env] = a.gap_in[tl.env] + 1u;
  }
}

// One CTA per resident slot; CTAs take tiles from the list in order (largest K first), the
// first one by block index, the next ones from a work counter that starts at 0.
template <int TX, int TY, bool TRACE, bool PACKED, int NC, bool STATS>
__global__ void __launch_bounds__(step_threads<TX, TY>(), step_min_blocks<TX, TY, NC>())
    step_kernel(const StepArgs a) {
  __shared__ int s_tile;
  int t = blockIdx.x;
  while (t < a.n_tiles) {
    run_tile<TX, TY, TRACE, PACKED, NC, STATS>(a, a.tiles[t]);
    __syncthreads();  // the tile's shared memory is free again
    if (threadIdx.x == 0) s_tile = static_cast<int>(gridDim.x + atomicAdd(a.work_counter, 1u));
    __syncthreads();
    t = s_tile;
  }
}

}  // namespace

template <int TX, int TY, bool TRACE, bool PACKED, int NC, bool STATS>
cudaError_t launch_shape(const StepArgs &a, int n_tiles, int grid_cap, cudaStream_t s) {
  // per device (the shared-memory attribute belongs to the device's context): resident CTAs
  // per SM x SMs, looked up at the first launch of this instantiation on that device
  constexpr int kMaxDevices = 64;
  static std::atomic<int> resident_of[kMaxDevices];
  const int smem = static_cast<int>(sizeof(StepSmem<TX, TY, step_pass<TX, TY, NC>()>));
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  int resident = resident_of[dev].load(std::memory_order_relaxed);
  if (!resident) {
    if ((e = cudaFuncSetAttribute(step_kernel<TX, TY, TRACE, PACKED, NC, STATS>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
      return e;
    int sms = 0, per_sm = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
      return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
             &per_sm, step_kernel<TX, TY, TRACE, PACKED, NC, STATS>, step_threads<TX, TY>(),
             smem)) != cudaSuccess)
      return e;
    resident = max(1, per_sm) * sms;
    resident_of[dev].store(resident, std::memory_order_relaxed);
  }
  int grid = n_tiles;
  if (grid_cap > 0) grid = min(grid, grid_cap * resident);  // persistent: a multiple of the SM slots
  step_kernel<TX, TY, TRACE, PACKED, NC, STATS><<<grid, step_threads<TX, TY>(), smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace evis
