// Internal declarations of libevis: device-side tables and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "evis.h"

namespace evis {

constexpr uint64_t kEmptyKey = ~0ull;
// Crossings one pixel may emit per sub-frame (per channel).  A pixel-sub-frame whose Eq. 4
// count n is larger emits none of them, still moves its reference level by the whole p n C,
// and is counted (ev_count[1] and the environment's kStatOverLimit word).
constexpr int kMaxCrossings = 4096;
// Per-environment statistics words (64-bit counters, accumulated by the step kernel).
enum StatWord {
  kStatHolesA = 0,      // target-sub-frames with no source of A (forward warp)
  kStatHolesB = 1,      // ... with no source of B (backward warp)
  kStatHolesBoth = 2,   // ... with neither (no sample)
  kStatEventsOn = 3,    // crossing events emitted with positive polarity
  kStatEventsOff = 4,   // ... negative polarity
  kStatNoise = 5,       // sensor noise events emitted
  kStatOverLimit = 6,   // pixel-sub-frames (per channel) beyond the emission limit
  kStatWords = 8
};
constexpr int64_t kNoEvent = INT64_MIN;     // t_last of a pixel that never fired
constexpr int kThreads = 256;               // threads per step CTA unless its tile shape sets more
constexpr int kEventStage = 512;            // fewest events staged in shared memory per CTA
constexpr int kSegW = 32;                   // motion bounds are kept per 32-pixel row segment
constexpr int kCandidates = 512;            // candidate segments per direction per tile
constexpr int kSplatItems = 1536;           // sources of partial segments listed for a splat
constexpr int kSplatOverflow = 128;         // segments beyond that list, one warp each

// Per-environment constants, resident in device memory.
struct DevEnv {
  int32_t W, H, K, tile_h;
  int64_t pix_off;
  int64_t seg_off;    // first row segment of this environment
  int32_t segs_x;     // row segments per image row
  int32_t margin;     // over-render margin: targets are [margin, W - margin) x [margin, H - margin)
  float c_on, c_off;
  const float *con_map, *coff_map;   // this environment's maps (device) or null
  int64_t refractory_ns;
  // sensor noise (Sec. 3.4); noise == 0 turns it off for this environment
  float leak_hz, shot_hz, hot_hz;   // event rates per pixel (1/s)
  float hot_fraction;               // probability that a pixel is hot
  float noise_lo, noise_hi;         // log-intensity range of the normalised intensity
  uint32_t key0, key1;              // Philox key: seed low word, seed high word ^ env
  int32_t noise, pad1;
  int32_t blur_r, blur_off;         // defocus radius and first weight in the weight table
};

// One target tile: environment and top-left pixel.
struct Tile {
  int32_t env, x0, y0, pad;
};

// Arguments of one step launch (packed base pointers; environment offsets are applied
// inside the kernel).
struct StepArgs {
  const DevEnv *envs;
  const Tile *tiles;          // the tiles of this launch, largest K first
  int n_tiles;
  unsigned *work_counter;     // zeroed before the launch
  const float *LA, *mvA, *ZA;
  const float *LB, *mvB, *ZB;
  float *Lref;
  int64_t *tlast;            // null when no environment has a refractory period
  const int64_t *clock_in;
  int64_t *clock_out;
  const uint32_t *gap_in;    // per environment: keyframe gaps done (the noise counter), or null
  uint32_t *gap_out;
  const float *flowA, *flowB;
  const float4 *segA, *segB;   // per row segment: (min dx, max dx, min dy, max dy)
  const float4 *packA, *packB; // per source: (mx, my, Z, Z at the other endpoint), or null
  ulonglong2 *events;
  unsigned long long *ev_count;    // [0] events produced, [1] pixel-sub-frames beyond the limit
  unsigned long long capacity;
  unsigned long long *env_stats;   // per environment kStatWords counters, or null
  bool stats;                      // collect holes, polarity and noise counts (EVIS_STATS)
  int64_t dt;
  uint32_t flags;
  bool noise;                // some environment of the launch has noise on (launch_noise)
  int nc;                    // event channels: 1, or 3 in colour mode (0 reads as 1)
  int64_t plane;             // channel stride of LA, LB, Lref, tlast (packed pixels)
  uint64_t *tr_keys;         // debug trace (null in the production path)
  float *tr_L;
  const int64_t *tr_koff, *tr_loff;
};

struct PrepArgs {
  const DevEnv *envs;
  const float *frames, *mv, *Z;  // caller's keyframe
  float *L_out;                  // log-intensity destination (null: frames are used as L)
  float *mv_out, *Z_out;         // copies (null under EVIS_KEEP_INPUTS)
  float *flow;                   // per-environment max |mv| (inf-norm), pre-zeroed
  float4 *seg;                   // per row segment motion bounds of this keyframe
  const float *mvA, *ZA;         // previous keyframe (null for the first one)
  float4 *packA, *packB;         // per-source packs of A and B for the gap (null: none)
  float eps;
  uint32_t mode;                 // EVIS_IN_LOG, EVIS_IN_LUM, or EVIS_IN_RGB; with nc = 3 the
                                 // frames are planar log (LOG), planar linear (LUM, what the
                                 // defocus pass writes) or interleaved linear RGB (RGB)
  int nc;                        // planes of L_out: 1, or 3 in colour mode (0 reads as 1)
  int64_t plane;                 // channel stride of frames (planar) and L_out
  int max_segs;                  // largest environment (row segments)
  unsigned long long *invalid;   // per environment: sources that cannot splat, accumulated (or null)
};

constexpr int kMaxBlurR = 24;                 // defocus radius limit (sigma <= 8 px)

// Arguments of the defocus kernel (Sec. 3.4): blurred linear luminance of every environment,
// or of one plane when envs is null (then W, H, r, w describe it).
struct BlurArgs {
  const DevEnv *envs;
  const float *wtab;            // weights of all environments, each at its blur_off
  int W, H, r;                  // the single-plane form
  float w[2 * kMaxBlurR + 1];
  const float *in;              // packed frames: luminance, or RGB triples
  float *out;                   // packed blurred luminance (or nc planes of blurred channels)
  uint32_t mode;                // EVIS_IN_LUM or EVIS_IN_RGB
  int nc;                       // 3: blur each channel of the RGB input into its own plane
  int64_t plane;                // channel stride of out
  int max_r;                    // largest radius of the launch (sizes shared memory)
};

cudaError_t launch_prep(const PrepArgs &a, int n_envs, cudaStream_t s);
// max_tiles: the largest environment's count of 64 x 32 tiles
cudaError_t launch_defocus(const BlurArgs &a, int n_envs, int max_tiles, cudaStream_t s);
cudaError_t launch_init_ref(const float *L, float *Lref, int64_t n, cudaStream_t s);
// One tile shape and variant of the synthesis kernel (defined in evis_step.cuh and
// instantiated in the evis_step_*.cu translation units).
// STATS compiles the statistics code (EVIS_STATS, checked at run time); the plain production
// variant is also built without it.
template <int TX, int TY, bool TRACE, bool PACKED, int NC, bool STATS>
cudaError_t launch_shape(const StepArgs &a, int n_tiles, int grid_cap, cudaStream_t s);

// grid_cap > 0: persistent launch of at most grid_cap x (resident CTAs) blocks that take
// tiles from a.work_counter; 0: one block per tile.
cudaError_t launch_step(const StepArgs &a, int tile_w, int tile_h, bool trace, int grid_cap,
                        cudaStream_t s);
bool tile_shape_supported(int tile_w, int tile_h);
// Sensor noise of one keyframe gap (Sec. 3.4) of every environment with noise on, appended
// to the event buffer.  Reads a.envs, a.LA and a.LB (the gap's prepared log-intensity
// planes), a.clock_in, a.gap_in, a.dt, a.nc, a.plane and writes a.events, a.ev_count and,
// with a.stats, a.env_stats.  max_px: the largest sensor (pixels) of those environments.
cudaError_t launch_noise(const StepArgs &a, int n_envs, int max_px, cudaStream_t s);
// Host-side check that a device pointer is a multiple of align bytes (kernels read motion
// vectors as float2, event records as 16-byte pairs); null counts as aligned.
inline bool aligned(const void *p, size_t align) {
  return reinterpret_cast<uintptr_t>(p) % align == 0;
}
// Error text reported by evis_last_error(NULL) for calls made without a context.
void set_detached_error(const std::string &msg);
cudaError_t launch_log(const float *in, int64_t n, uint32_t mode, float eps, float *out,
                       cudaStream_t s);

}  // namespace evis
