/*
 * evis.h -- C ABI of libevis.so, the CUDA (sm_103a) event-synthesis path of EVIS.
 *
 * The library turns a sequence of rendered keyframes (linear-HDR radiance or log-intensity,
 * the renderer's backward motion vectors and depth) into an event stream.  For every
 * keyframe gap it synthesises K sub-frames by splatting keyframe A forward and keyframe B
 * backward (Sec. 3.3, Eq. 5), resolves collisions with a per-pixel depth z-buffer
 * (Eqs. 6-7), blends the two directions in time with hole filling, and runs the event
 * model on each sub-frame: log-intensity against a per-pixel reference level, contrast
 * threshold, polarity, reference update keeping the residual (Sec. 3.2, Eq. 4), per-pixel
 * ON/OFF thresholds (Eq. 8) and a refractory period (Sec. 3.4).  Each crossing is emitted
 * as (env, x, y, t, polarity) with a timestamp interpolated linearly between sub-frames.
 *
 * Conventions shared by every entry point
 *  - Pointers named "device" must be CUDA device (or managed) memory of the current device;
 *    pointers named "host" must be host memory (pinned for asynchronous copies).
 *  - Packed layout: the environments of a context are stored back to back.  Environment e
 *    owns pixels [pix_off(e), pix_off(e) + H_e * W_e), pix_off being the prefix sum of
 *    H * W rounded up to a multiple of 4 (16-byte aligned starts).  Pixel (x, y) of an
 *    environment has index y * W + x.  Per-pixel arrays hold one float per pixel;
 *    motion vectors hold two (dx, dy interleaved); RGB frames hold three (R, G, B).
 *  - Motion vectors follow the renderer's convention (Sec. 3.3): mv(p) of a keyframe is the
 *    displacement, in pixels (+x right, +y down), from p to the position of the same surface
 *    point in the previous keyframe.
 *  - Depth: a source pixel takes part in the splat iff its depth is finite and > 0.
 *  - All work is enqueued on the context's stream; nothing blocks unless stated.
 *  - Errors detected on the host return immediately and change nothing.  Conditions detected
 *    on the device (event buffer overflow, pixels beyond the crossing limit) are latched and
 *    returned by the next call that synchronises (evis_read_events, evis_event_count).
 *  - Crossing limit: Eq. 4 gives a pixel n = floor(|L - L_ref| / C) crossings in one
 *    sub-frame, without bound.  A pixel emits at most EVIS_MAX_CROSSINGS of them per
 *    sub-frame (per channel in colour mode).  A pixel-sub-frame whose n is larger emits none
 *    of its crossings (no truncated stream), still moves its reference level by the whole
 *    p n C of Eq. 4, and is counted: the next read returns EVIS_ERR_RANGE and
 *    evis_get_env_stats reports the count per environment.
 *  - One context must not be used by two host threads at the same time.
 */
#ifndef EVIS_H
#define EVIS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t; 0 means the legacy default stream. */
typedef struct CUstream_st *evis_stream_t;
typedef struct evis_ctx evis_ctx;

typedef enum {
  EVIS_OK = 0,
  EVIS_ERR_INVALID_ARG = 1, /* bad size, pointer, flag or threshold; nothing was done */
  EVIS_ERR_CUDA = 2,        /* a CUDA call failed; see evis_last_error */
  EVIS_ERR_OOM = 3,         /* device allocation failed */
  EVIS_ERR_OVERFLOW = 4,    /* more events than the buffer (or the caller's array) holds */
  EVIS_ERR_STATE = 5,       /* call not valid in the context's current state */
  EVIS_ERR_TIMEOUT = 6,     /* reserved: no kernel of the library waits on another CTA, a
                             * flag or a peer, so no call returns it */
  EVIS_ERR_RANGE = 7        /* some pixel-sub-frame had more crossings than a pixel may emit
                             * (EVIS_MAX_CROSSINGS); its crossings were withheld, the state
                             * follows Eq. 4 exactly, everything else was delivered */
} evis_status;

/* Crossings one pixel may emit in one sub-frame (per channel). */
#define EVIS_MAX_CROSSINGS 4096

/* One event (16 bytes): time in ns, pixel, environment index, polarity +1 / -1. */
typedef struct {
  int64_t t_ns;
  uint16_t x, y, env;
  int16_t p;
} evis_event;

/* Input modes (Sec. 3.2): frames are log-intensity L, linear luminance I (L = log(I + eps)),
 * or linear RGB radiance (I = 0.2126 R + 0.7152 G + 0.0722 B, Eq. 3, then the log). */
#define EVIS_IN_LOG 0x0u
#define EVIS_IN_LUM 0x1u
#define EVIS_IN_RGB 0x2u
/* Blend of the two warp directions: time blend (1-f) A + f B with hole filling (default),
 * or B primary with A filling only B's holes (Sec. 3.3). */
#define EVIS_MODE_BLEND 0x0u
#define EVIS_MODE_B_PRIMARY 0x10u
/* Eq. 6 read literally: one argmin of interpolated depth over both directions' winners
 * (equal depths go to B); not combinable with EVIS_MODE_B_PRIMARY. */
#define EVIS_MODE_JOINT 0x40u
/* z-buffer tie-break among equal depths: larger bilinear weight then lower source index
 * (default), or lower source index only. */
#define EVIS_TIE_WEIGHT 0x0u
#define EVIS_TIE_INDEX 0x20u
/* The caller keeps the previous keyframe's mv and depth (and, in EVIS_IN_LOG mode, its
 * frames) alive and unmodified until the next evis_step has completed on the stream, so the
 * library reads them in place instead of keeping its own copy. */
#define EVIS_KEEP_INPUTS 0x100u
/* Colour events (Sec. 3.2): the event model runs on the R, G and B log intensities
 * independently, over one set of warp winners (they depend on motion and depth only).
 * Frames are linear RGB triples (EVIS_IN_RGB, [total][3], L_c = log(c + eps)) or three
 * log-intensity planes (EVIS_IN_LOG, [3][total]: R, G, B); EVIS_IN_LUM is rejected.  An
 * event's polarity field is +-(1 + c), c = 0, 1, 2 for R, G, B.  Reference levels and
 * refractory times are kept per channel: the per-pixel state arrays of evis_get_state hold
 * three planes [3][total], and the traced log-intensity is [K][3][H*W] per environment.
 * Threshold maps serve all channels; each channel draws its own noise streams (the last
 * counter word is stream + 4 c); defocus blurs each channel. */
#define EVIS_COLOR 0x200u
/* Collect the per-environment statistics of evis_get_env_stats that cost kernel work (holes
 * per warp direction, ON / OFF and noise event counts): about 3 to 4 % of the synthesis
 * kernel's time.  Without it those counts read 0; target-sub-frames and the crossing-limit
 * count are always kept. */
#define EVIS_STATS 0x400u

typedef struct {
  int32_t width, height; /* rendered frame, 1..65535 each, width * height <= 2^24 */
  int32_t K;             /* sub-frames per keyframe gap, 1..4096 (f = i/K, i = 1..K) */
  float c_on, c_off;     /* contrast thresholds (log units), finite and > 0 */
  int32_t margin;        /* over-render margin (Appendix B): every rendered pixel splats, but
                          * only the sensor, the frame without `margin` pixels on each side,
                          * is synthesised; events carry sensor coordinates (x - margin,
                          * y - margin).  0 <= 2 * margin < min(width, height); 0 = none.
                          * Per-pixel arrays (state, threshold maps) stay rendered-frame sized. */
  const float *c_on_map; /* optional device [H*W] per-pixel thresholds (Eq. 8); both or */
  const float *c_off_map;/* neither, 4-byte aligned; caller-owned, read at every step, must
                          * outlive ctx */
  int64_t refractory_ns; /* 0 = off (Sec. 3.4) */
  int64_t t0_ns;         /* time of the first keyframe */
} evis_env_desc;

typedef struct {
  float eps;              /* added before the log (Sec. 3.2), finite and >= 0 */
  uint32_t flags;         /* EVIS_IN_* | EVIS_MODE_* (one) | EVIS_TIE_* | EVIS_KEEP_INPUTS |
                           * EVIS_COLOR | EVIS_STATS */
  int64_t event_capacity; /* events the device buffer holds between two reads, >= 1 */
} evis_config;

/* Creates a context for n_envs environments (1..65535) on the current CUDA device and
 * allocates all device memory it will use (keyframe copies, reference levels, refractory
 * times, event buffer).  The descriptor array is copied; threshold maps are referenced.
 * Returns EVIS_ERR_INVALID_ARG for a bad descriptor or config (checked before any CUDA
 * call), EVIS_ERR_OOM when the device memory does not fit.  *out is set only on success. */
evis_status evis_create(const evis_env_desc *envs, int32_t n_envs, const evis_config *cfg,
                        evis_stream_t stream, evis_ctx **out);

/* Feeds the next keyframe (device pointers, packed layout; frames per the input mode).
 * The first call on a context sets the reference level of every pixel to the keyframe's
 * log-intensity and emits nothing (Sec. 3.2).  Each later call synthesises the K_e
 * sub-frames between the previous keyframe and this one (Sec. 3.3, Eqs. 5-7) and appends
 * their events (Sec. 3.2 Eq. 4, Sec. 3.4) to the device buffer; sub-frame i of environment
 * e is at t = T_e + (i * dt_ns) / K_e, T_e being the previous keyframe's time.
 * Asynchronous; inputs may be reused once the stream has passed this call, except under
 * EVIS_KEEP_INPUTS.  0 < dt_ns <= 2^40.  frames and depth must be 4-byte aligned, mv 8-byte
 * (it is read as float pairs); EVIS_ERR_INVALID_ARG otherwise. */
evis_status evis_step(evis_ctx *ctx, const float *frames, const float *mv, const float *depth,
                      int64_t dt_ns);

/* Same as evis_step with HOST inputs: the library copies them into its own device buffers
 * on the context's stream (host memory should be pinned) and then steps.  The first call
 * allocates those buffers. */
evis_status evis_step_host(evis_ctx *ctx, const float *frames, const float *mv,
                           const float *depth, int64_t dt_ns);

/* Synchronises the stream, copies the buffered events (in no particular order) to dst
 * (host or device, up to cap events), empties the buffer and clears latched errors.  The
 * reads (this one, evis_read_events_async and evis_event_count) wait for the context's own
 * stream only: their copies run on it, so work of other contexts on other streams, blocking
 * or not, keeps running.
 * *n_out = number of events produced since the last read.  Returns EVIS_ERR_RANGE when
 * some pixel-sub-frame since the last read exceeded the crossing limit (see the
 * conventions above; the events are delivered as usual), else EVIS_ERR_OVERFLOW when the
 * number produced exceeds the buffer capacity or cap: the first min(capacity, cap) stored
 * events are delivered and the per-pixel state has advanced as if none were lost. */
evis_status evis_read_events(evis_ctx *ctx, evis_event *dst, int64_t cap, int64_t *n_out);

/* Pipelined read-back: waits until the stream has passed every step enqueued so far (and
 * for the previous call's copy), starts copying the buffered events (in no particular
 * order, up to cap) to dst on the library's own copy stream, and switches the context to
 * its second event buffer, so that the steps enqueued next run while the copy proceeds.
 * *n_out and EVIS_ERR_OVERFLOW as for evis_read_events.  dst (host memory should be
 * pinned) is complete once the next evis_read_events_async or evis_read_wait returns, and
 * must stay valid until then.  The first call allocates the second buffer (event_capacity
 * records) and the copy stream.  Captured graphs are discarded (they hold the other
 * buffer's address). */
evis_status evis_read_events_async(evis_ctx *ctx, evis_event *dst, int64_t cap, int64_t *n_out);

/* Waits for the copy started by the last evis_read_events_async (no-op if none). */
evis_status evis_read_wait(evis_ctx *ctx);

/* Synchronises and reports the number of events produced since the last read (status as
 * for evis_read_events; nothing is cleared). */
evis_status evis_event_count(evis_ctx *ctx, int64_t *n_out);

/* Device-side view of the event buffer for consumers on the GPU: *events points to the
 * capacity-sized array, *count to the 64-bit produced-event counter (followed by the
 * counter of pixel-sub-frames beyond the crossing limit).  Valid until destroy or the next
 * evis_read_events_async (which switches buffers). */
evis_status evis_events_device(evis_ctx *ctx, evis_event **events, uint64_t **count);

/* Asynchronously empties the event buffer and clears the latched crossing-limit condition
 * (stream-ordered, no synchronisation; evis_get_env_stats keeps its counts). */
evis_status evis_clear_events(evis_ctx *ctx);

/* Synchronises and copies the per-pixel reference levels [nc][total px] and last emitted
 * event times [nc][total px] (INT64_MIN = none; nc = 3 in colour mode, else 1) and the
 * per-environment keyframe times [n_envs] to host memory (any pointer may be null).
 * Last-event times are tracked only when some environment of the context has a refractory
 * period; otherwise all read INT64_MIN. */
evis_status evis_get_state(evis_ctx *ctx, float *Lref, int64_t *t_last, int64_t *clocks);

/* Statistics since creation (any pointer may be null): keyframes fed and keyframe gaps
 * synthesised (as counted by the gap counter, which evis_set_state can restore), and per
 * environment [n_envs] the sources, summed over all keyframes, that cannot splat: depth
 * not finite and > 0, or a motion vector that is not finite.  Synchronises. */
evis_status evis_get_stats(evis_ctx *ctx, uint64_t *keyframes, uint64_t *gaps,
                           uint64_t *invalid_sources);

/* Per-environment statistics since creation (event count, ON/OFF split, hole fraction per
 * warp direction; Sec. 3.3 fills the holes of one direction from the other).  A
 * target-sub-frame is one sensor pixel at one sub-frame i = 1..K. */
typedef struct {
  uint64_t target_subframes; /* sensor pixels x K x keyframe gaps synthesised */
  uint64_t holes_a;          /* target-sub-frames that no source of A (forward warp) reached */
  uint64_t holes_b;          /* ... that no source of B (backward warp) reached */
  uint64_t holes_both;       /* ... that neither reached: no sample, the pixel held its state */
  uint64_t events_on;        /* events emitted with positive polarity (crossings and noise) */
  uint64_t events_off;       /* ... with negative polarity */
  uint64_t noise_events;     /* of those, sensor noise events (evis_set_noise) */
  uint64_t over_limit;       /* pixel-sub-frames (per channel) beyond EVIS_MAX_CROSSINGS */
} evis_env_stats;

/* Copies the statistics of every environment to out (host array of n_envs).  Holes, ON /
 * OFF and noise counts need EVIS_STATS (else 0).  Events past the buffer's capacity are
 * counted too (they were produced).  The autotuner's trial gaps are not counted.
 * Synchronises. */
evis_status evis_get_env_stats(evis_ctx *ctx, evis_env_stats *out);

/* Synchronises and copies the per-environment count of keyframe gaps processed (the noise
 * generator's gap counter) [n_envs] to host memory. */
evis_status evis_get_gaps(evis_ctx *ctx, uint32_t *gaps);

/* Restores state read by evis_get_state and evis_get_gaps: checkpoint and resume.  To
 * resume, create a context with the same environments and configuration, feed the last
 * keyframe before the checkpoint as its first keyframe (evis_step), then call this.  The
 * following gaps then produce what the uninterrupted context would have.  Arrays are laid
 * out as evis_get_state's (host or device memory); a null pointer keeps that part.  t_last
 * is ignored when the context tracks no refractory times.  EVIS_ERR_STATE before the first
 * keyframe.  Synchronises; a captured graph stays valid. */
evis_status evis_set_state(evis_ctx *ctx, const float *Lref, const int64_t *t_last,
                           const int64_t *clocks, const uint32_t *gaps);

/* Sensor non-idealities of one environment (Sec. 3.4).  The paper lists leak events, shot
 * noise and hot pixels without fixing their distributions; this library treats them as
 * competing sources of at most one noise event per sensor pixel, channel and sub-frame
 * [t_{i-1}, t_i), d = t_i - t_{i-1} ns, dts = d * 1e-9 s:
 *   leak: probability p_leak = leak_hz * dts, polarity +1;
 *   shot: p_shot = shot_hz * dts * (1 - clamp((L_i - lo) / (hi - lo), 0, 1)) with
 *         L_i = (1 - f) LA + f LB (f = i / K) the pixel's own log intensity interpolated
 *         between the gap's two keyframes (dark pixels fire most), random polarity;
 *   hot:  p_hot = hot_hz * dts on a fixed subset of pixels (each with probability
 *         hot_fraction, the same in every gap), polarity +1.
 * One uniform word u decides: with x = (float)(u >> 8), leak if x < p_leak * 2^24, else shot
 * if x < (p_leak + p_shot) * 2^24, else hot if x < (p_leak + p_shot + p_hot) * 2^24
 * (binary32, 1 / (hi - lo) rounded once, sums left to right; past a total of 1 the last
 * sources lose probability).  Words come from the counter-based generator Philox4x32-10
 * (Salmon et al., SC 2011) keyed by (seed low 32 bits, seed high 32 bits ^ environment index)
 * at counters (p, g, floor((i - 1) / 4), 4c), word (i - 1) mod 4, with p = y * W + x the
 * sensor pixel index, g the count of keyframe gaps the environment has processed and c the
 * channel; a fired event's time is t_{i-1} + floor(v * d / 2^32) with v word 0 at
 * (p, g, i, 1 + 4c), and a shot event is ON when bit 0 of word 3 there is set; the hot
 * subset uses word 0 at (p, 2^32 - 1, 0, 2 + 4c) against hot_fraction.  Noise events do not
 * depend on the launch shape, pass no refractory filter and leave the reference levels
 * unchanged. */
typedef struct {
  float leak_hz, shot_hz, hot_hz; /* rates per pixel (1/s), finite and >= 0; all 0 = off */
  float hot_fraction;             /* 0..1 */
  float lo, hi;                   /* log-intensity range of the normalised intensity, hi > lo */
  uint64_t seed;
} evis_noise_desc;

/* Sets the noise of every environment (host array of n_envs entries; NULL turns it off
 * everywhere).  Stream-ordered: applies from the next step.  Drops a captured graph (capture
 * again).  EVIS_ERR_INVALID_ARG for a negative or non-finite rate, hot_fraction outside 0..1
 * or hi <= lo, checked before anything changes. */
evis_status evis_set_noise(evis_ctx *ctx, const evis_noise_desc *noise);

/* Defocus (Sec. 3.4): before the log, each keyframe's linear luminance is convolved with a
 * separable Gaussian of standard deviation sigma pixels: taps k = -r..r, r = int(3 sigma +
 * 0.5), weights exp(-k^2 / (2 sigma^2)) normalised to sum 1 in binary64 and rounded to
 * binary32; edge pixels repeat; the horizontal pass runs first, then the vertical one, each
 * summing its taps in order in binary32.  For RGB input the blur acts on the Rec. 709
 * luminance.  sigma_px is a host array of n_envs values in 0..8 (0: none), or NULL for none;
 * any sigma > 0 needs EVIS_IN_LUM or EVIS_IN_RGB (EVIS_ERR_INVALID_ARG otherwise, nothing
 * changed).  Synchronises the stream; applies from the next keyframe; drops a captured graph.
 * Allocates a keyframe-sized buffer on first use. */
evis_status evis_set_defocus(evis_ctx *ctx, const float *sigma_px);

/* The defocus of one image alone: in is [height][width] luminance (mode EVIS_IN_LUM) or
 * [height][width][3] linear RGB (EVIS_IN_RGB); out is the blurred luminance [height][width].
 * Device pointers (4-byte aligned); asynchronous on stream; sizes as for an environment. */
evis_status evis_defocus(const float *in, int32_t width, int32_t height, uint32_t mode,
                         float sigma_px, float *out, evis_stream_t stream);

/* Event voxel grid (the speed-regression input of the paper's appendix): for each
 * environment's segment [t0_ns, t1_ns], per polarity (slot 0: ON, p > 0; slot 1: OFF, p < 0;
 * colour events count by their sign) and time bin b = 0..bins-1, the events linearly
 * interpolated along time, each (environment, polarity, bin) plane divided by its largest
 * value.  An event at t sits at tau = (bins - 1)(t - t0) / (t1 - t0) and adds 1 - frac(tau)
 * to bin floor(tau) and frac(tau) to the next, in units of 2^-16: with D = t1 - t0,
 * N = (bins - 1)(t - t0), b = N / D, r = N mod D, w_next = floor(r 2^16 / D) and
 * w_b = 2^16 - w_next, summed exactly in uint32 (exact while a voxel receives fewer than
 * 65536 events).  The normalised value is the binary32 quotient of the sum by the plane's
 * maximum (0 for an empty plane).  Events outside the segment or the sensor, of an
 * environment >= n_envs, or with p = 0, are skipped. */
typedef struct {
  int32_t width, height;   /* sensor, 1..65535 each, width * height <= 2^24 */
  int64_t t0_ns, t1_ns;    /* segment, 0 < t1_ns - t0_ns < 2^32 */
} evis_voxel_env;

/* Device workspace bytes of evis_voxel_grid for up to max_events records (a descriptor
 * table, one uint32 per plane for its maximum, two uint64 per region of 32 pixels of a row
 * across 256 planes, and one uint32 per record, two when bins > 128). */
evis_status evis_voxel_workspace_size(const evis_voxel_env *envs, int32_t n_envs, int32_t bins,
                                      int64_t max_events, int64_t *bytes);

/* Builds the grid of every environment (host array envs of n_envs, bins in 1..1024) from
 * the device event records events[0 .. n), n = min(*count, max_events) with count a device
 * pointer (for example evis_events_device's, so no host synchronisation is needed) or
 * max_events when count is NULL.  grid is a device float array, per environment in order
 * [2][bins][height][width].  workspace is device memory of evis_voxel_workspace_size(...,
 * max_events, ...) bytes (its contents need not be initialised).  events and workspace must
 * be 16-byte aligned, count 8-byte and grid 4-byte aligned.  Asynchronous on stream;
 * EVIS_ERR_INVALID_ARG (evis_last_error(NULL) says why) before any work for a bad
 * argument. */
evis_status evis_voxel_grid(const evis_event *events, const uint64_t *count, int64_t max_events,
                            const evis_voxel_env *envs, int32_t n_envs, int32_t bins,
                            void *workspace, int64_t workspace_bytes, float *grid,
                            evis_stream_t stream);

/* Debug form of evis_step: also writes, for every environment in order and every
 * sub-frame i = 1..K_e, the two z-buffers (keys[((i-1)*2 + dir) * H*W + p], dir 0 = A
 * forward, dir 1 = B backward; key = depth bits << 32 | quantised (1 - weight) << 24 |
 * source index, all ones = no source) and the blended log-intensity (Lint[(i-1) * H*W + p],
 * NaN where the pixel got no sample).  keys / Lint are device arrays of
 * sum_e K_e * 2 * H_e * W_e uint64 and sum_e K_e * H_e * W_e floats.  With a margin, only
 * the sensor's entries are written; the margin's are left as they were.  keys must be
 * 8-byte aligned, Lint 4-byte, the inputs as for evis_step. */
evis_status evis_step_trace(evis_ctx *ctx, const float *frames, const float *mv,
                            const float *depth, int64_t dt_ns, uint64_t *keys, float *Lint);

/* Log-intensity of n samples (Sec. 3.2, Eq. 3): mode EVIS_IN_LUM reads n floats, EVIS_IN_RGB
 * n RGB triplets; out[i] = log(I + eps) (non-positive arguments clamp to the smallest
 * normal float).  Device pointers (4-byte aligned), enqueued on stream. */
evis_status evis_log_intensity(const float *in, int64_t n, uint32_t mode, float eps, float *out,
                               evis_stream_t stream);

/* Selects the target tile of the synthesis kernel: tile_w x tile_h pixels per CTA, one of
 * 32x8, 32x16 (default), 32x32, 64x16, 64x32, 128x16.  Results do not depend on the shape, only
 * speed does.  Synchronises the stream; EVIS_ERR_INVALID_ARG for another shape. */
evis_status evis_set_tile_shape(evis_ctx *ctx, int32_t tile_w, int32_t tile_h);

/* Per-environment tile shapes (host arrays of n_envs entries, each a supported shape; at
 * most 8 distinct shapes).  Environments sharing a shape run in one launch of the
 * synthesis kernel.  Synchronises; invalidates captured graphs. */
evis_status evis_set_env_tile_shapes(evis_ctx *ctx, const int32_t *tile_w, const int32_t *tile_h);

/* Copies the current per-environment tile shapes to host arrays of n_envs entries. */
evis_status evis_get_tile_shapes(evis_ctx *ctx, int32_t *tile_w, int32_t *tile_h);

/* Autotuner: for each resolution class (environments of equal width and height) times the
 * synthesis kernel with every supported tile shape on the gap from the retained keyframe to
 * the given keyframe B (device pointers, as for evis_step), best of reps runs after one
 * warm-up, and keeps the fastest shape per class.  Nothing is consumed: the per-pixel
 * state and the event buffer's count are restored, so the caller then steps with the same
 * B as usual.  *best_ms (optional) receives the sum over classes of the best times.
 * Alignment as for evis_step.  EVIS_ERR_STATE before the first keyframe.  Synchronises;
 * invalidates captured graphs. */
evis_status evis_autotune(evis_ctx *ctx, const float *frames, const float *mv,
                          const float *depth, int64_t dt_ns, int32_t reps, float *best_ms);

/* Library-owned device input buffers (packed layout; frames sized for the input mode) for
 * callers that write the next keyframe in place, as evis_replay requires.  Two sets
 * alternate from keyframe to keyframe: call this before writing each keyframe.  The first
 * call allocates them. */
evis_status evis_input_buffers(evis_ctx *ctx, float **frames, float **mv, float **depth);

/* Captures one keyframe gap (preparation and synthesis kernels of every tile group, reading
 * the input buffers) into CUDA graphs with the fixed interval dt_ns, so that evis_replay
 * replaces evis_step for the following keyframes.  Needs a retained keyframe, a context
 * without EVIS_KEEP_INPUTS and a non-default stream (EVIS_ERR_STATE otherwise).  Any later
 * evis_step, evis_step_host, evis_step_trace or shape change discards the graphs. */
evis_status evis_capture(evis_ctx *ctx, int64_t dt_ns);

/* Replays the captured gap on the keyframe written to the current input buffers
 * (evis_input_buffers): the same work and results as evis_step with those buffers and the
 * captured dt_ns, as one graph launch.  Asynchronous. */
evis_status evis_replay(evis_ctx *ctx);

/* Differentiable soft event counts of one keyframe gap.  The paper has no backward pass;
 * this surrogate keeps the event path's discrete decisions frozen (z-buffer winners,
 * holes, and the reference trajectory L_ref^(i) of Eq. 4 with each environment's c_on and
 * c_off) and makes the rest smooth.  Per direction and sub-frame, the value at a target is the bilinear
 * splat of L normalised over the winner surface: footprint sources whose interpolated
 * depth is <= Z* (1 + delta), Z* the winning depth.  The two directions are blended as in
 * the event path, and the counts are
 *   N_on  = sum_i sig((L_i - L_ref^(i-1) - C) / tau),
 *   N_off = sum_i sig((L_ref^(i-1) - L_i - C) / tau)
 * over the sub-frames with a sample; C [n_envs] is the differentiable threshold and
 * enters only the sigmoids.  envs gives width, height, K and the event thresholds c_on,
 * c_off of the frozen trajectory (margin must be 0: the counts cover the whole rendered
 * frame; other fields are ignored); inputs are device arrays in the packed layout (log-intensity L_A, L_B, motion
 * vectors, depth, start-of-gap reference levels Lref0) and C [n_envs]; counts is
 * [2][H][W] per environment at offset 2 * pix_off.  The workspace (device, at least
 * evis_soft_workspace_size bytes) keeps what the backward needs; the forward is
 * deterministic.  Motion vectors (and, in the backward, their gradients) must be 8-byte
 * aligned, the other arrays 4-byte, the workspace 16-byte; EVIS_ERR_INVALID_ARG otherwise.
 * Asynchronous on stream. */
evis_status evis_soft_workspace_size(const evis_env_desc *envs, int32_t n_envs, int64_t *bytes);
evis_status evis_soft_forward(const evis_env_desc *envs, int32_t n_envs, float tau, float delta,
                              const float *L_A, const float *L_B, const float *mv_A,
                              const float *mv_B, const float *Z_A, const float *Z_B,
                              const float *Lref0, const float *C, float *counts,
                              void *workspace, int64_t workspace_bytes, evis_stream_t stream);

/* Gradients of sum(gcounts * counts) with respect to L_A, L_B, mv_A, mv_B (packed like the
 * inputs) and C [n_envs], from the workspace of the forward call with the same inputs
 * (overwritten, not accumulated).  Gather form: no atomics except one per block for dC. */
evis_status evis_soft_backward(const evis_env_desc *envs, int32_t n_envs, float tau, float delta,
                               const float *L_A, const float *L_B, const float *mv_A,
                               const float *mv_B, const float *Z_A, const float *Z_B,
                               const float *C, const float *gcounts, float *dL_A, float *dL_B,
                               float *dmv_A, float *dmv_B, float *dC, void *workspace,
                               int64_t workspace_bytes, evis_stream_t stream);

/* Per-kernel timing for profiling.  With max_steps > 0, each following evis_step (or
 * evis_step_host / evis_step_trace) records CUDA events on the context's stream around its
 * two phases, for at most max_steps steps; max_steps = 0 disables and forgets the records.
 * The events cost nothing on the device.  The keyframe that only sets the reference level
 * records no synthesis phase (its duration reads 0). */
evis_status evis_profile_enable(evis_ctx *ctx, int32_t max_steps);

/* Synchronises and writes, for each recorded step s (at most cap), ms[2*s] = duration of
 * the input preparation (log-intensity, copies, motion bound) and ms[2*s+1] = duration of
 * the synthesis kernel (splat, blend, events), in milliseconds; *n_steps = steps written. */
evis_status evis_profile_read(evis_ctx *ctx, float *ms, int32_t cap, int32_t *n_steps);

/* One keyframe gap of ONE environment with no device allocation at all.  The paper has no
 * counterpart: this is for callers that cannot call cudaMalloc when they need events, such
 * as a simulator or engine that owns the whole GPU memory pool and hands out buffers, or a
 * latency-critical loop that must not meet the allocator.  The caller passes every buffer
 * (device pointers): keyframes A (previous) and B (new) as log-intensity, motion vectors
 * and depth in the single-environment layout; the reference levels Lref [H*W] (set them to
 * the first keyframe's log-intensity before the first call) and, when refractory_ns > 0,
 * the last-event times t_last [H*W] (INT64_MIN = none), both updated in place; the event
 * array (capacity entries) and two 64-bit counters count[0..1]: count[0] receives the number
 * of events of this gap exactly as evis_step adds them to a context's buffer, count[1] the
 * number of pixel-sub-frames beyond the crossing limit (the caller resets both).
 * Sub-frame i is at t_a_ns + (i * dt_ns) / K.  The results equal those of evis_step.
 * flags may hold EVIS_MODE_B_PRIMARY and EVIS_TIE_INDEX only.
 *
 * Invalid arguments return EVIS_ERR_INVALID_ARG before any work, among them misaligned
 * buffers: the float arrays need 4-byte alignment, mv_A, mv_B, t_last and count 8-byte,
 * events 16-byte.
 *
 * Limits: width, height <= 4096 and width * height <= 1048576, set by a static scratch
 * array of about 1.3 MB that every GPU loading the library holds until the process exits
 * (it keeps the environment descriptor, tile list, clocks and motion bounds).  Larger
 * sizes return EVIS_ERR_INVALID_ARG with the reason in evis_last_error(NULL).  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  All calls share the
 * array, so calls whose work overlaps on the GPU (other streams, other host threads) race;
 * serialise them on one stream.  Asynchronous on stream. */
evis_status evis_step_noalloc(const evis_env_desc *env, uint32_t flags, const float *L_A,
                              const float *mv_A, const float *Z_A, const float *L_B,
                              const float *mv_B, const float *Z_B, float *Lref,
                              int64_t *t_last, int64_t t_a_ns, int64_t dt_ns,
                              evis_event *events, uint64_t *count, int64_t capacity,
                              evis_stream_t stream);

/* Total packed pixels of the context (the length of its per-pixel arrays). */
evis_status evis_total_pixels(evis_ctx *ctx, int64_t *n_out);

/* Releases the context and all its device memory (synchronises the stream first). */
evis_status evis_destroy(evis_ctx *ctx);

/* Static description of a status code. */
const char *evis_status_string(evis_status s);

/* Text of the last CUDA or validation error seen by ctx (empty if none); with ctx = NULL,
 * why the calling thread's last failed evis_create or evis_step_noalloc failed. */
const char *evis_last_error(evis_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* EVIS_H */
