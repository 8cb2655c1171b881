// Host side of libevis: argument validation, device memory, stream ordering and the C ABI
// declared in include/evis.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "evis_internal.h"

using evis::DevEnv;
using evis::Tile;

struct evis_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  evis_config cfg{};
  uint32_t mode = 0;
  bool keep = false;
  bool need_L = false;     // library holds converted / copied log-intensity slots
  int nc = 1;              // event channels: 3 in colour mode (L, Lref, t_last hold nc planes)
  int n = 0;
  std::vector<evis_env_desc> envs;
  std::vector<int64_t> off;
  int64_t total = 0;
  int max_px = 0;
  int max_segs = 0;
  int64_t total_segs = 0;
  // tile shape per environment; environments sharing a shape form one launch group
  std::vector<int> env_tw, env_th;
  struct Group {
    int tw, th;
    int64_t offset;  // first tile in d_tiles
    int count;
  };
  std::vector<Group> groups;
  int grid_cap = 1;        // persistent launches: one wave of resident CTAs per group
  bool any_refr = false;

  std::vector<DevEnv> h_envs;  // host copy of d_envs (noise and defocus parameters change it)
  bool any_noise = false;
  int noise_max_px = 0;        // largest sensor (pixels) among the environments with noise on
  int blur_r_max = -1;         // largest defocus radius; -1: no defocus pass
  float *d_blur = nullptr;     // [total] blurred luminance of the keyframe being prepared
  float *d_blur_w = nullptr;   // [n][2 kMaxBlurR + 1] defocus weights
  DevEnv *d_envs = nullptr;
  Tile *d_tiles = nullptr;
  unsigned *d_work = nullptr;  // per-group work counters, zeroed every step
  float *d_L[2] = {nullptr, nullptr};
  float *d_mv[2] = {nullptr, nullptr};
  float *d_Z[2] = {nullptr, nullptr};
  float *d_Lref = nullptr;
  int64_t *d_tlast = nullptr;
  float *d_flow = nullptr;     // [2][n]
  float4 *d_seg[2] = {nullptr, nullptr};  // per keyframe slot: row-segment motion bounds
  float4 *d_pack[2] = {nullptr, nullptr}; // per-source packs of A and B for the current gap
  int64_t *d_clock = nullptr;  // [2][n]
  uint32_t *d_gap = nullptr;   // [2][n]: keyframe gaps processed, alternating like d_clock
  unsigned long long *d_invalid = nullptr;  // [n]: sources that could not splat, all keyframes
  ulonglong2 *d_events = nullptr;          // the buffer the steps append to
  unsigned long long *d_count = nullptr;   // [0] events produced, [1] pixel-sub-frames over the limit
  unsigned long long *d_stats = nullptr;   // [n][kStatWords] statistics since creation
  // pipelined read-back: the second buffer, and the copy of the other one in flight
  ulonglong2 *d_events_alt = nullptr;
  unsigned long long *d_count_alt = nullptr;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t copy_done = nullptr;
  bool copy_ready = false;   // the second buffer, the copy stream and its event all exist
  bool copy_pending = false;
  int64_t *d_tr_off = nullptr; // [2][n]: key offsets, then L offsets
  float *d_in[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
  int in_slot = 0;

  int slot = 0;       // keyframe slot currently holding A
  int clk = 0;        // clock buffer holding the time of A
  bool have_A = false;
  const float *A_L = nullptr, *A_mv = nullptr, *A_Z = nullptr;

  // graph replay: two graphs (the keyframe slots and clocks alternate every gap)
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int64_t graph_dt = 0;
  int graph_phase = 0;
  // autotuner scratch (allocated on first use)
  float *d_tune_Lref = nullptr;
  int64_t *d_tune_tlast = nullptr;
  Tile *d_tune_tiles = nullptr;

  std::vector<cudaEvent_t> prof;   // 3 events per profiled step
  int prof_max = 0, prof_n = 0;

  std::vector<void *> allocs;
  std::string err;
};

namespace {

constexpr int64_t kMaxDt = int64_t(1) << 40;
thread_local std::string g_create_error;  // why the last evis_create on this thread failed

evis_status fail(evis_ctx *c, evis_status s, const std::string &msg) {
  if (c) c->err = msg;
  return s;
}

evis_status cuda_fail(evis_ctx *c, cudaError_t e, const char *where) {
  if (c) c->err = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? EVIS_ERR_OOM : EVIS_ERR_CUDA;
}

bool finite_pos(float v) { return std::isfinite(v) && v > 0.0f; }

std::string validate(const evis_env_desc *envs, int32_t n, const evis_config *cfg) {
  if (!envs) return "envs is null";
  if (!cfg) return "cfg is null";
  if (n < 1 || n > 65535) return "n_envs must be in 1..65535";
  if (!std::isfinite(cfg->eps) || cfg->eps < 0.0f) return "eps must be finite and >= 0";
  const uint32_t known = 0x3u | EVIS_MODE_B_PRIMARY | EVIS_MODE_JOINT | EVIS_TIE_INDEX |
                         EVIS_KEEP_INPUTS | EVIS_COLOR | EVIS_STATS;
  if (cfg->flags & ~known) return "unknown flag bits";
  if ((cfg->flags & EVIS_COLOR) && (cfg->flags & 0x3u) == EVIS_IN_LUM)
    return "EVIS_COLOR needs EVIS_IN_RGB (linear RGB) or EVIS_IN_LOG (three log-intensity planes)";
  if ((cfg->flags & EVIS_MODE_B_PRIMARY) && (cfg->flags & EVIS_MODE_JOINT))
    return "EVIS_MODE_B_PRIMARY and EVIS_MODE_JOINT exclude each other";
  if ((cfg->flags & 0x3u) == 0x3u) return "invalid input mode";
  if (cfg->event_capacity < 1 || cfg->event_capacity > (int64_t(1) << 40))
    return "event_capacity must be in 1..2^40";
  for (int i = 0; i < n; ++i) {
    const evis_env_desc &d = envs[i];
    char buf[96];
    std::snprintf(buf, sizeof buf, "env %d: ", i);
    std::string p(buf);
    if (d.width < 1 || d.width > 65535 || d.height < 1 || d.height > 65535)
      return p + "width and height must be in 1..65535";
    if (int64_t(d.width) * d.height > (int64_t(1) << 24)) return p + "width*height must be <= 2^24";
    if (d.K < 1 || d.K > 4096) return p + "K must be in 1..4096";
    if (!finite_pos(d.c_on) || !finite_pos(d.c_off)) return p + "thresholds must be finite and > 0";
    if ((d.c_on_map == nullptr) != (d.c_off_map == nullptr))
      return p + "give both threshold maps or neither";
    if (!evis::aligned(d.c_on_map, 4) || !evis::aligned(d.c_off_map, 4))
      return p + "threshold maps need 4-byte alignment";
    if (d.refractory_ns < 0) return p + "refractory_ns must be >= 0";
    if (d.margin < 0 || 2 * int64_t(d.margin) >= d.width || 2 * int64_t(d.margin) >= d.height)
      return p + "margin must satisfy 0 <= 2 * margin < min(width, height)";
  }
  return "";
}

template <class T>
cudaError_t dalloc(evis_ctx *c, T **p, size_t count) {
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  c->allocs.push_back(q);
  *p = static_cast<T *>(q);
  return cudaSuccess;
}

void release(evis_ctx *c) {
  if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);  // a read-back may be in flight
  if (c->copy_done) cudaEventDestroy(c->copy_done);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  c->copy_done = nullptr;
  c->copy_stream = nullptr;
  c->copy_ready = false;
  c->copy_pending = false;
  for (auto &g : c->graph) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
  for (void *p : c->allocs) cudaFree(p);
  c->allocs.clear();
  for (cudaEvent_t ev : c->prof) cudaEventDestroy(ev);
  c->prof.clear();
  c->prof_max = c->prof_n = 0;
}

__global__ void fill_i64(int64_t *p, int64_t v, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    p[i] = v;
}

constexpr int kMaxGroups = 8;

// Tiles of the environments whose index passes `take`, for shape tw x th, longest-running
// (largest K) first so that the tail of a launch holds the short ones.
template <class Pred>
std::vector<Tile> tiles_for(const evis_ctx *c, int tw, int th, Pred take) {
  std::vector<Tile> tiles;
  for (int i = 0; i < c->n; ++i) {
    if (!take(i)) continue;
    const evis_env_desc &d = c->envs[i];  // tiles cover the sensor (inside the margin)
    for (int y = d.margin; y < d.height - d.margin; y += th)
      for (int x = d.margin; x < d.width - d.margin; x += tw) tiles.push_back(Tile{i, x, y, 0});
  }
  std::stable_sort(tiles.begin(), tiles.end(), [&](const Tile &a, const Tile &b) {
    return c->envs[a.env].K > c->envs[b.env].K;
  });
  return tiles;
}

// Tile count of the smallest supported tile (the capacity of the device tile table).
int64_t max_tiles(const evis_ctx *c) {
  int64_t n = 0;
  for (const evis_env_desc &d : c->envs) n += int64_t((d.width + 31) / 32) * ((d.height + 7) / 8);
  return n;
}

// Regroups the environments by tile shape and uploads the tile lists (host-synchronous).
cudaError_t rebuild_groups(evis_ctx *c) {
  c->groups.clear();
  std::vector<Tile> all;
  for (int i = 0; i < c->n; ++i) {
    bool seen = false;
    for (const auto &g : c->groups) seen |= g.tw == c->env_tw[i] && g.th == c->env_th[i];
    if (seen) continue;
    const int tw = c->env_tw[i], th = c->env_th[i];
    std::vector<Tile> t = tiles_for(c, tw, th, [&](int e) { return c->env_tw[e] == tw && c->env_th[e] == th; });
    c->groups.push_back(evis_ctx::Group{tw, th, static_cast<int64_t>(all.size()), static_cast<int>(t.size())});
    all.insert(all.end(), t.begin(), t.end());
  }
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return e;
  return cudaMemcpy(c->d_tiles, all.data(), sizeof(Tile) * all.size(), cudaMemcpyHostToDevice);
}

// Launches the synthesis kernel for every tile group, then the sensor noise of the gap.
cudaError_t launch_groups(evis_ctx *c, evis::StepArgs s, bool trace) {
  for (size_t gi = 0; gi < c->groups.size(); ++gi) {
    const auto &g = c->groups[gi];
    s.tiles = c->d_tiles + g.offset;
    s.n_tiles = g.count;
    s.work_counter = c->d_work + gi;
    cudaError_t e = evis::launch_step(s, g.tw, g.th, trace, c->grid_cap, c->stream);
    if (e != cudaSuccess) return e;
  }
  return evis::launch_noise(s, c->n, c->noise_max_px, c->stream);
}

// The new keyframe B as the synthesis kernel reads it.
struct KeyframeB {
  const float *L, *mv, *Z;
};

// Enqueues the preparation of keyframe B into slot b = slot ^ 1: clears the motion maxima and
// work counters, converts / copies B, records its motion bounds and the per-source packs.
cudaError_t enqueue_prep(evis_ctx *c, const float *frames, const float *mv, const float *depth,
                         KeyframeB *out) {
  const int b = c->slot ^ 1;
  float *flowB = c->d_flow + b * c->n;
  cudaError_t e = cudaMemsetAsync(flowB, 0, sizeof(float) * c->n, c->stream);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(c->d_work, 0, sizeof(unsigned) * kMaxGroups, c->stream)) != cudaSuccess)
    return e;
  uint32_t mode = c->mode;
  if (c->blur_r_max >= 0) {  // defocus: blurred luminance first, then prepared like luminance input
    evis::BlurArgs ba{};
    ba.envs = c->d_envs;
    ba.wtab = c->d_blur_w;
    ba.in = frames;
    ba.out = c->d_blur;
    ba.mode = c->mode;
    ba.nc = c->nc;
    ba.plane = c->total;
    ba.max_r = c->blur_r_max;
    int max_t = 1;
    for (const evis_env_desc &d : c->envs) max_t = std::max(max_t, ((d.width + 63) / 64) * ((d.height + 31) / 32));
    if ((e = evis::launch_defocus(ba, c->n, max_t, c->stream)) != cudaSuccess) return e;
    frames = c->d_blur;
    mode = EVIS_IN_LUM;
  }
  evis::PrepArgs pa{};
  pa.envs = c->d_envs;
  pa.frames = frames;
  pa.mv = mv;
  pa.Z = depth;
  pa.L_out = c->need_L ? c->d_L[b] : nullptr;
  pa.mv_out = c->keep ? nullptr : c->d_mv[b];
  pa.Z_out = c->keep ? nullptr : c->d_Z[b];
  pa.flow = flowB;
  pa.seg = c->d_seg[b];
  pa.mvA = c->have_A ? c->A_mv : nullptr;
  pa.ZA = c->have_A ? c->A_Z : nullptr;
  pa.packA = c->d_pack[0];
  pa.packB = c->d_pack[1];
  pa.eps = c->cfg.eps;
  pa.mode = mode;
  pa.nc = c->nc;
  pa.plane = c->total;
  pa.invalid = c->d_invalid;
  pa.max_segs = c->max_segs;
  if ((e = evis::launch_prep(pa, c->n, c->stream)) != cudaSuccess) return e;
  out->L = c->need_L ? c->d_L[b] : frames;
  out->mv = c->keep ? mv : c->d_mv[b];
  out->Z = c->keep ? depth : c->d_Z[b];
  return cudaSuccess;
}

// Arguments of the synthesis kernel for the gap from the retained A to B (tiles unset).
evis::StepArgs step_args(const evis_ctx *c, const KeyframeB &B, int64_t dt) {
  const int b = c->slot ^ 1;
  evis::StepArgs s{};
  s.envs = c->d_envs;
  s.LA = c->A_L;
  s.mvA = c->A_mv;
  s.ZA = c->A_Z;
  s.LB = B.L;
  s.mvB = B.mv;
  s.ZB = B.Z;
  s.Lref = c->d_Lref;
  s.tlast = c->d_tlast;
  s.clock_in = c->d_clock + c->clk * c->n;
  s.clock_out = c->d_clock + (c->clk ^ 1) * c->n;
  s.gap_in = c->d_gap + c->clk * c->n;
  s.gap_out = c->d_gap + (c->clk ^ 1) * c->n;
  s.noise = c->any_noise;
  s.flowA = c->d_flow + c->slot * c->n;
  s.flowB = c->d_flow + b * c->n;
  s.segA = c->d_seg[c->slot];
  s.segB = c->d_seg[b];
  s.packA = c->d_pack[0];
  s.packB = c->d_pack[1];
  s.events = c->d_events;
  s.ev_count = c->d_count;
  s.capacity = static_cast<unsigned long long>(c->cfg.event_capacity);
  s.env_stats = c->d_stats;
  s.stats = (c->cfg.flags & EVIS_STATS) != 0;
  s.dt = dt;
  s.flags = c->cfg.flags;
  s.nc = c->nc;
  s.plane = c->total;
  s.tr_koff = c->d_tr_off;
  s.tr_loff = c->d_tr_off + c->n;
  return s;
}

evis_status do_step(evis_ctx *c, const float *frames, const float *mv, const float *depth,
                    int64_t dt, uint64_t *tr_keys, float *tr_L) {
  if (!frames || !mv || !depth) return fail(c, EVIS_ERR_INVALID_ARG, "null input pointer");
  if (!evis::aligned(frames, 4) || !evis::aligned(mv, 8) || !evis::aligned(depth, 4))
    return fail(c, EVIS_ERR_INVALID_ARG, "frames and depth need 4-byte alignment, mv 8-byte");
  if (dt <= 0 || dt > kMaxDt) return fail(c, EVIS_ERR_INVALID_ARG, "dt_ns must be in 1..2^40");
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  const bool prof = c->prof_n < c->prof_max;
  cudaEvent_t *pev = prof ? &c->prof[3 * c->prof_n] : nullptr;
  if (prof && (e = cudaEventRecord(pev[0], c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "profile event");
  KeyframeB B{};
  if ((e = enqueue_prep(c, frames, mv, depth, &B)) != cudaSuccess) return cuda_fail(c, e, "prep kernel");
  if (prof && (e = cudaEventRecord(pev[1], c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "profile event");
  if (c->have_A) {
    evis::StepArgs s = step_args(c, B, dt);
    s.tr_keys = tr_keys;
    s.tr_L = tr_L;
    if ((e = launch_groups(c, s, tr_keys != nullptr)) != cudaSuccess)
      return cuda_fail(c, e, "step kernel");
    c->clk ^= 1;
  } else {
    e = evis::launch_init_ref(B.L, c->d_Lref, c->nc * c->total, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
    c->have_A = true;
  }
  if (prof) {
    if ((e = cudaEventRecord(pev[2], c->stream)) != cudaSuccess) return cuda_fail(c, e, "profile event");
    ++c->prof_n;
  }
  c->slot ^= 1;
  c->A_L = B.L;
  c->A_mv = B.mv;
  c->A_Z = B.Z;
  return EVIS_OK;
}

// Library-owned input buffers (two sets, alternating per keyframe), allocated once.
cudaError_t ensure_inputs(evis_ctx *c) {
  if (c->d_in[0][0]) return cudaSuccess;
  const size_t fw = (c->mode == EVIS_IN_RGB || c->nc == 3) ? 3 : 1;
  cudaError_t e;
  for (int s = 0; s < 2; ++s) {
    if ((e = dalloc(c, &c->d_in[s][0], fw * c->total)) != cudaSuccess ||
        (e = dalloc(c, &c->d_in[s][1], 2 * c->total)) != cudaSuccess ||
        (e = dalloc(c, &c->d_in[s][2], c->total)) != cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

// Graphs bake the context's keyframe slots; any step taken outside them invalidates them.
void drop_graphs(evis_ctx *c) {
  for (auto &g : c->graph) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
}

}  // namespace

namespace evis {
void set_detached_error(const std::string &msg) { g_create_error = msg; }
}  // namespace evis

extern "C" {

evis_status evis_create(const evis_env_desc *envs, int32_t n_envs, const evis_config *cfg,
                        evis_stream_t stream, evis_ctx **out) {
  if (!out) return EVIS_ERR_INVALID_ARG;
  g_create_error = validate(envs, n_envs, cfg);
  if (!g_create_error.empty()) return EVIS_ERR_INVALID_ARG;
  evis_ctx *c = new evis_ctx();
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  c->cfg = *cfg;
  c->mode = cfg->flags & 0x3u;
  c->nc = (cfg->flags & EVIS_COLOR) ? 3 : 1;
  c->keep = (cfg->flags & EVIS_KEEP_INPUTS) != 0;
  c->need_L = c->mode != EVIS_IN_LOG || !c->keep;
  c->n = n_envs;
  c->envs.assign(envs, envs + n_envs);
  std::vector<DevEnv> denv(n_envs);
  std::vector<int64_t> troff(2 * n_envs);
  int64_t ko = 0, lo = 0;
  for (int i = 0; i < n_envs; ++i) {
    const evis_env_desc &d = envs[i];
    c->off.push_back(c->total);
    const int64_t px = int64_t(d.width) * d.height;
    DevEnv &v = denv[i];
    v.W = d.width;
    v.H = d.height;
    v.K = d.K;
    v.tile_h = 16;
    v.pix_off = c->total;
    v.segs_x = (d.width + evis::kSegW - 1) / evis::kSegW;
    v.seg_off = c->total_segs;
    c->total_segs += int64_t(v.segs_x) * d.height;
    c->max_segs = std::max<int>(c->max_segs, v.segs_x * d.height);
    v.c_on = d.c_on;
    v.c_off = d.c_off;
    v.con_map = d.c_on_map;
    v.coff_map = d.c_off_map;
    v.refractory_ns = d.refractory_ns;
    v.margin = d.margin;
    c->total += (px + 3) / 4 * 4;
    c->max_px = std::max<int>(c->max_px, static_cast<int>(px));
    c->any_refr |= d.refractory_ns > 0;
    troff[i] = ko;
    troff[n_envs + i] = lo;
    ko += int64_t(d.K) * 2 * px;
    lo += int64_t(d.K) * c->nc * px;
  }
  c->env_tw.assign(n_envs, 32);
  c->env_th.assign(n_envs, 16);

  cudaError_t e = cudaGetDevice(&c->device);
  auto bail = [&](cudaError_t err, const char *where) {
    evis_status s = cuda_fail(c, err, where);
    g_create_error = c->err;
    release(c);
    delete c;
    return s;
  };
  if (e != cudaSuccess) return bail(e, "cudaGetDevice");
  if ((e = dalloc(c, &c->d_envs, n_envs)) != cudaSuccess) return bail(e, "alloc envs");
  if ((e = dalloc(c, &c->d_tiles, max_tiles(c))) != cudaSuccess) return bail(e, "alloc tiles");
  if ((e = dalloc(c, &c->d_work, kMaxGroups)) != cudaSuccess) return bail(e, "alloc work counters");
  if ((e = dalloc(c, &c->d_Lref, c->nc * c->total)) != cudaSuccess) return bail(e, "alloc Lref");
  if (c->any_refr && (e = dalloc(c, &c->d_tlast, c->nc * c->total)) != cudaSuccess)
    return bail(e, "alloc t_last");
  if ((e = dalloc(c, &c->d_flow, 2 * n_envs)) != cudaSuccess) return bail(e, "alloc flow");
  for (int s = 0; s < 2; ++s)
    if ((e = dalloc(c, &c->d_seg[s], c->total_segs)) != cudaSuccess) return bail(e, "alloc segments");
  for (int s = 0; s < 2; ++s)
    if ((e = dalloc(c, &c->d_pack[s], c->total)) != cudaSuccess) return bail(e, "alloc source packs");
  if ((e = dalloc(c, &c->d_clock, 2 * n_envs)) != cudaSuccess) return bail(e, "alloc clock");
  if ((e = dalloc(c, &c->d_gap, 2 * n_envs)) != cudaSuccess) return bail(e, "alloc gap counters");
  if ((e = dalloc(c, &c->d_invalid, n_envs)) != cudaSuccess) return bail(e, "alloc statistics");
  if ((e = dalloc(c, &c->d_events, cfg->event_capacity)) != cudaSuccess) return bail(e, "alloc events");
  if ((e = dalloc(c, &c->d_count, 2)) != cudaSuccess) return bail(e, "alloc count");
  if ((e = dalloc(c, &c->d_stats, static_cast<size_t>(evis::kStatWords) * n_envs)) != cudaSuccess)
    return bail(e, "alloc statistics");
  if ((e = dalloc(c, &c->d_tr_off, 2 * n_envs)) != cudaSuccess) return bail(e, "alloc trace offsets");
  for (int s = 0; s < 2; ++s) {
    if (c->need_L && (e = dalloc(c, &c->d_L[s], c->nc * c->total)) != cudaSuccess) return bail(e, "alloc L");
    if (!c->keep) {
      if ((e = dalloc(c, &c->d_mv[s], 2 * c->total)) != cudaSuccess) return bail(e, "alloc mv");
      if ((e = dalloc(c, &c->d_Z[s], c->total)) != cudaSuccess) return bail(e, "alloc Z");
    }
  }
  std::vector<int64_t> clocks(2 * n_envs);
  for (int i = 0; i < n_envs; ++i) clocks[i] = clocks[n_envs + i] = envs[i].t0_ns;
  cudaStream_t s = c->stream;
  if ((e = cudaMemcpyAsync(c->d_envs, denv.data(), sizeof(DevEnv) * n_envs, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(c->d_clock, clocks.data(), sizeof(int64_t) * 2 * n_envs, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(c->d_tr_off, troff.data(), sizeof(int64_t) * 2 * n_envs, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemsetAsync(c->d_count, 0, 2 * sizeof(unsigned long long), s)) ||
      (e = cudaMemsetAsync(c->d_stats, 0, sizeof(unsigned long long) * evis::kStatWords * n_envs, s)) ||
      (e = cudaMemsetAsync(c->d_gap, 0, sizeof(uint32_t) * 2 * n_envs, s)) ||
      (e = cudaMemsetAsync(c->d_invalid, 0, sizeof(unsigned long long) * n_envs, s)) ||
      // packing pads of the L slots are never written by a step: zero them once
      (c->d_L[0] && (e = cudaMemsetAsync(c->d_L[0], 0, sizeof(float) * c->nc * c->total, s))) ||
      (c->d_L[1] && (e = cudaMemsetAsync(c->d_L[1], 0, sizeof(float) * c->nc * c->total, s))) ||
      (e = cudaMemsetAsync(c->d_flow, 0, sizeof(float) * 2 * n_envs, s)))
    return bail(e, "upload tables");
  if (c->d_tlast) {
    fill_i64<<<1024, 256, 0, s>>>(c->d_tlast, evis::kNoEvent, c->nc * c->total);
    if ((e = cudaGetLastError()) != cudaSuccess) return bail(e, "fill t_last");
  }
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return bail(e, "create sync");
  if ((e = rebuild_groups(c)) != cudaSuccess) return bail(e, "upload tiles");
  c->h_envs = std::move(denv);
  *out = c;
  return EVIS_OK;
}

evis_status evis_step(evis_ctx *c, const float *frames, const float *mv, const float *depth,
                      int64_t dt_ns) {
  if (!c) return EVIS_ERR_INVALID_ARG;
  drop_graphs(c);
  return do_step(c, frames, mv, depth, dt_ns, nullptr, nullptr);
}

evis_status evis_step_trace(evis_ctx *c, const float *frames, const float *mv,
                            const float *depth, int64_t dt_ns, uint64_t *keys, float *Lint) {
  if (!c) return EVIS_ERR_INVALID_ARG;
  if (!keys || !Lint) return fail(c, EVIS_ERR_INVALID_ARG, "null trace buffer");
  if (!evis::aligned(keys, 8) || !evis::aligned(Lint, 4))
    return fail(c, EVIS_ERR_INVALID_ARG, "trace buffers need 8-byte (keys) and 4-byte alignment");
  drop_graphs(c);
  return do_step(c, frames, mv, depth, dt_ns, keys, Lint);
}

evis_status evis_step_host(evis_ctx *c, const float *frames, const float *mv,
                           const float *depth, int64_t dt_ns) {
  if (!c) return EVIS_ERR_INVALID_ARG;
  if (!frames || !mv || !depth) return fail(c, EVIS_ERR_INVALID_ARG, "null input pointer");
  if (dt_ns <= 0 || dt_ns > kMaxDt) return fail(c, EVIS_ERR_INVALID_ARG, "dt_ns must be in 1..2^40");
  const size_t fw = (c->mode == EVIS_IN_RGB || c->nc == 3) ? 3 : 1;
  drop_graphs(c);
  cudaError_t e = ensure_inputs(c);
  if (e != cudaSuccess) return cuda_fail(c, e, "alloc input buffers");
  float **in = c->d_in[c->in_slot];
  if ((e = cudaMemcpyAsync(in[0], frames, sizeof(float) * fw * c->total, cudaMemcpyHostToDevice, c->stream)) ||
      (e = cudaMemcpyAsync(in[1], mv, sizeof(float) * 2 * c->total, cudaMemcpyHostToDevice, c->stream)) ||
      (e = cudaMemcpyAsync(in[2], depth, sizeof(float) * c->total, cudaMemcpyHostToDevice, c->stream)))
    return cuda_fail(c, e, "host to device copy");
  evis_status st = do_step(c, in[0], in[1], in[2], dt_ns, nullptr, nullptr);
  if (st == EVIS_OK) c->in_slot ^= 1;  // keep the previous keyframe's buffers intact
  return st;
}

// Status of a read: pixel-sub-frames beyond the emission limit first, then overflow.
static evis_status read_status(const evis_ctx *c, const unsigned long long cnt[2], int64_t cap) {
  const int64_t produced = static_cast<int64_t>(cnt[0]);
  if (cnt[1] != 0) return EVIS_ERR_RANGE;
  return (produced > c->cfg.event_capacity || produced > cap) ? EVIS_ERR_OVERFLOW : EVIS_OK;
}

// The two counter words, copied on the context's own stream once it is idle.  A copy on the
// legacy default stream would also wait for every blocking stream of the device, such as
// other contexts' steps, and so serialise contexts that overlap on their own streams.
static cudaError_t read_counter(evis_ctx *c, unsigned long long cnt[2]) {
  cudaError_t e = cudaMemcpyAsync(cnt, c->d_count, 2 * sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e;
}

evis_status evis_read_events(evis_ctx *c, evis_event *dst, int64_t cap, int64_t *n_out) {
  if (!c || !n_out || cap < 0 || (cap > 0 && !dst)) return EVIS_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "read sync");
  unsigned long long cnt[2] = {0, 0};
  if ((e = read_counter(c, cnt)) != cudaSuccess) return cuda_fail(c, e, "read count");
  const int64_t produced = static_cast<int64_t>(cnt[0]);
  const int64_t n = std::min<int64_t>(produced, std::min<int64_t>(c->cfg.event_capacity, cap));
  if (n > 0 && (e = cudaMemcpyAsync(dst, c->d_events, sizeof(evis_event) * n, cudaMemcpyDefault,
                                    c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "copy events");
  if ((e = cudaMemsetAsync(c->d_count, 0, 2 * sizeof(unsigned long long), c->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "reset count");
  *n_out = produced;
  return read_status(c, cnt, cap);
}

evis_status evis_read_events_async(evis_ctx *c, evis_event *dst, int64_t cap, int64_t *n_out) {
  if (!c || !n_out || cap < 0 || (cap > 0 && !dst)) return EVIS_ERR_INVALID_ARG;
  cudaError_t e;
  if (!c->copy_ready) {  // first call: the copy stream, its event and the second buffer
    // a set-up that failed part way is retried whole: whatever exists is used, the rest made
    if (!c->copy_stream &&
        (e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(c, e, "copy stream");
    if (!c->copy_done &&
        (e = cudaEventCreateWithFlags(&c->copy_done, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(c, e, "copy event");
    if (!c->d_events_alt && (e = dalloc(c, &c->d_events_alt, c->cfg.event_capacity)) != cudaSuccess)
      return cuda_fail(c, e, "alloc second event buffer");
    if (!c->d_count_alt && (e = dalloc(c, &c->d_count_alt, 2)) != cudaSuccess)
      return cuda_fail(c, e, "alloc second event counter");
    c->copy_ready = true;
  }
  // every step enqueued so far has finished, and so has the previous read-back, whose
  // buffer the next steps will fill
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "read sync");
  if (c->copy_pending) {
    if ((e = cudaEventSynchronize(c->copy_done)) != cudaSuccess) return cuda_fail(c, e, "copy wait");
    c->copy_pending = false;
  }
  unsigned long long cnt[2] = {0, 0};
  if ((e = read_counter(c, cnt)) != cudaSuccess) return cuda_fail(c, e, "read count");
  const int64_t produced = static_cast<int64_t>(cnt[0]);
  const int64_t n = std::min<int64_t>(produced, std::min<int64_t>(c->cfg.event_capacity, cap));
  if (n > 0 && (e = cudaMemcpyAsync(dst, c->d_events, sizeof(evis_event) * n, cudaMemcpyDefault,
                                    c->copy_stream)) != cudaSuccess)
    return cuda_fail(c, e, "copy events");
  if ((e = cudaEventRecord(c->copy_done, c->copy_stream)) != cudaSuccess)
    return cuda_fail(c, e, "copy record");
  c->copy_pending = true;
  // the next steps append to the other buffer, its count zeroed first in stream order;
  // captured graphs hold the old buffer's address
  std::swap(c->d_events, c->d_events_alt);
  std::swap(c->d_count, c->d_count_alt);
  if ((e = cudaMemsetAsync(c->d_count, 0, 2 * sizeof(unsigned long long), c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "reset count");
  drop_graphs(c);
  *n_out = produced;
  return read_status(c, cnt, cap);
}

evis_status evis_read_wait(evis_ctx *c) {
  if (!c) return EVIS_ERR_INVALID_ARG;
  if (c->copy_pending) {
    cudaError_t e = cudaEventSynchronize(c->copy_done);
    if (e != cudaSuccess) return cuda_fail(c, e, "copy wait");
    c->copy_pending = false;
  }
  return EVIS_OK;
}

evis_status evis_event_count(evis_ctx *c, int64_t *n_out) {
  if (!c || !n_out) return EVIS_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "count sync");
  unsigned long long cnt[2] = {0, 0};
  if ((e = read_counter(c, cnt)) != cudaSuccess) return cuda_fail(c, e, "read count");
  *n_out = static_cast<int64_t>(cnt[0]);
  return read_status(c, cnt, INT64_MAX);
}

evis_status evis_events_device(evis_ctx *c, evis_event **events, uint64_t **count) {
  if (!c || !events || !count) return EVIS_ERR_INVALID_ARG;
  *events = reinterpret_cast<evis_event *>(c->d_events);
  *count = reinterpret_cast<uint64_t *>(c->d_count);
  return EVIS_OK;
}

evis_status evis_clear_events(evis_ctx *c) {
  if (!c) return EVIS_ERR_INVALID_ARG;
  cudaError_t e = cudaMemsetAsync(c->d_count, 0, 2 * sizeof(unsigned long long), c->stream);
  return e == cudaSuccess ? EVIS_OK : cuda_fail(c, e, "clear events");
}

evis_status evis_get_state(evis_ctx *c, float *Lref, int64_t *t_last, int64_t *clocks) {
  if (!c) return EVIS_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "state sync");
  if (Lref && (e = cudaMemcpy(Lref, c->d_Lref, sizeof(float) * c->nc * c->total, cudaMemcpyDefault)))
    return cuda_fail(c, e, "copy Lref");
  if (t_last) {
    if (c->d_tlast) {
      if ((e = cudaMemcpy(t_last, c->d_tlast, sizeof(int64_t) * c->nc * c->total, cudaMemcpyDefault)))
        return cuda_fail(c, e, "copy t_last");
    } else {
      std::fill(t_last, t_last + c->nc * c->total, evis::kNoEvent);
    }
  }
  if (clocks && (e = cudaMemcpy(clocks, c->d_clock + c->clk * c->n, sizeof(int64_t) * c->n,
                                cudaMemcpyDefault)))
    return cuda_fail(c, e, "copy clocks");
  return EVIS_OK;
}

evis_status evis_get_gaps(evis_ctx *c, uint32_t *gaps) {
  if (!c || !gaps) return EVIS_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpy(gaps, c->d_gap + c->clk * c->n, sizeof(uint32_t) * c->n, cudaMemcpyDefault);
  return e == cudaSuccess ? EVIS_OK : cuda_fail(c, e, "copy gap counters");
}

evis_status evis_get_stats(evis_ctx *c, uint64_t *keyframes, uint64_t *gaps,
                           uint64_t *invalid_sources) {
  if (!c) return EVIS_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stats sync");
  uint32_t g0 = 0;
  if ((e = cudaMemcpy(&g0, c->d_gap + c->clk * c->n, sizeof g0, cudaMemcpyDeviceToHost)))
    return cuda_fail(c, e, "copy gap counter");
  if (gaps) *gaps = g0;
  if (keyframes) *keyframes = c->have_A ? static_cast<uint64_t>(g0) + 1 : 0;
  if (invalid_sources &&
      (e = cudaMemcpy(invalid_sources, c->d_invalid, sizeof(uint64_t) * c->n, cudaMemcpyDefault)))
    return cuda_fail(c, e, "copy statistics");
  return EVIS_OK;
}

evis_status evis_get_env_stats(evis_ctx *c, evis_env_stats *out) {
  if (!c || !out) return EVIS_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stats sync");
  std::vector<unsigned long long> w(static_cast<size_t>(evis::kStatWords) * c->n);
  uint32_t gaps = 0;
  if ((e = cudaMemcpy(w.data(), c->d_stats, sizeof(unsigned long long) * w.size(), cudaMemcpyDeviceToHost)) ||
      (e = cudaMemcpy(&gaps, c->d_gap + c->clk * c->n, sizeof gaps, cudaMemcpyDeviceToHost)))
    return cuda_fail(c, e, "copy statistics");
  for (int i = 0; i < c->n; ++i) {
    const evis_env_desc &d = c->envs[i];
    const unsigned long long *v = w.data() + static_cast<size_t>(evis::kStatWords) * i;
    evis_env_stats &o = out[i];
    o.target_subframes = static_cast<uint64_t>(d.width - 2 * d.margin) * (d.height - 2 * d.margin) *
                         static_cast<uint64_t>(d.K) * gaps;
    o.holes_a = v[evis::kStatHolesA];
    o.holes_b = v[evis::kStatHolesB];
    o.holes_both = v[evis::kStatHolesBoth];
    o.events_on = v[evis::kStatEventsOn];
    o.events_off = v[evis::kStatEventsOff];
    o.noise_events = v[evis::kStatNoise];
    o.over_limit = v[evis::kStatOverLimit];
  }
  return EVIS_OK;
}

evis_status evis_set_state(evis_ctx *c, const float *Lref, const int64_t *t_last,
                           const int64_t *clocks, const uint32_t *gaps) {
  if (!c) return EVIS_ERR_INVALID_ARG;
  if (!c->have_A) return fail(c, EVIS_ERR_STATE, "set_state needs the retained keyframe (step once first)");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "state sync");
  const size_t px = static_cast<size_t>(c->nc) * c->total;
  if (Lref && (e = cudaMemcpy(c->d_Lref, Lref, sizeof(float) * px, cudaMemcpyDefault)))
    return cuda_fail(c, e, "restore Lref");
  if (t_last && c->d_tlast && (e = cudaMemcpy(c->d_tlast, t_last, sizeof(int64_t) * px, cudaMemcpyDefault)))
    return cuda_fail(c, e, "restore t_last");
  if (clocks && (e = cudaMemcpy(c->d_clock + c->clk * c->n, clocks, sizeof(int64_t) * c->n,
                                cudaMemcpyDefault)))
    return cuda_fail(c, e, "restore clocks");
  if (gaps && (e = cudaMemcpy(c->d_gap + c->clk * c->n, gaps, sizeof(uint32_t) * c->n,
                              cudaMemcpyDefault)))
    return cuda_fail(c, e, "restore gap counters");
  return EVIS_OK;
}

evis_status evis_log_intensity(const float *in, int64_t n, uint32_t mode, float eps, float *out,
                               evis_stream_t stream) {
  if (n < 0 || (n > 0 && (!in || !out)) || (mode != EVIS_IN_LUM && mode != EVIS_IN_RGB) ||
      !std::isfinite(eps) || eps < 0.0f || !evis::aligned(in, 4) || !evis::aligned(out, 4))
    return EVIS_ERR_INVALID_ARG;
  cudaError_t e = evis::launch_log(in, n, mode, eps, out, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? EVIS_OK : EVIS_ERR_CUDA;
}

// Defocus weights (Sec. 3.4): exp(-k^2 / (2 sigma^2)) for k = -r..r, r = int(3 sigma + 0.5),
// normalised to sum 1 in binary64 and rounded to binary32.  Returns r (0: the identity).
static int defocus_weights(float sigma, float *w) {
  const int r = sigma > 0.0f ? static_cast<int>(3.0 * sigma + 0.5) : 0;
  if (r == 0) {
    w[0] = 1.0f;
    return 0;
  }
  double v[2 * evis::kMaxBlurR + 1], sum = 0.0;
  const double s2 = 2.0 * sigma * static_cast<double>(sigma);
  for (int k = -r; k <= r; ++k) sum += (v[k + r] = std::exp(-(static_cast<double>(k) * k) / s2));
  for (int i = 0; i <= 2 * r; ++i) w[i] = static_cast<float>(v[i] / sum);
  return r;
}

static bool defocus_sigma_ok(float s) { return s >= 0.0f && s <= 8.0f; }

evis_status evis_defocus(const float *in, int32_t width, int32_t height, uint32_t mode,
                         float sigma_px, float *out, evis_stream_t stream) {
  if (!in || !out || width < 1 || height < 1 || width > 65535 || height > 65535 ||
      int64_t(width) * height > (int64_t(1) << 24) || (mode != EVIS_IN_LUM && mode != EVIS_IN_RGB) ||
      !defocus_sigma_ok(sigma_px) || !evis::aligned(in, 4) || !evis::aligned(out, 4))
    return EVIS_ERR_INVALID_ARG;
  evis::BlurArgs ba{};
  ba.W = width;
  ba.H = height;
  ba.r = defocus_weights(sigma_px, ba.w);
  ba.in = in;
  ba.out = out;
  ba.mode = mode;
  ba.max_r = ba.r;
  const int tiles = ((width + 63) / 64) * ((height + 31) / 32);
  cudaError_t e = evis::launch_defocus(ba, 1, tiles, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? EVIS_OK : EVIS_ERR_CUDA;
}

evis_status evis_set_defocus(evis_ctx *c, const float *sigma_px) {
  if (!c) return EVIS_ERR_INVALID_ARG;
  bool any = false;
  for (int i = 0; sigma_px && i < c->n; ++i) {
    if (!defocus_sigma_ok(sigma_px[i]))
      return fail(c, EVIS_ERR_INVALID_ARG, "defocus sigma must be in 0..8 pixels");
    any |= sigma_px[i] > 0.0f;
  }
  if (any && c->mode == EVIS_IN_LOG)
    return fail(c, EVIS_ERR_INVALID_ARG, "defocus acts on linear intensity: needs EVIS_IN_LUM or EVIS_IN_RGB");
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  const int taps = 2 * evis::kMaxBlurR + 1;
  if (any && !c->d_blur) {
    if ((e = dalloc(c, &c->d_blur, c->nc * c->total)) != cudaSuccess ||
        (e = dalloc(c, &c->d_blur_w, static_cast<int64_t>(taps) * c->n)) != cudaSuccess)
      return cuda_fail(c, e, "alloc defocus buffers");
  }
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "defocus sync");
  drop_graphs(c);
  std::vector<float> w(static_cast<size_t>(taps) * c->n, 0.0f);
  int rmax = -1;
  for (int i = 0; i < c->n; ++i) {
    const float sg = sigma_px ? sigma_px[i] : 0.0f;
    DevEnv &v = c->h_envs[i];
    v.blur_r = defocus_weights(sg, w.data() + static_cast<size_t>(taps) * i);
    v.blur_off = taps * i;
    rmax = std::max(rmax, v.blur_r);
  }
  if (any && (e = cudaMemcpy(c->d_blur_w, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(c, e, "upload defocus weights");
  if ((e = cudaMemcpy(c->d_envs, c->h_envs.data(), sizeof(DevEnv) * c->n, cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(c, e, "upload defocus radii");
  c->blur_r_max = any ? rmax : -1;
  return EVIS_OK;
}

evis_status evis_set_noise(evis_ctx *c, const evis_noise_desc *nz) {
  if (!c) return EVIS_ERR_INVALID_ARG;
  auto rate = [](float v) { return std::isfinite(v) && v >= 0.0f; };
  for (int i = 0; nz && i < c->n; ++i) {
    const evis_noise_desc &d = nz[i];
    if (!rate(d.leak_hz) || !rate(d.shot_hz) || !rate(d.hot_hz))
      return fail(c, EVIS_ERR_INVALID_ARG, "noise rates must be finite and >= 0");
    if (!(d.hot_fraction >= 0.0f && d.hot_fraction <= 1.0f))
      return fail(c, EVIS_ERR_INVALID_ARG, "hot_fraction must be in 0..1");
    if (!std::isfinite(d.lo) || !std::isfinite(d.hi) || !(d.hi > d.lo))
      return fail(c, EVIS_ERR_INVALID_ARG, "noise range needs finite lo < hi");
  }
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  drop_graphs(c);
  bool any = false;
  int max_px = 0;
  for (int i = 0; i < c->n; ++i) {
    DevEnv &v = c->h_envs[i];
    const evis_noise_desc d = nz ? nz[i] : evis_noise_desc{0, 0, 0, 0, 0, 1, 0};
    v.leak_hz = d.leak_hz;
    v.shot_hz = d.shot_hz;
    v.hot_hz = d.hot_hz;
    v.hot_fraction = d.hot_fraction;
    v.noise_lo = d.lo;
    v.noise_hi = d.hi;
    v.key0 = static_cast<uint32_t>(d.seed);
    v.key1 = static_cast<uint32_t>(d.seed >> 32) ^ static_cast<uint32_t>(i);
    v.noise = (d.leak_hz > 0.0f || d.shot_hz > 0.0f || d.hot_hz > 0.0f) ? 1 : 0;
    any |= v.noise != 0;
    if (v.noise) max_px = std::max(max_px, (v.W - 2 * v.margin) * (v.H - 2 * v.margin));
  }
  // pageable source: the call returns once the table is staged, so h_envs may change after
  if ((e = cudaMemcpyAsync(c->d_envs, c->h_envs.data(), sizeof(DevEnv) * c->n,
                           cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "upload noise parameters");
  c->any_noise = any;
  c->noise_max_px = max_px;
  return EVIS_OK;
}

evis_status evis_set_tile_shape(evis_ctx *c, int32_t tile_w, int32_t tile_h) {
  if (!c) return EVIS_ERR_INVALID_ARG;
  if (!evis::tile_shape_supported(tile_w, tile_h))
    return fail(c, EVIS_ERR_INVALID_ARG, "unsupported tile shape");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "tile shape sync");
  c->env_tw.assign(c->n, tile_w);
  c->env_th.assign(c->n, tile_h);
  if ((e = rebuild_groups(c)) != cudaSuccess) return cuda_fail(c, e, "upload tiles");
  return EVIS_OK;
}

evis_status evis_set_env_tile_shapes(evis_ctx *c, const int32_t *tile_w, const int32_t *tile_h) {
  if (!c || !tile_w || !tile_h) return EVIS_ERR_INVALID_ARG;
  int distinct = 0;
  for (int i = 0; i < c->n; ++i) {
    if (!evis::tile_shape_supported(tile_w[i], tile_h[i]))
      return fail(c, EVIS_ERR_INVALID_ARG, "unsupported tile shape");
    bool seen = false;
    for (int j = 0; j < i; ++j) seen |= tile_w[j] == tile_w[i] && tile_h[j] == tile_h[i];
    distinct += seen ? 0 : 1;
  }
  if (distinct > kMaxGroups) return fail(c, EVIS_ERR_INVALID_ARG, "too many tile shapes");
  c->env_tw.assign(tile_w, tile_w + c->n);
  c->env_th.assign(tile_h, tile_h + c->n);
  drop_graphs(c);
  cudaError_t e = rebuild_groups(c);
  return e == cudaSuccess ? EVIS_OK : cuda_fail(c, e, "upload tiles");
}

evis_status evis_get_tile_shapes(evis_ctx *c, int32_t *tile_w, int32_t *tile_h) {
  if (!c || !tile_w || !tile_h) return EVIS_ERR_INVALID_ARG;
  std::copy(c->env_tw.begin(), c->env_tw.end(), tile_w);
  std::copy(c->env_th.begin(), c->env_th.end(), tile_h);
  return EVIS_OK;
}

evis_status evis_autotune(evis_ctx *c, const float *frames, const float *mv, const float *depth,
                          int64_t dt_ns, int32_t reps, float *best_ms) {
  if (!c) return EVIS_ERR_INVALID_ARG;
  if (!frames || !mv || !depth || reps < 1 || reps > 100 || dt_ns <= 0 || dt_ns > kMaxDt ||
      !evis::aligned(frames, 4) || !evis::aligned(mv, 8) || !evis::aligned(depth, 4))
    return fail(c, EVIS_ERR_INVALID_ARG, "bad autotune arguments");
  if (!c->have_A) return fail(c, EVIS_ERR_STATE, "autotune needs a retained keyframe (step once first)");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "autotune sync");
  if (!c->d_tune_Lref) {
    if ((e = dalloc(c, &c->d_tune_Lref, c->nc * c->total)) != cudaSuccess ||
        (c->d_tlast && (e = dalloc(c, &c->d_tune_tlast, c->nc * c->total)) != cudaSuccess) ||
        (e = dalloc(c, &c->d_tune_tiles, max_tiles(c))) != cudaSuccess)
      return cuda_fail(c, e, "alloc autotune scratch");
  }
  // save the per-pixel state and the event counter; every trial starts from them
  unsigned long long count0[2] = {0, 0};
  if ((e = cudaMemcpy(count0, c->d_count, sizeof count0, cudaMemcpyDeviceToHost)) ||
      (e = cudaMemcpy(c->d_tune_Lref, c->d_Lref, sizeof(float) * c->nc * c->total, cudaMemcpyDeviceToDevice)) ||
      (c->d_tlast && (e = cudaMemcpy(c->d_tune_tlast, c->d_tlast, sizeof(int64_t) * c->nc * c->total,
                                     cudaMemcpyDeviceToDevice))))
    return cuda_fail(c, e, "autotune save");
  KeyframeB B{};
  unsigned long long *stats = c->d_invalid;  // the trial keyframe is not counted
  c->d_invalid = nullptr;
  e = enqueue_prep(c, frames, mv, depth, &B);
  c->d_invalid = stats;
  if (e != cudaSuccess) return cuda_fail(c, e, "autotune prep");
  evis::StepArgs base = step_args(c, B, dt_ns);
  base.env_stats = nullptr;  // trials are not counted
  base.stats = false;
  const int shapes[6][2] = {{32, 16}, {32, 8}, {32, 32}, {64, 16}, {64, 32}, {128, 16}};
  cudaEvent_t ev0, ev1;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  std::vector<int> tw(c->n, 64), th(c->n, 16);
  std::vector<bool> done(c->n, false);
  float total_best = 0.0f;
  for (int i = 0; i < c->n && e == cudaSuccess; ++i) {
    if (done[i]) continue;  // one trial per resolution class (same width and height)
    const int W = c->envs[i].width, H = c->envs[i].height;
    auto in_class = [&](int k) { return c->envs[k].width == W && c->envs[k].height == H; };
    float best = 1e30f;
    for (const auto &sh : shapes) {
      std::vector<Tile> tiles = tiles_for(c, sh[0], sh[1], in_class);
      if ((e = cudaMemcpy(c->d_tune_tiles, tiles.data(), sizeof(Tile) * tiles.size(),
                          cudaMemcpyHostToDevice)) != cudaSuccess)
        break;
      evis::StepArgs s = base;
      s.tiles = c->d_tune_tiles;
      s.n_tiles = static_cast<int>(tiles.size());
      s.work_counter = c->d_work + kMaxGroups - 1;
      float t_min = 1e30f;
      for (int r = 0; r <= reps && e == cudaSuccess; ++r) {  // r = 0 warms up
        // every trial starts from the saved state and event count, so each one writes its
        // events to the same part of the buffer (none is timed past a full buffer)
        if ((e = cudaMemcpyAsync(c->d_count, count0, sizeof count0, cudaMemcpyHostToDevice,
                                 c->stream)) ||
            (e = cudaMemcpyAsync(c->d_Lref, c->d_tune_Lref, sizeof(float) * c->nc * c->total,
                                 cudaMemcpyDeviceToDevice, c->stream)) ||
            (c->d_tlast && (e = cudaMemcpyAsync(c->d_tlast, c->d_tune_tlast, sizeof(int64_t) * c->nc * c->total,
                                                cudaMemcpyDeviceToDevice, c->stream))) ||
            (e = cudaMemsetAsync(s.work_counter, 0, sizeof(unsigned), c->stream)) ||
            (e = cudaEventRecord(ev0, c->stream)) ||
            (e = evis::launch_step(s, sh[0], sh[1], false, c->grid_cap, c->stream)) ||
            (e = cudaEventRecord(ev1, c->stream)) || (e = cudaEventSynchronize(ev1)))
          break;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        if (r > 0) t_min = std::min(t_min, ms);
      }
      if (e != cudaSuccess) break;
      if (t_min < best) {
        best = t_min;
        for (int k = 0; k < c->n; ++k)
          if (in_class(k)) tw[k] = sh[0], th[k] = sh[1];
      }
    }
    for (int k = 0; k < c->n; ++k) done[k] = done[k] || in_class(k);
    total_best += best;
  }
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  // restore the state and the counter whatever happened above
  cudaError_t r = cudaStreamSynchronize(c->stream);
  if (r == cudaSuccess) r = cudaMemcpy(c->d_Lref, c->d_tune_Lref, sizeof(float) * c->nc * c->total, cudaMemcpyDeviceToDevice);
  if (r == cudaSuccess && c->d_tlast)
    r = cudaMemcpy(c->d_tlast, c->d_tune_tlast, sizeof(int64_t) * c->nc * c->total, cudaMemcpyDeviceToDevice);
  if (r == cudaSuccess) r = cudaMemcpy(c->d_count, count0, sizeof count0, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = r;
  if (e != cudaSuccess) return cuda_fail(c, e, "autotune");
  if (best_ms) *best_ms = total_best;
  return evis_set_env_tile_shapes(c, tw.data(), th.data());
}

evis_status evis_input_buffers(evis_ctx *c, float **frames, float **mv, float **depth) {
  if (!c || !frames || !mv || !depth) return EVIS_ERR_INVALID_ARG;
  cudaError_t e = ensure_inputs(c);
  if (e != cudaSuccess) return cuda_fail(c, e, "alloc input buffers");
  *frames = c->d_in[c->in_slot][0];
  *mv = c->d_in[c->in_slot][1];
  *depth = c->d_in[c->in_slot][2];
  return EVIS_OK;
}

evis_status evis_capture(evis_ctx *c, int64_t dt_ns) {
  if (!c) return EVIS_ERR_INVALID_ARG;
  if (dt_ns <= 0 || dt_ns > kMaxDt) return fail(c, EVIS_ERR_INVALID_ARG, "dt_ns must be in 1..2^40");
  if (!c->have_A) return fail(c, EVIS_ERR_STATE, "capture needs a retained keyframe (step once first)");
  if (c->keep) return fail(c, EVIS_ERR_STATE, "capture needs a context without EVIS_KEEP_INPUTS");
  if (c->stream == nullptr) return fail(c, EVIS_ERR_STATE, "capture needs a non-default stream");
  cudaError_t e = ensure_inputs(c);
  if (e != cudaSuccess) return cuda_fail(c, e, "alloc input buffers");
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "capture sync");
  drop_graphs(c);
  const int prof_max = c->prof_max;
  c->prof_max = c->prof_n;  // no profiling events inside graphs
  evis_status st = EVIS_OK;
  for (int ph = 0; ph < 2 && st == EVIS_OK; ++ph) {
    if ((e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
      st = cuda_fail(c, e, "begin capture");
      break;
    }
    float **in = c->d_in[c->in_slot];
    st = do_step(c, in[0], in[1], in[2], dt_ns, nullptr, nullptr);  // records, runs nothing
    c->in_slot ^= 1;
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(c->stream, &g);
    if (st == EVIS_OK && e != cudaSuccess) st = cuda_fail(c, e, "end capture");
    if (st == EVIS_OK && (e = cudaGraphInstantiate(&c->graph[ph], g, 0)) != cudaSuccess)
      st = cuda_fail(c, e, "instantiate graph");
    if (g) cudaGraphDestroy(g);
  }
  c->prof_max = prof_max;
  if (st != EVIS_OK) {
    drop_graphs(c);
    return st;
  }
  // two recorded gaps brought the slots, clocks and input buffers back to where they were
  c->graph_dt = dt_ns;
  c->graph_phase = 0;
  return EVIS_OK;
}

evis_status evis_replay(evis_ctx *c) {
  if (!c) return EVIS_ERR_INVALID_ARG;
  if (!c->graph[c->graph_phase]) return fail(c, EVIS_ERR_STATE, "no captured graph (evis_capture)");
  cudaError_t e = cudaGraphLaunch(c->graph[c->graph_phase], c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "graph launch");
  // the host-side bookkeeping of one evis_step from the input buffers
  c->graph_phase ^= 1;
  c->slot ^= 1;
  c->clk ^= 1;
  c->in_slot ^= 1;
  c->A_L = c->d_L[c->slot];
  c->A_mv = c->d_mv[c->slot];
  c->A_Z = c->d_Z[c->slot];
  return EVIS_OK;
}

evis_status evis_profile_enable(evis_ctx *c, int32_t max_steps) {
  if (!c || max_steps < 0 || max_steps > (1 << 20)) return EVIS_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "profile sync");
  for (cudaEvent_t ev : c->prof) cudaEventDestroy(ev);
  c->prof.clear();
  c->prof_max = c->prof_n = 0;
  for (int i = 0; i < 3 * max_steps; ++i) {
    cudaEvent_t ev;
    if ((e = cudaEventCreate(&ev)) != cudaSuccess) return cuda_fail(c, e, "profile events");
    c->prof.push_back(ev);
  }
  c->prof_max = max_steps;
  return EVIS_OK;
}

evis_status evis_profile_read(evis_ctx *c, float *ms, int32_t cap, int32_t *n_steps) {
  if (!c || !n_steps || cap < 0 || (cap > 0 && !ms)) return EVIS_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "profile sync");
  const int n = std::min(cap, c->prof_n);
  for (int s = 0; s < n; ++s) {
    float a = 0.f, b = 0.f;
    if ((e = cudaEventElapsedTime(&a, c->prof[3 * s], c->prof[3 * s + 1])) != cudaSuccess ||
        (e = cudaEventElapsedTime(&b, c->prof[3 * s + 1], c->prof[3 * s + 2])) != cudaSuccess)
      return cuda_fail(c, e, "profile elapsed");
    ms[2 * s] = a;
    ms[2 * s + 1] = b;
  }
  *n_steps = n;
  return EVIS_OK;
}

evis_status evis_total_pixels(evis_ctx *c, int64_t *n_out) {
  if (!c || !n_out) return EVIS_ERR_INVALID_ARG;
  *n_out = c->total;
  return EVIS_OK;
}

evis_status evis_destroy(evis_ctx *c) {
  if (!c) return EVIS_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  release(c);
  delete c;
  return e == cudaSuccess ? EVIS_OK : EVIS_ERR_CUDA;
}

const char *evis_status_string(evis_status s) {
  switch (s) {
    case EVIS_OK: return "ok";
    case EVIS_ERR_INVALID_ARG: return "invalid argument";
    case EVIS_ERR_CUDA: return "CUDA error";
    case EVIS_ERR_OOM: return "out of device memory";
    case EVIS_ERR_OVERFLOW: return "event buffer overflow";
    case EVIS_ERR_STATE: return "invalid state";
    case EVIS_ERR_TIMEOUT: return "device wait timed out (reserved)";
    case EVIS_ERR_RANGE: return "a pixel exceeded the per-sub-frame crossing limit";
  }
  return "unknown status";
}

const char *evis_last_error(evis_ctx *c) { return c ? c->err.c_str() : g_create_error.c_str(); }

}  // extern "C"
