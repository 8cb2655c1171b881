// evis_step_noalloc: one keyframe gap of one environment that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the time they want events: code running inside a
// host that owns every device allocation itself (a simulator or game engine with its own
// GPU memory pool, a plugin that is handed buffers but may not allocate), or code that must
// not hit the allocator's synchronisation in a latency-critical loop.  They pass every input
// and output buffer; the small per-call tables the synthesis kernels need (environment
// descriptor, tile list, motion bounds of both keyframes, clocks) live in the file-scope
// device array below, which every GPU that loads the library holds until the process exits.
//
// The kernels are the same as evis_step's (prep_kernel and step_kernel); only where their
// scratch lives differs.
#include <mutex>
#include <string>

#include "evis_internal.h"

namespace {

using evis::DevEnv;
using evis::Tile;

// Limits of the entry point (they size the scratch array).
constexpr int kNaMaxSide = 4096;            // width and height
constexpr int64_t kNaMaxPixels = 1 << 20;   // width * height
constexpr int kNaTileW = 64, kNaTileH = 16; // tile shape used by this entry point
constexpr int kNaMaxTiles = 2048;           // >= ceil(W/64) * ceil(H/16) within the limits
constexpr int kNaMaxSegs = 40960;           // >= ceil(W/32) * H within the limits

// Byte layout of the scratch array.
constexpr size_t kOffEnv = 0;
constexpr size_t kOffClock = 256;                                     // int64 [2]
constexpr size_t kOffWork = 384;                                      // unsigned work counter
constexpr size_t kOffFlow = 512;                                      // float [2]
constexpr size_t kOffTiles = 768;                                     // Tile [kNaMaxTiles]
constexpr size_t kOffSeg = kOffTiles + sizeof(Tile) * kNaMaxTiles;    // float4 [2][kNaMaxSegs]
constexpr size_t kScratchBytes = kOffSeg + sizeof(float4) * 2 * kNaMaxSegs;  // ~1.3 MB
static_assert(sizeof(DevEnv) <= 256, "descriptor slot");
static_assert(kOffSeg % 256 == 0, "segment bounds alignment");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch per device (host code must not use the symbol itself).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_scratch_ptr[kMaxDevices] = {};

cudaError_t scratch_for_current_device(unsigned char **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    unsigned char *p = nullptr;
    e = cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Writes the environment descriptor, the tile list and the clocks into the scratch array
// and clears the motion maxima (every call starts from these values).
__global__ void noalloc_setup(unsigned char *scratch, DevEnv env, int tiles_x, int n_tiles,
                              int64_t t_a) {
  Tile *tiles = reinterpret_cast<Tile *>(scratch + kOffTiles);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_tiles; i += gridDim.x * blockDim.x)
    tiles[i] = Tile{0, env.margin + (i % tiles_x) * kNaTileW, env.margin + (i / tiles_x) * kNaTileH, 0};
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *reinterpret_cast<DevEnv *>(scratch + kOffEnv) = env;
    int64_t *clock = reinterpret_cast<int64_t *>(scratch + kOffClock);
    clock[0] = t_a;
    clock[1] = t_a;
    float *flow = reinterpret_cast<float *>(scratch + kOffFlow);
    flow[0] = 0.0f;
    flow[1] = 0.0f;
    *reinterpret_cast<unsigned *>(scratch + kOffWork) = 0u;
  }
}

bool finite_pos(float v) { return v > 0.0f && v < INFINITY; }

}  // namespace

extern "C" evis_status evis_step_noalloc(const evis_env_desc *env, uint32_t flags,
                                         const float *L_A, const float *mv_A, const float *Z_A,
                                         const float *L_B, const float *mv_B, const float *Z_B,
                                         float *Lref, int64_t *t_last, int64_t t_a_ns,
                                         int64_t dt_ns, evis_event *events, uint64_t *count,
                                         int64_t capacity, evis_stream_t stream) {
  auto reject = [](const char *why) {
    evis::set_detached_error(std::string("evis_step_noalloc: ") + why);
    return EVIS_ERR_INVALID_ARG;
  };
  if (!env) return reject("env is null");
  const evis_env_desc &d = *env;
  if (d.width < 1 || d.height < 1 || d.width > kNaMaxSide || d.height > kNaMaxSide ||
      int64_t(d.width) * d.height > kNaMaxPixels)
    return reject("width and height must be in 1..4096 with width*height <= 1048576 "
                  "(the size of the library's static scratch array)");
  if (d.K < 1 || d.K > 4096) return reject("K must be in 1..4096");
  if (!finite_pos(d.c_on) || !finite_pos(d.c_off)) return reject("thresholds must be finite and > 0");
  if ((d.c_on_map == nullptr) != (d.c_off_map == nullptr))
    return reject("give both threshold maps or neither");
  if (!evis::aligned(d.c_on_map, 4) || !evis::aligned(d.c_off_map, 4))
    return reject("threshold maps need 4-byte alignment");
  if (d.refractory_ns < 0) return reject("refractory_ns must be >= 0");
  if (d.margin < 0 || 2 * int64_t(d.margin) >= d.width || 2 * int64_t(d.margin) >= d.height)
    return reject("margin must satisfy 0 <= 2 * margin < min(width, height)");
  if (flags & ~(EVIS_MODE_B_PRIMARY | EVIS_TIE_INDEX))
    return reject("only EVIS_MODE_B_PRIMARY and EVIS_TIE_INDEX are accepted (inputs are log-intensity)");
  if (!L_A || !mv_A || !Z_A || !L_B || !mv_B || !Z_B || !Lref || !count)
    return reject("null buffer");  // count: two 64-bit words (events, pixels over the limit)
  if (!evis::aligned(L_A, 4) || !evis::aligned(Z_A, 4) || !evis::aligned(L_B, 4) ||
      !evis::aligned(Z_B, 4) || !evis::aligned(Lref, 4) || !evis::aligned(mv_A, 8) ||
      !evis::aligned(mv_B, 8) || !evis::aligned(t_last, 8) || !evis::aligned(count, 8) ||
      !evis::aligned(events, 16))
    return reject("misaligned buffer: floats 4 bytes, mv, t_last and count 8, events 16");
  if (d.refractory_ns > 0 && !t_last) return reject("t_last is required with a refractory period");
  if (dt_ns <= 0 || dt_ns > (int64_t(1) << 40)) return reject("dt_ns must be in 1..2^40");
  if (capacity < 0 || capacity > (int64_t(1) << 40) || (capacity > 0 && !events))
    return reject("capacity must be in 0..2^40 with a non-null event buffer");

  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  DevEnv de{};
  de.W = d.width;
  de.H = d.height;
  de.K = d.K;
  de.tile_h = kNaTileH;
  de.pix_off = 0;
  de.segs_x = (d.width + evis::kSegW - 1) / evis::kSegW;
  de.seg_off = 0;
  de.c_on = d.c_on;
  de.c_off = d.c_off;
  de.con_map = d.c_on_map;
  de.coff_map = d.c_off_map;
  de.refractory_ns = d.refractory_ns;
  de.margin = d.margin;
  const int tiles_x = (d.width - 2 * d.margin + kNaTileW - 1) / kNaTileW;  // sensor tiles
  const int n_tiles = tiles_x * ((d.height - 2 * d.margin + kNaTileH - 1) / kNaTileH);
  const int n_segs = de.segs_x * d.height;
  // the size checks above keep both tables inside the scratch array; this guards them
  if (n_tiles < 1 || n_tiles > kNaMaxTiles || n_segs < 1 || n_segs > kNaMaxSegs)
    return reject("the tile or segment table would not fit the scratch array");

  unsigned char *scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) {
    evis::set_detached_error(std::string("evis_step_noalloc: scratch address: ") +
                             cudaGetErrorString(e));
    return EVIS_ERR_CUDA;
  }

  DevEnv *s_env = reinterpret_cast<DevEnv *>(scratch + kOffEnv);
  int64_t *s_clock = reinterpret_cast<int64_t *>(scratch + kOffClock);
  float *s_flow = reinterpret_cast<float *>(scratch + kOffFlow);
  Tile *s_tiles = reinterpret_cast<Tile *>(scratch + kOffTiles);
  float4 *s_seg = reinterpret_cast<float4 *>(scratch + kOffSeg);

  noalloc_setup<<<(n_tiles + 255) / 256, 256, 0, s>>>(scratch, de, tiles_x, n_tiles, t_a_ns);
  if ((e = cudaGetLastError()) != cudaSuccess) goto cuda_error;
  // motion bounds of A (slot 0) and B (slot 1); inputs are read in place
  for (int k = 0; k < 2; ++k) {
    evis::PrepArgs pa{};
    pa.envs = s_env;
    pa.frames = k ? L_B : L_A;
    pa.mv = k ? mv_B : mv_A;
    pa.Z = k ? Z_B : Z_A;
    pa.flow = s_flow + k;
    pa.seg = s_seg + k * kNaMaxSegs;
    pa.mode = EVIS_IN_LOG;
    pa.nc = 1;
    pa.max_segs = n_segs;
    if ((e = evis::launch_prep(pa, 1, s)) != cudaSuccess) goto cuda_error;
  }
  {
    evis::StepArgs sa{};
    sa.envs = s_env;
    sa.tiles = s_tiles;
    sa.n_tiles = n_tiles;
    sa.work_counter = reinterpret_cast<unsigned *>(scratch + kOffWork);
    sa.LA = L_A;
    sa.mvA = mv_A;
    sa.ZA = Z_A;
    sa.LB = L_B;
    sa.mvB = mv_B;
    sa.ZB = Z_B;
    sa.Lref = Lref;
    sa.tlast = t_last;
    sa.clock_in = s_clock;
    sa.clock_out = s_clock + 1;
    sa.flowA = s_flow;
    sa.flowB = s_flow + 1;
    sa.segA = s_seg;
    sa.segB = s_seg + kNaMaxSegs;
    sa.events = reinterpret_cast<ulonglong2 *>(events);
    sa.ev_count = reinterpret_cast<unsigned long long *>(count);
    sa.capacity = static_cast<unsigned long long>(capacity);
    sa.dt = dt_ns;
    sa.flags = flags;
    sa.nc = 1;
    if ((e = evis::launch_step(sa, kNaTileW, kNaTileH, /*trace=*/false, /*grid_cap=*/0, s)) !=
        cudaSuccess)
      goto cuda_error;
  }
  return EVIS_OK;
cuda_error:
  evis::set_detached_error(std::string("evis_step_noalloc: ") + cudaGetErrorString(e));
  return EVIS_ERR_CUDA;
}
