// EVIS event-synthesis ORACLE — test infrastructure, not the product.
//
// A plain, slow, single-threaded C++17 restatement of the data-parallel path of EVIS
// ("bidirectional motion-vector warping with depth splatting" followed by the "HDR event
// formation model").  Only the tests, the smoke check and the benchmark's CPU-baseline leg
// load it; the CUDA library never does, and this file shares no code, header or constant
// table with it.  Compiled with -O2 -ffp-contract=off so every float operation below is one
// IEEE-754 binary32 operation rounded to nearest (no fused multiply-add), which is the
// operation order the CUDA kernels must reproduce bit for bit.
//
// Precision: the decisions the method takes (z-buffer argmin, event count floor) are taken
// in binary32 on both sides; timestamps use one binary64 multiply and llrint.  The paper
// fixes no precision.
//
// Parity status: every function below is pinned by a test under tests/ (brute force,
// closed forms or invariants) except the full event stream of a textured scene, which has
// nothing but this oracle to compare against (parity unpinned beyond these pins).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>

namespace {

// Flag bits of the oracle's configuration word (same numeric meaning as the library's).
constexpr uint32_t IN_MASK = 0x3u, IN_LOG = 0u, IN_LUM = 1u, IN_RGB = 2u;
constexpr uint32_t MODE_B_PRIMARY = 0x10u;  // Sec. 3.3: B primary, A only fills B's holes
constexpr uint32_t MODE_JOINT = 0x40u;      // Eq. 6: one argmin of depth over both directions
constexpr uint32_t TIE_INDEX = 0x20u;       // key = (depth, source index), no weight field
constexpr uint32_t COLOR = 0x200u;          // Sec. 3.2: the event model on R, G and B apart

constexpr uint64_t EMPTY = ~0ull;
// Events one pixel may emit in one sub-frame (per channel).  Eq. 4 bounds n only by the
// input; a pixel-sub-frame with n above this limit emits none of its crossings, still moves
// its reference level by the whole p n C of Eq. 4, and is counted (status 2 of orc_step).
constexpr int MAX_CROSSINGS = 4096;
constexpr int64_t NO_EVENT = std::numeric_limits<int64_t>::min();

struct Env {
  int W, H, K;
  float c_on, c_off;
  int margin;            // rendered pixels cropped on each side (Appendix B); events cover the rest
  int64_t refractory_ns, t0_ns;
  bool has_map;
};

struct Event {  // 16 bytes: t, x, y, env, polarity
  int64_t t_ns;
  uint16_t x, y, env;
  int16_t p;
};

// Sensor non-idealities of one environment (Sec. 3.4); all rates zero = off.
struct Noise {
  float leak_hz, shot_hz, hot_hz;  // event rates per pixel (1/s)
  float hot_fraction;              // probability that a pixel is hot (fixed per pixel)
  float lo, hi;                    // log-intensity range mapped to the normalised intensity
  uint64_t seed;
};

struct Ctx {
  std::vector<Env> envs;
  std::vector<Noise> noise;                // per env (zeros: no noise)
  std::vector<float> defocus;              // per env Gaussian sigma in pixels (0: none)
  uint32_t gap = 0;                        // keyframe gaps processed (the noise counter)
  std::vector<int64_t> off;   // packed pixel offsets (H*W rounded up to 4)
  int64_t total = 0;
  float eps = 1e-4f;
  uint32_t flags = 0;
  int nc = 1;                              // event channels: 1, or 3 (R, G, B) in colour mode
  bool have_A = false;
  std::vector<float> LA, mvA, ZA;          // retained keyframe A (Sec. 3.3 needs A and B)
  std::vector<float> Lref;                 // per channel and pixel: reference level (Sec. 3.2)
  std::vector<int64_t> t_last;             // per channel and pixel: last event time (Sec. 3.4)
  // L, Lref and t_last hold nc planes of `total` values each (channel c at c * total)
  std::vector<float> con, coff;            // per-pixel thresholds (Eq. 8), if any env has them
  std::vector<int64_t> clock;              // time of keyframe A per env
  std::vector<Event> events;
  std::vector<uint64_t> over_limit;        // per env: pixel-sub-frames with n > MAX_CROSSINGS
  bool gap_over_limit = false;             // some pixel-sub-frame of the last gap had one
};

inline bool valid_depth(float z) { return z > 0.0f && z < INFINITY; }

inline uint32_t float_bits(float v) {
  uint32_t u;
  std::memcpy(&u, &v, 4);
  return u;
}

// Eq. 3 (Rec. 709 luminance) and L = log(I + eps) (Sec. 3.2).  The log is taken in binary64
// and rounded once; non-positive or NaN arguments are clamped to the smallest normal float.
float log_intensity(float I, float eps) {
  float s = I + eps;
  if (!(s > 0.0f)) s = std::numeric_limits<float>::min();
  return static_cast<float>(std::log(static_cast<double>(s)));
}

float rec709(float R, float G, float B) {
  float a = 0.2126f * R;
  float b = 0.7152f * G;
  float c = 0.0722f * B;
  return (a + b) + c;
}

// Bilinear footprint z-test splat of one source (Sec. 3.3, Eq. 6).  The target q is spread
// over the integer pixels around it; a pixel belongs to the footprint iff its bilinear weight
// is > 0 and it lies inside the image.  The z-buffer keeps the smallest 64-bit key
// [depth bits | quantised (1 - weight) | source index]: nearest surface first, then the larger
// bilinear weight, then the lower source index.
void splat_source(uint64_t* zbuf, int W, int H, float qx, float qy, float Zt, uint32_t src,
                  bool tie_index) {
  // No footprint pixel can be inside unless -1 < q < size; this also rejects NaN.
  if (!(qx > -1.0f && qx < static_cast<float>(W) && qy > -1.0f && qy < static_cast<float>(H)))
    return;
  float fx0 = std::floor(qx), fy0 = std::floor(qy);
  float ax = qx - fx0, ay = qy - fy0;
  int x0 = static_cast<int>(fx0), y0 = static_cast<int>(fy0);
  float wx[2] = {1.0f - ax, ax};
  float wy[2] = {1.0f - ay, ay};
  uint64_t hi = static_cast<uint64_t>(float_bits(Zt)) << 32;
  for (int dy = 0; dy < 2; ++dy) {
    for (int dx = 0; dx < 2; ++dx) {
      float w = wx[dx] * wy[dy];
      int cx = x0 + dx, cy = y0 + dy;
      if (!(w > 0.0f) || cx < 0 || cx >= W || cy < 0 || cy >= H) continue;
      uint32_t wq = 0;
      if (!tie_index) {
        uint32_t v = static_cast<uint32_t>((1.0f - w) * 256.0f);
        wq = v < 255u ? v : 255u;
      }
      uint64_t key = hi | (static_cast<uint64_t>(wq) << 24) | src;
      uint64_t& slot = zbuf[static_cast<size_t>(cy) * W + cx];
      if (key < slot) slot = key;
    }
  }
}

// Depth of the other keyframe at the correspondence endpoint (Eq. 7 needs Z_A(p_A) and
// Z_B(p_B)): nearest pixel, rounding half up; the source's own depth when the endpoint
// falls outside the image or has no valid depth.
float other_depth(const float* Zother, int W, int H, float ux, float uy, float own) {
  float nx = std::floor(ux + 0.5f), ny = std::floor(uy + 0.5f);
  if (!(nx >= 0.0f && nx <= static_cast<float>(W - 1) && ny >= 0.0f &&
        ny <= static_cast<float>(H - 1)))
    return own;
  float z = Zother[static_cast<size_t>(ny) * W + static_cast<size_t>(nx)];
  return valid_depth(z) ? z : own;
}

// Splat every source of keyframe A forward (q_A = p - f m_A, Eq. 5) with
// Z~ = (1-f) Z_A(p) + f Z_B(p - m_A(p)) (Eq. 7; m_A reused as the forward velocity).
void splat_A(uint64_t* zbuf, int W, int H, const float* mvA, const float* ZA, const float* ZB,
             float f, float g, bool tie_index) {
  for (int y = 0; y < H; ++y) {
    for (int x = 0; x < W; ++x) {
      size_t p = static_cast<size_t>(y) * W + x;
      float zs = ZA[p];
      if (!valid_depth(zs)) continue;
      float mx = mvA[2 * p], my = mvA[2 * p + 1];
      float qx = static_cast<float>(x) - f * mx;
      float qy = static_cast<float>(y) - f * my;
      float zo = other_depth(ZB, W, H, static_cast<float>(x) - mx, static_cast<float>(y) - my, zs);
      float zt = g * zs + f * zo;
      splat_source(zbuf, W, H, qx, qy, zt, static_cast<uint32_t>(p), tie_index);
    }
  }
}

// Splat every source of keyframe B backward (q_B = p + (1-f) m_B, Eq. 5) with
// Z~ = (1-f) Z_A(p + m_B(p)) + f Z_B(p) (Eq. 7; m_B is the exact B->A correspondence).
void splat_B(uint64_t* zbuf, int W, int H, const float* mvB, const float* ZA, const float* ZB,
             float f, float g, bool tie_index) {
  for (int y = 0; y < H; ++y) {
    for (int x = 0; x < W; ++x) {
      size_t p = static_cast<size_t>(y) * W + x;
      float zs = ZB[p];
      if (!valid_depth(zs)) continue;
      float mx = mvB[2 * p], my = mvB[2 * p + 1];
      float qx = static_cast<float>(x) + g * mx;
      float qy = static_cast<float>(y) + g * my;
      float zo = other_depth(ZA, W, H, static_cast<float>(x) + mx, static_cast<float>(y) + my, zs);
      float zt = g * zo + f * zs;
      splat_source(zbuf, W, H, qx, qy, zt, static_cast<uint32_t>(p), tie_index);
    }
  }
}

// Threshold crossings of one pixel at one substep (Eq. 4 and the reference update of
// Sec. 3.2, with the per-pixel thresholds of Eq. 8 and the refractory period of Sec. 3.4).
// Each crossed level Lref + p k theta is timestamped by linear interpolation between the
// previous defined sample (t_prev, L_prev) and this one (t_i, L).
void cross_pixel(Ctx& c, int env, int x, int y, int ch, float L, float& Lref, float& Lprev,
                 int64_t& tprev, int64_t ti, int64_t& tlast, float th_on, float th_off,
                 int64_t refr) {
  float d = L - Lref;
  int pol = d > 0.0f ? 1 : -1;
  float th = pol > 0 ? th_on : th_off;
  float q = std::fabs(d) / th;
  float nf = q >= 1.0f ? std::floor(q) : 0.0f;  // n of Eq. 4 (NaN compares false: n = 0)
  if (nf > static_cast<float>(MAX_CROSSINGS)) {
    // beyond the emission limit: no crossing of this pixel-sub-frame is emitted (none is
    // truncated either); the reference update of Eq. 4 is the exact one
    ++c.over_limit[env];
    c.gap_over_limit = true;
    Lref = Lref + (pol > 0 ? nf : -nf) * th;
    Lprev = L;
    tprev = ti;
    return;
  }
  int n = static_cast<int>(nf);
  float lev = Lref;
  for (int k = 1; k <= n; ++k) {
    lev = Lref + static_cast<float>(pol * k) * th;
    float num = lev - Lprev;
    float den = L - Lprev;
    float fr = den == 0.0f ? 1.0f : num / den;
    if (!(fr > 0.0f)) fr = 0.0f;
    else if (fr > 1.0f) fr = 1.0f;
    int64_t t = tprev + std::llrint(static_cast<double>(fr) * static_cast<double>(ti - tprev));
    if (refr <= 0 || tlast == NO_EVENT || t - tlast >= refr) {
      c.events.push_back(Event{t, static_cast<uint16_t>(x), static_cast<uint16_t>(y),
                               static_cast<uint16_t>(env), static_cast<int16_t>(pol * (1 + ch))});
      tlast = t;
    }
  }
  if (n > 0) Lref = lev;  // keeps the sub-threshold residual (Sec. 3.2)
  Lprev = L;
  tprev = ti;
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as easy as 1, 2,
// 3", SC 2011): ten rounds of two 32x32->64 multiplies, the key bumped by the Weyl
// constants between rounds.
void philox4x32_10(uint32_t ctr[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = static_cast<uint64_t>(0xD2511F53u) * ctr[0];
    const uint64_t p1 = static_cast<uint64_t>(0xCD9E8D57u) * ctr[2];
    const uint32_t hi0 = static_cast<uint32_t>(p0 >> 32), lo0 = static_cast<uint32_t>(p0);
    const uint32_t hi1 = static_cast<uint32_t>(p1 >> 32), lo1 = static_cast<uint32_t>(p1);
    const uint32_t n0 = hi1 ^ ctr[1] ^ k0, n2 = hi0 ^ ctr[3] ^ k1;
    ctr[0] = n0;
    ctr[1] = lo1;
    ctr[2] = n2;
    ctr[3] = lo0;
  }
}

// Bernoulli draw with probability p from a 32-bit uniform (24 bits used, binary32 compare).
inline bool fires(uint32_t u, float p) { return static_cast<float>(u >> 8) < p * 16777216.0f; }

// Leak, shot and hot-pixel events of one keyframe gap of environment e (Sec. 3.4).  They
// pass no refractory filter, leave the reference levels unchanged and depend only on the
// gap's two keyframes.  Per sensor pixel, channel ch and sub-frame i, over [t_{i-1}, t_i)
// with d = t_i - t_{i-1} ns and dts = d 1e-9 s, the sources compete:
//   leak  p_leak = leak_hz dts;
//   shot  p_shot = shot_hz dts (1 - clamp((L_i - lo) / (hi - lo), 0, 1)), where
//         L_i = (1 - f) LA + f LB (f = i / K) is the pixel's own log intensity between the
//         keyframes, so darker pixels fire more;
//   hot   p_hot = hot_hz dts for the fixed hot subset, 0 elsewhere.
// One uniform word u picks at most one of them: with x = (float)(u >> 8), leak when
// x < p_leak 2^24, else shot when x < (p_leak + p_shot) 2^24, else hot when
// x < (p_leak + p_shot + p_hot) 2^24 (probabilities and sums in binary32, left to right).
// Words: Philox4x32-10 at (pixel, gap, floor((i - 1) / 4), 4 ch), word (i - 1) mod 4.  A
// fired event takes its time t_{i-1} + floor(v d / 2^32) from word 0 of (pixel, gap, i,
// 1 + 4 ch) and, for shot noise, its polarity from bit 0 of word 3 (1: ON); leak and hot
// events are ON.  The hot subset: word 0 of (pixel, 2^32 - 1, 0, 2 + 4 ch) fires with
// probability hot_fraction.  The pixel index is the sensor's, y * W + x inside the margin.
void noise_gap(Ctx& c, int e, const float* LB, int64_t dt) {
  const Noise& nz = c.noise[e];
  if (!(nz.leak_hz > 0.0f || nz.shot_hz > 0.0f || nz.hot_hz > 0.0f)) return;
  const Env& en = c.envs[e];
  const int W = en.W, K = en.K, m = en.margin, SW = en.W - 2 * m, SH = en.H - 2 * m;
  const size_t o = static_cast<size_t>(c.off[e]), plane = static_cast<size_t>(c.total);
  const uint32_t k0 = static_cast<uint32_t>(nz.seed);
  const uint32_t k1 = static_cast<uint32_t>(nz.seed >> 32) ^ static_cast<uint32_t>(e);
  const int64_t T0 = c.clock[e];
  const float inv_range = 1.0f / (nz.hi - nz.lo);
  for (int ch = 0; ch < c.nc; ++ch) {
    const uint32_t cw = 4u * static_cast<uint32_t>(ch);
    for (int sy = 0; sy < SH; ++sy) {
      for (int sx = 0; sx < SW; ++sx) {
        const uint32_t pix = static_cast<uint32_t>(sy * SW + sx);
        const size_t t = static_cast<size_t>(sy + m) * W + (sx + m);
        const float la = c.LA[ch * plane + o + t], lb = LB[ch * plane + t];
        uint32_t rh[4] = {pix, 0xFFFFFFFFu, 0u, 2u + cw};
        philox4x32_10(rh, k0, k1);
        const bool hot = nz.hot_hz > 0.0f && fires(rh[0], nz.hot_fraction);
        uint32_t r[4] = {0u, 0u, 0u, 0u};
        for (int i = 1; i <= K; ++i) {
          const int64_t t0 = T0 + (static_cast<int64_t>(i - 1) * dt) / K;
          const int64_t d = T0 + (static_cast<int64_t>(i) * dt) / K - t0;
          if ((i - 1) % 4 == 0) {
            r[0] = pix;
            r[1] = c.gap;
            r[2] = static_cast<uint32_t>((i - 1) / 4);
            r[3] = cw;
            philox4x32_10(r, k0, k1);
          }
          const uint32_t u = r[(i - 1) % 4];
          const float dts = static_cast<float>(d) * 1e-9f;
          const float f = static_cast<float>(i) / static_cast<float>(K);
          const float L = (1.0f - f) * la + f * lb;
          float ib = (L - nz.lo) * inv_range;
          ib = ib < 0.0f ? 0.0f : (ib > 1.0f ? 1.0f : ib);
          const float s1 = nz.leak_hz * dts;
          const float s2 = s1 + nz.shot_hz * dts * (1.0f - ib);
          const float s3 = hot ? s2 + nz.hot_hz * dts : s2;
          const float x = static_cast<float>(u >> 8);
          if (!(x < s3 * 16777216.0f)) continue;
          uint32_t rt[4] = {pix, c.gap, static_cast<uint32_t>(i), 1u + cw};
          philox4x32_10(rt, k0, k1);
          const bool leak = x < s1 * 16777216.0f, shot = !leak && x < s2 * 16777216.0f;
          const int p = (shot && !(rt[3] & 1u)) ? -1 : 1;
          const int64_t te = t0 + static_cast<int64_t>((static_cast<unsigned __int128>(rt[0]) *
                                                        static_cast<uint64_t>(d)) >> 32);
          c.events.push_back(Event{te, static_cast<uint16_t>(sx), static_cast<uint16_t>(sy),
                                   static_cast<uint16_t>(e), static_cast<int16_t>(p * (1 + ch))});
        }
      }
    }
  }
}

// One keyframe gap of one environment: K substeps f = i/K (Sec. 3.3), each a bidirectional
// splat, a time blend with hole filling, and the event model.  Optional trace outputs:
// keys[(i-1)*2 + dir][p] and Lint[(i-1)*nc + channel][p] (NaN where the pixel got no sample).
void run_pair(Ctx& c, int e, const float* LB, const float* mvB, const float* ZB, int64_t dt,
              uint64_t* keys, float* Lint) {
  const Env& en = c.envs[e];
  const int W = en.W, H = en.H, K = en.K;
  const size_t HW = static_cast<size_t>(W) * H;
  const size_t o = static_cast<size_t>(c.off[e]);
  const size_t plane = static_cast<size_t>(c.total);  // channel stride of L, Lref, t_last
  const int nc = c.nc;
  const float* mvA = c.mvA.data() + 2 * o;
  const float* ZA = c.ZA.data() + o;
  const int64_t T0 = c.clock[e];
  const bool tie_index = (c.flags & TIE_INDEX) != 0;
  const bool b_primary = (c.flags & MODE_B_PRIMARY) != 0;
  const bool joint = (c.flags & MODE_JOINT) != 0;

  std::vector<float> Lprev(nc * HW);
  for (int ch = 0; ch < nc; ++ch)
    std::copy(c.LA.data() + ch * plane + o, c.LA.data() + ch * plane + o + HW, Lprev.begin() + ch * HW);
  std::vector<int64_t> tprev(nc * HW, T0);
  std::vector<uint64_t> zA(HW), zB(HW);
  for (int i = 1; i <= K; ++i) {
    float f = static_cast<float>(i) / static_cast<float>(K);
    float g = 1.0f - f;
    int64_t ti = T0 + (static_cast<int64_t>(i) * dt) / K;
    std::fill(zA.begin(), zA.end(), EMPTY);
    std::fill(zB.begin(), zB.end(), EMPTY);
    splat_A(zA.data(), W, H, mvA, ZA, ZB, f, g, tie_index);
    splat_B(zB.data(), W, H, mvB, ZA, ZB, f, g, tie_index);
    if (keys) {
      std::memcpy(keys + (static_cast<size_t>(i - 1) * 2) * HW, zA.data(), HW * 8);
      std::memcpy(keys + (static_cast<size_t>(i - 1) * 2 + 1) * HW, zB.data(), HW * 8);
    }
    // targets: the sensor, i.e. the rendered frame without its margin (Appendix B); every
    // rendered pixel splats, and events carry sensor coordinates
    const int m = en.margin;
    for (int y = m; y < H - m; ++y) {
      for (int x = m; x < W - m; ++x) {
        size_t t = static_cast<size_t>(y) * W + x;
        const int sx = x - m, sy = y - m;
        bool hasA = zA[t] != EMPTY, hasB = zB[t] != EMPTY;
        // one set of winners serves every channel (it depends on motion and depth only)
        for (int ch = 0; ch < nc; ++ch) {
          const float* LAc = c.LA.data() + ch * plane + o;
          const float* LBc = LB + ch * plane;
          float la = hasA ? LAc[zA[t] & 0xFFFFFFu] : 0.0f;
          float lb = hasB ? LBc[zB[t] & 0xFFFFFFu] : 0.0f;
          float L;
          if (joint) {      // Eq. 6: the nearer of the two winners; equal depths go to B
            const uint32_t za = static_cast<uint32_t>(zA[t] >> 32), zb2 = static_cast<uint32_t>(zB[t] >> 32);
            if (hasA && hasB) L = za < zb2 ? la : lb;
            else if (hasA) L = la;
            else if (hasB) L = lb;
            else L = NAN;
          } else if (b_primary) {  // Sec. 3.3: backward-warped B is primary, A fills B's holes
            if (hasB) L = lb;
            else if (hasA) L = la;
            else L = NAN;
          } else {          // time blend of both directions, hole filled from the other one
            if (hasA && hasB) L = g * la + f * lb;
            else if (hasA) L = la;
            else if (hasB) L = lb;
            else L = NAN;
          }
          if (Lint) Lint[(static_cast<size_t>(i - 1) * nc + ch) * HW + t] = L;
          if (!hasA && !hasB) continue;  // no sample this substep: the pixel holds its state
          float th_on = en.c_on, th_off = en.c_off;
          if (en.has_map) {  // one threshold map for all channels
            th_on = c.con[o + t];
            th_off = c.coff[o + t];
          }
          cross_pixel(c, e, sx, sy, ch, L, c.Lref[ch * plane + o + t], Lprev[ch * HW + t],
                      tprev[ch * HW + t], ti, c.t_last[ch * plane + o + t], th_on, th_off,
                      en.refractory_ns);
        }
      }
    }
  }
}

// Defocus (Sec. 3.4): the linear intensity convolved with a separable Gaussian of standard
// deviation sigma pixels.  Taps k = -r..r with r = int(3 sigma + 0.5); weights
// exp(-k^2 / (2 sigma^2)) normalised to sum 1 in binary64, then rounded to binary32.  Edges
// repeat the border pixel.  The horizontal pass runs first, then the vertical pass on its
// result; each sums its taps in binary32 in the order k = -r..r.
int defocus_radius(float sigma) { return sigma > 0.0f ? static_cast<int>(3.0 * sigma + 0.5) : 0; }

std::vector<float> defocus_weights(float sigma) {
  const int r = defocus_radius(sigma);
  if (r == 0) return {1.0f};
  std::vector<double> w(2 * r + 1);
  double sum = 0.0;
  for (int k = -r; k <= r; ++k) {
    w[k + r] = std::exp(-(static_cast<double>(k) * k) / (2.0 * sigma * static_cast<double>(sigma)));
    sum += w[k + r];
  }
  std::vector<float> out(w.size());
  for (size_t i = 0; i < w.size(); ++i) out[i] = static_cast<float>(w[i] / sum);
  return out;
}

void defocus_plane(const float* in, int W, int H, float sigma, float* out) {
  const std::vector<float> w = defocus_weights(sigma);
  const int r = static_cast<int>(w.size() / 2);
  std::vector<float> h(static_cast<size_t>(W) * H);
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      float acc = 0.0f;
      for (int k = -r; k <= r; ++k) {
        const int xs = std::min(std::max(x + k, 0), W - 1);
        acc += w[k + r] * in[static_cast<size_t>(y) * W + xs];
      }
      h[static_cast<size_t>(y) * W + x] = acc;
    }
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      float acc = 0.0f;
      for (int k = -r; k <= r; ++k) {
        const int ys = std::min(std::max(y + k, 0), H - 1);
        acc += w[k + r] * h[static_cast<size_t>(ys) * W + x];
      }
      out[static_cast<size_t>(y) * W + x] = acc;
    }
}

// Log-intensity planes of a keyframe (Sec. 3.2, Eq. 3): one plane (log of the luminance, or
// the given log-intensity), or in colour mode the R, G and B planes (log of each channel, or
// the given planar log-intensities).  Defocus blurs the linear plane before the log.
void to_log(const Ctx& c, const float* frames, std::vector<float>& L) {
  const size_t plane = static_cast<size_t>(c.total);
  L.assign(c.nc * plane, 0.0f);
  uint32_t mode = c.flags & IN_MASK;
  for (size_t e = 0; e < c.envs.size(); ++e) {
    size_t o = static_cast<size_t>(c.off[e]);
    size_t n = static_cast<size_t>(c.envs[e].W) * c.envs[e].H;
    for (int ch = 0; ch < c.nc; ++ch) {
      float* Lc = L.data() + ch * plane + o;
      if (mode == IN_LOG) {
        std::copy(frames + ch * plane + o, frames + ch * plane + o + n, Lc);
        continue;
      }
      std::vector<float> I(n);  // the linear plane
      for (size_t p = 0; p < n; ++p) {
        const float* px = frames + 3 * (o + p);
        I[p] = mode == IN_LUM ? frames[o + p] : (c.nc == 3 ? px[ch] : rec709(px[0], px[1], px[2]));
      }
      if (c.defocus[e] > 0.0f) {
        std::vector<float> B(n);
        defocus_plane(I.data(), c.envs[e].W, c.envs[e].H, c.defocus[e], B.data());
        I.swap(B);
      }
      for (size_t p = 0; p < n; ++p) Lc[p] = log_intensity(I[p], c.eps);
    }
  }
}

}  // namespace

extern "C" {

typedef struct {
  int32_t width, height, K;
  float c_on, c_off;
  int32_t margin;          // over-render margin per side, 0 <= 2 margin < min(width, height)
  const float* c_on_map;   // optional host [H*W]
  const float* c_off_map;
  int64_t refractory_ns;
  int64_t t0_ns;
} orc_env;

// Returns a new oracle context or null on invalid arguments.
void* orc_create(const orc_env* envs, int32_t n_envs, float eps, uint32_t flags) {
  if (!envs || n_envs <= 0 || n_envs > 65536 || !(eps >= 0.0f)) return nullptr;
  if ((flags & IN_MASK) == 3u) return nullptr;
  if ((flags & MODE_JOINT) && (flags & MODE_B_PRIMARY)) return nullptr;
  if ((flags & COLOR) && (flags & IN_MASK) == IN_LUM) return nullptr;  // colour needs RGB or planes
  Ctx* c = new Ctx();
  c->eps = eps;
  c->flags = flags;
  c->nc = (flags & COLOR) ? 3 : 1;
  bool any_map = false;
  for (int i = 0; i < n_envs; ++i) {
    const orc_env& d = envs[i];
    if (d.width <= 0 || d.height <= 0 || d.width > 65535 || d.height > 65535 ||
        static_cast<int64_t>(d.width) * d.height > (1 << 24) || d.K < 1 ||
        !(d.c_on > 0.0f) || !(d.c_off > 0.0f) || d.refractory_ns < 0 ||
        ((d.c_on_map == nullptr) != (d.c_off_map == nullptr)) || d.margin < 0 ||
        2 * static_cast<int64_t>(d.margin) >= d.width || 2 * static_cast<int64_t>(d.margin) >= d.height) {
      delete c;
      return nullptr;
    }
    c->envs.push_back(Env{d.width, d.height, d.K, d.c_on, d.c_off, d.margin, d.refractory_ns,
                          d.t0_ns, d.c_on_map != nullptr});
    c->off.push_back(c->total);
    c->total += (static_cast<int64_t>(d.width) * d.height + 3) / 4 * 4;
    any_map |= d.c_on_map != nullptr;
  }
  if (any_map) {
    c->con.assign(c->total, 0.0f);
    c->coff.assign(c->total, 0.0f);
    for (int i = 0; i < n_envs; ++i) {
      if (!envs[i].c_on_map) continue;
      size_t n = static_cast<size_t>(envs[i].width) * envs[i].height;
      std::memcpy(c->con.data() + c->off[i], envs[i].c_on_map, n * 4);
      std::memcpy(c->coff.data() + c->off[i], envs[i].c_off_map, n * 4);
    }
  }
  c->noise.assign(n_envs, Noise{0, 0, 0, 0, 0, 1, 0});
  c->defocus.assign(n_envs, 0.0f);
  c->Lref.assign(c->nc * c->total, 0.0f);
  c->t_last.assign(c->nc * c->total, NO_EVENT);
  for (int i = 0; i < n_envs; ++i) c->clock.push_back(envs[i].t0_ns);
  c->over_limit.assign(n_envs, 0);
  return c;
}

void orc_destroy(void* h) { delete static_cast<Ctx*>(h); }

// One keyframe (host arrays in the packed layout).  The first call only sets the reference
// level to the keyframe's log-intensity; each later call synthesises the K substeps between
// the retained keyframe and this one and appends the events.  Trace pointers (optional)
// receive, per env in order, K*2*H*W keys and K*H*W interpolated values.  Returns 0, 1 for
// rejected arguments, or 2 when some pixel-sub-frame of this gap had more crossings than a
// pixel may emit (the gap is otherwise complete; see cross_pixel).
int32_t orc_step(void* h, const float* frames, const float* mv, const float* depth,
                 int64_t dt_ns, uint64_t* trace_keys, float* trace_L) {
  Ctx& c = *static_cast<Ctx*>(h);
  if (!frames || !mv || !depth || dt_ns <= 0) return 1;
  std::vector<float> LB;
  to_log(c, frames, LB);
  if (!c.have_A) {
    c.Lref = LB;
    c.LA = LB;
    c.mvA.assign(mv, mv + 2 * c.total);
    c.ZA.assign(depth, depth + c.total);
    c.have_A = true;
    return 0;
  }
  size_t tk = 0, tl = 0;
  c.gap_over_limit = false;
  for (size_t e = 0; e < c.envs.size(); ++e) {
    size_t o = static_cast<size_t>(c.off[e]);
    size_t HW = static_cast<size_t>(c.envs[e].W) * c.envs[e].H;
    noise_gap(c, static_cast<int>(e), LB.data() + o, dt_ns);
    run_pair(c, static_cast<int>(e), LB.data() + o, mv + 2 * o, depth + o, dt_ns,
             trace_keys ? trace_keys + tk : nullptr, trace_L ? trace_L + tl : nullptr);
    tk += static_cast<size_t>(c.envs[e].K) * 2 * HW;
    tl += static_cast<size_t>(c.envs[e].K) * c.nc * HW;
    c.clock[e] += dt_ns;
  }
  ++c.gap;
  c.LA = LB;
  c.mvA.assign(mv, mv + 2 * c.total);
  c.ZA.assign(depth, depth + c.total);
  return c.gap_over_limit ? 2 : 0;
}

typedef struct {
  float leak_hz, shot_hz, hot_hz, hot_fraction, lo, hi;
  uint64_t seed;
} orc_noise;

// Per-environment noise parameters (array of n_envs); 0 on success.
int32_t orc_set_noise(void* h, const orc_noise* nz) {
  Ctx& c = *static_cast<Ctx*>(h);
  for (size_t e = 0; e < c.envs.size(); ++e) {
    const orc_noise& n = nz[e];
    auto rate = [](float v) { return std::isfinite(v) && v >= 0.0f; };
    if (!(rate(n.leak_hz) && rate(n.shot_hz) && rate(n.hot_hz) && n.hot_fraction >= 0 &&
          n.hot_fraction <= 1 && std::isfinite(n.lo) && std::isfinite(n.hi) && n.hi > n.lo))
      return 1;
    c.noise[e] = Noise{n.leak_hz, n.shot_hz, n.hot_hz, n.hot_fraction, n.lo, n.hi, n.seed};
  }
  return 0;
}

// Per-environment defocus sigma in pixels (array of n_envs; 0 = none, at most 8).  Needs
// linear inputs (luminance or RGB).  0 on success.
int32_t orc_set_defocus(void* h, const float* sigma) {
  Ctx& c = *static_cast<Ctx*>(h);
  for (size_t e = 0; e < c.envs.size(); ++e)
    if (!(sigma[e] >= 0.0f && sigma[e] <= 8.0f)) return 1;
  bool any = false;
  for (size_t e = 0; e < c.envs.size(); ++e) any |= sigma[e] > 0.0f;
  if (any && (c.flags & IN_MASK) == IN_LOG) return 1;
  c.defocus.assign(sigma, sigma + c.envs.size());
  return 0;
}

// Rec. 709 luminance of n RGB triples (Eq. 3).
void orc_rec709(const float* rgb, int64_t n, float* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = rec709(rgb[3 * i], rgb[3 * i + 1], rgb[3 * i + 2]);
}

// Defocus of one linear plane [H][W] (for the blur's own tests).
void orc_defocus(const float* in, int32_t W, int32_t H, float sigma, float* out) {
  defocus_plane(in, W, H, sigma, out);
}

// The binary32 weights of a defocus sigma (2 r + 1 of them; returns r).
int32_t orc_defocus_weights(float sigma, float* out) {
  const std::vector<float> w = defocus_weights(sigma);
  std::memcpy(out, w.data(), w.size() * sizeof(float));
  return static_cast<int32_t>(w.size() / 2);
}

typedef struct {
  int32_t width, height;  // sensor
  int64_t t0_ns, t1_ns;   // the segment [t0, t1]; 0 < t1 - t0 < 2^32
} orc_voxel_env;

// Event voxel grid (the speed-regression input of the paper's appendix): per environment,
// polarity (0: ON, p > 0; 1: OFF, p < 0) and bin b = 0..B-1, the events linearly
// interpolated along time and each bin divided by its largest value.  An event at time t
// sits at tau = (B - 1)(t - t0) / (t1 - t0) and adds 1 - frac(tau) to bin floor(tau) and
// frac(tau) to the next one.  Weights are in units of 2^-16 so that the sums are exact
// integers: with D = t1 - t0, N = (B - 1)(t - t0), b = N / D and r = N mod D,
// w_next = floor(r 2^16 / D) and w_b = 2^16 - w_next.  Events outside the segment or the
// sensor, or of an environment >= n_envs, are skipped.  acc [sum 2 B H W] receives the
// sums (uint32), out the normalised grid: acc / max(acc over the bin's plane), 0 for an empty
// plane, one binary32 division of the two sums rounded to binary32.
void orc_voxel_grid(const Event* ev, int64_t n, const orc_voxel_env* envs, int32_t n_envs,
                    int32_t bins, uint32_t* acc, float* out) {
  std::vector<int64_t> off(n_envs + 1, 0);
  for (int e = 0; e < n_envs; ++e)
    off[e + 1] = off[e] + 2LL * bins * envs[e].width * envs[e].height;
  std::fill(acc, acc + off[n_envs], 0u);
  for (int64_t k = 0; k < n; ++k) {
    const Event& v = ev[k];
    if (v.env >= n_envs) continue;
    const orc_voxel_env& E = envs[v.env];
    if (v.x >= E.width || v.y >= E.height || v.p == 0) continue;
    if (v.t_ns < E.t0_ns || v.t_ns > E.t1_ns) continue;
    const int64_t D = E.t1_ns - E.t0_ns;
    const int64_t N = static_cast<int64_t>(bins - 1) * (v.t_ns - E.t0_ns);
    const int64_t b = N / D, r = N % D;
    const uint32_t w_next = static_cast<uint32_t>((static_cast<uint64_t>(r) << 16) / static_cast<uint64_t>(D));
    const uint32_t w_b = 65536u - w_next;
    const int pol = v.p > 0 ? 0 : 1;
    const size_t plane = static_cast<size_t>(E.width) * E.height;
    const size_t px = static_cast<size_t>(v.y) * E.width + v.x;
    acc[off[v.env] + (static_cast<size_t>(pol) * bins + b) * plane + px] += w_b;
    if (w_next > 0 && b + 1 < bins) acc[off[v.env] + (static_cast<size_t>(pol) * bins + b + 1) * plane + px] += w_next;
  }
  for (int e = 0; e < n_envs; ++e) {
    const size_t plane = static_cast<size_t>(envs[e].width) * envs[e].height;
    for (int q = 0; q < 2 * bins; ++q) {
      const uint32_t* a = acc + off[e] + q * plane;
      float* o = out + off[e] + q * plane;
      uint32_t mx = 0;
      for (size_t i = 0; i < plane; ++i) mx = std::max(mx, a[i]);
      for (size_t i = 0; i < plane; ++i)
        o[i] = mx ? static_cast<float>(a[i]) / static_cast<float>(mx) : 0.0f;
    }
  }
}

// The generator alone, for its tests: n outputs of Philox4x32-10 at counters
// (base + j, c1, c2, c3), written as 4 x n words.
void orc_philox(uint32_t base, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                int64_t n, uint32_t* out) {
  for (int64_t j = 0; j < n; ++j) {
    uint32_t r[4] = {base + static_cast<uint32_t>(j), c1, c2, c3};
    philox4x32_10(r, k0, k1);
    std::memcpy(out + 4 * j, r, 16);
  }
}

int64_t orc_num_events(void* h) { return static_cast<int64_t>(static_cast<Ctx*>(h)->events.size()); }

// Moves up to cap events (16 bytes each) into dst in emission order; returns the count.
int64_t orc_take_events(void* h, void* dst, int64_t cap) {
  Ctx& c = *static_cast<Ctx*>(h);
  int64_t n = static_cast<int64_t>(c.events.size());
  if (n > cap) n = cap;
  std::memcpy(dst, c.events.data(), static_cast<size_t>(n) * sizeof(Event));
  c.events.erase(c.events.begin(), c.events.begin() + n);
  return n;
}

// Per environment: pixel-sub-frames (per channel) since creation whose crossing count
// exceeded the emission limit.
void orc_over_limit(void* h, uint64_t* out) {
  Ctx& c = *static_cast<Ctx*>(h);
  std::memcpy(out, c.over_limit.data(), c.over_limit.size() * 8);
}

// Copies the per-pixel state out (any pointer may be null).
int32_t orc_get_state(void* h, float* Lref, int64_t* t_last, int64_t* clocks) {
  Ctx& c = *static_cast<Ctx*>(h);
  if (Lref) std::memcpy(Lref, c.Lref.data(), c.Lref.size() * 4);
  if (t_last) std::memcpy(t_last, c.t_last.data(), c.t_last.size() * 8);
  if (clocks) std::memcpy(clocks, c.clock.data(), c.clock.size() * 8);
  return 0;
}

// a1 alone: log-intensity of n linear (mode 1) or RGB (mode 2) samples.
void orc_log_intensity(const float* in, int64_t n, int32_t mode, float eps, float* out) {
  for (int64_t i = 0; i < n; ++i)
    out[i] = mode == 2 ? log_intensity(rec709(in[3 * i], in[3 * i + 1], in[3 * i + 2]), eps)
                       : log_intensity(in[i], eps);
}

}  // extern "C"

// ==========================================================================================
// Differentiable soft event-count surrogate (no counterpart in the paper, which has no
// backward pass).  Definition, per environment, per sub-frame i and warp direction X:
//  * discrete decisions, frozen and taken in binary32 exactly as in the event path: the
//    z-buffer winners (Eqs. 5-7), hole flags, and the reference-level trajectory L_ref^(i)
//    of the event model (Eq. 4) with the environment's thresholds c_on, c_off (the smooth
//    threshold C below enters only the sigmoids);
//  * the winner surface W_X(t): footprint sources p of target t whose interpolated depth is
//    within a relative delta of the winning depth, Z~(p) <= Z* (1 + delta) (binary32 test);
//  * soft value S_X(t) = sum_W w(p,t) L_X(p) / sum_W w(p,t), w the bilinear weight of q(p)
//    (smooth in the motion vectors through q = p - f m_A or p + (1-f) m_B);
//  * L_i(t) = (1-f) S_A + f S_B where both directions have a sample, else the present one;
//  * N_on(t) = sum_i sig((L_i - L_ref^(i-1) - C) / tau), N_off(t) = sum_i sig((L_ref^(i-1)
//    - L_i - C) / tau), over the sub-frames where t has a sample.
// The smooth part is evaluated in binary64; the gradient is hand-derived (and checked by
// central differences in the tests).
// ==========================================================================================
namespace {

struct SoftIn {
  const float *LA, *LB, *mvA, *mvB, *ZA, *ZB, *Lref0;  // decisions (binary32)
  const double *dLA, *dLB, *dmvA, *dmvB;               // smooth part (binary64)
};

inline double sigm(double u) { return 1.0 / (1.0 + std::exp(-u)); }

// One environment, one keyframe gap.  counts: [2][H][W]; grads (optional): dL*, dmv* packed
// like the inputs, dC scalar.
void soft_env(int W, int H, int K, float Con, float Coff, double Cd, double tau, float delta,
              const SoftIn &in, double *counts, const double *gcounts, double *gLA, double *gLB,
              double *gmvA, double *gmvB, double *gC) {
  const size_t HW = static_cast<size_t>(W) * H;
  std::vector<float> Lref(in.Lref0, in.Lref0 + HW);
  std::vector<uint64_t> zb[2] = {std::vector<uint64_t>(HW), std::vector<uint64_t>(HW)};
  std::vector<double> SW[2], SWL[2], GX[2], SH[2];
  for (int d = 0; d < 2; ++d) {
    SW[d].resize(HW);
    SWL[d].resize(HW);
    GX[d].resize(HW);
    SH[d].resize(HW);
  }
  std::fill(counts, counts + 2 * HW, 0.0);
  for (int i = 1; i <= K; ++i) {
    const float f = static_cast<float>(i) / static_cast<float>(K), g = 1.0f - f;
    const double fd = static_cast<double>(i) / K, gd = 1.0 - fd;
    std::fill(zb[0].begin(), zb[0].end(), EMPTY);
    std::fill(zb[1].begin(), zb[1].end(), EMPTY);
    splat_A(zb[0].data(), W, H, in.mvA, in.ZA, in.ZB, f, g, false);
    splat_B(zb[1].data(), W, H, in.mvB, in.ZA, in.ZB, f, g, false);
    // visits every (source, footprint cell) pair of the winner surfaces
    auto for_members = [&](int dir, auto &&visit) {
      const float *mv = dir ? in.mvB : in.mvA;
      const float *Zs = dir ? in.ZB : in.ZA;
      const float *Zo = dir ? in.ZA : in.ZB;
      const double *mvd = dir ? in.dmvB : in.dmvA;
      for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
          const size_t p = static_cast<size_t>(y) * W + x;
          const float zs = Zs[p];
          if (!valid_depth(zs)) continue;
          const float mx = mv[2 * p], my = mv[2 * p + 1];
          float qx, qy, zt;
          if (dir == 0) {
            qx = static_cast<float>(x) - f * mx;
            qy = static_cast<float>(y) - f * my;
            zt = g * zs + f * other_depth(Zo, W, H, static_cast<float>(x) - mx, static_cast<float>(y) - my, zs);
          } else {
            qx = static_cast<float>(x) + g * mx;
            qy = static_cast<float>(y) + g * my;
            zt = g * other_depth(Zo, W, H, static_cast<float>(x) + mx, static_cast<float>(y) + my, zs) + f * zs;
          }
          if (!(qx > -1.0f && qx < static_cast<float>(W) && qy > -1.0f && qy < static_cast<float>(H))) continue;
          const float fx0 = std::floor(qx), fy0 = std::floor(qy);
          const float ax = qx - fx0, ay = qy - fy0;
          const float wx[2] = {1.0f - ax, ax}, wy[2] = {1.0f - ay, ay};
          const double s = dir ? gd : -fd;  // q = p + s m
          const double qxd = x + s * mvd[2 * p], qyd = y + s * mvd[2 * p + 1];
          for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
              const int cx = static_cast<int>(fx0) + dx, cy = static_cast<int>(fy0) + dy;
              if (!(wx[dx] * wy[dy] > 0.0f) || cx < 0 || cx >= W || cy < 0 || cy >= H) continue;
              const size_t t = static_cast<size_t>(cy) * W + cx;
              uint32_t zbits = static_cast<uint32_t>(zb[dir][t] >> 32);
              float zstar;
              std::memcpy(&zstar, &zbits, 4);
              if (!(zt <= zstar * (1.0f + delta))) continue;
              // the footprint side of each cell is a frozen decision: the weight is the
              // bilinear factor on that side (1 - e for the left/top cell, 1 + e for the
              // right/bottom one), linear in the binary64 target
              const double ex = qxd - cx, ey = qyd - cy;
              const double wxd = dx ? 1.0 + ex : 1.0 - ex, wyd = dy ? 1.0 + ey : 1.0 - ey;
              const double sx = dx ? 1.0 : -1.0, sy = dy ? 1.0 : -1.0;
              visit(p, t, wxd * wyd, sx * wyd * s, sy * wxd * s);
            }
        }
    };
    for (int d = 0; d < 2; ++d) {
      std::fill(SW[d].begin(), SW[d].end(), 0.0);
      std::fill(SWL[d].begin(), SWL[d].end(), 0.0);
      const double *Ld = d ? in.dLB : in.dLA;
      for_members(d, [&](size_t p, size_t t, double w, double, double) {
        SW[d][t] += w;
        SWL[d][t] += w * Ld[p];
      });
    }
    for (size_t t = 0; t < HW; ++t) {
      const bool hA = zb[0][t] != EMPTY, hB = zb[1][t] != EMPTY;
      GX[0][t] = GX[1][t] = 0.0;
      if (!hA && !hB) continue;
      const double SA = hA ? SWL[0][t] / SW[0][t] : 0.0, SB = hB ? SWL[1][t] / SW[1][t] : 0.0;
      SH[0][t] = SA;
      SH[1][t] = SB;
      const double Ls = (hA && hB) ? gd * SA + fd * SB : (hA ? SA : SB);
      const double lr = Lref[t];
      const double uon = (Ls - lr - Cd) / tau, uoff = (lr - Ls - Cd) / tau;
      const double son = sigm(uon), soff = sigm(uoff);
      counts[t] += son;
      counts[HW + t] += soff;
      if (gcounts) {
        const double don = son * (1.0 - son) / tau, doff = soff * (1.0 - soff) / tau;
        const double G = gcounts[t] * don - gcounts[HW + t] * doff;
        *gC += -(gcounts[t] * don + gcounts[HW + t] * doff);
        if (hA) GX[0][t] = G * (hB ? gd : 1.0) / SW[0][t];
        if (hB) GX[1][t] = G * (hA ? fd : 1.0) / SW[1][t];
      }
      // frozen discrete trajectory of the reference level (binary32, Eq. 4)
      const float la = hA ? in.LA[zb[0][t] & 0xFFFFFFu] : 0.0f, lb = hB ? in.LB[zb[1][t] & 0xFFFFFFu] : 0.0f;
      const float L = (hA && hB) ? g * la + f * lb : (hA ? la : lb);
      const float dd = L - Lref[t];
      const int pol = dd > 0.0f ? 1 : -1;
      const float th = pol > 0 ? Con : Coff;
      const float q = std::fabs(dd) / th;
      // n of Eq. 4 without bound: the trajectory emits nothing, so no emission limit applies
      const float nf = q >= 1.0f ? std::floor(q) : 0.0f;
      if (nf > 0.0f) Lref[t] = Lref[t] + (pol > 0 ? nf : -nf) * th;
    }
    if (gcounts) {
      for (int d = 0; d < 2; ++d) {
        const double *Ld = d ? in.dLB : in.dLA;
        double *gL = d ? gLB : gLA;
        double *gm = d ? gmvB : gmvA;
        for_members(d, [&](size_t p, size_t t, double w, double dwdmx, double dwdmy) {
          gL[p] += GX[d][t] * w;
          gm[2 * p] += GX[d][t] * (Ld[p] - SH[d][t]) * dwdmx;
          gm[2 * p + 1] += GX[d][t] * (Ld[p] - SH[d][t]) * dwdmy;
        });
      }
    }
  }
}

}  // namespace

extern "C" {

// Soft event counts of one keyframe gap for every environment (packed layout; counts are
// [2][H][W] per environment at 2 * pix_off).  Decision inputs are binary32, the smooth
// inputs binary64 (the same values, or perturbed ones for finite differences).  With
// gcounts non-null, also accumulates the gradients (arrays zeroed by the caller).
int32_t orc_soft(const orc_env *envs, int32_t n_envs, double tau, float delta,
                 const float *LA, const float *LB, const float *mvA, const float *mvB,
                 const float *ZA, const float *ZB, const float *Lref0,
                 const double *dLA, const double *dLB, const double *dmvA, const double *dmvB,
                 const double *Cd, double *counts, const double *gcounts, double *gLA,
                 double *gLB, double *gmvA, double *gmvB, double *gC) {
  for (int e = 0; e < n_envs; ++e)
    if (envs[e].margin != 0) return 1;  // the surrogate covers the whole rendered frame
  size_t off = 0;
  for (int e = 0; e < n_envs; ++e) {
    const int W = envs[e].width, H = envs[e].height;
    SoftIn in{LA + off, LB + off, mvA + 2 * off, mvB + 2 * off, ZA + off, ZB + off, Lref0 + off,
              dLA + off, dLB + off, dmvA + 2 * off, dmvB + 2 * off};
    soft_env(W, H, envs[e].K, envs[e].c_on, envs[e].c_off, Cd[e], tau, delta, in, counts + 2 * off,
             gcounts ? gcounts + 2 * off : nullptr, gLA ? gLA + off : nullptr,
             gLB ? gLB + off : nullptr, gmvA ? gmvA + 2 * off : nullptr,
             gmvB ? gmvB + 2 * off : nullptr, gC ? gC + e : nullptr);
    off += (static_cast<size_t>(W) * H + 3) / 4 * 4;
  }
  return 0;
}

}  // extern "C"
