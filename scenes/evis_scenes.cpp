// Seeded synthetic layered scenes: the input generator shared by the CUDA path's tests and
// benchmark and by the oracle's tests.
//
// This module stands in for the physics engine and ray-traced renderer of the paper
// (Sec. 3.1, Eqs. 1-2): for keyframe k it renders, per environment, the scene's
// log-radiance, linear radiance, optional RGB radiance, the backward motion-vector map and
// the depth map (Sec. 3.3: each pixel of a keyframe stores the displacement to its position
// in the previous keyframe).  It holds none of the event-synthesis arithmetic (no warping,
// splatting, blending or threshold logic); it only defines what the scene looks like.
//
// Scene model: an environment is a stack of rigid 2D layers.  Layer 0 is usually a
// full-frame plane, the others textured disks.  Layer l has a depth d_l(k) = d0 + dd*k, a
// centre c_l(k) = c0 + v*k and an angle a_l(k) = a0 + w*k.  A pixel p shows the nearest layer
// that covers it (disk: |p - c| < r).  Its layer-local coordinate is u = R(-a)(p - c), its
// texture value is evaluated at u, and its motion vector is the analytic position of the
// same layer point in keyframe k-1 minus p.  Textures are value noise (Gaussian lattice,
// smoothstep bilinear, two octaves) mapped to log10 radiance and clipped.
//
// Build: g++ -O2 -std=c++17 -shared -fPIC -pthread evis_scenes.cpp -o libevis_scenes.so
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <thread>
#include <vector>

namespace {

// One layer, stored by the caller as SCENE_LAYER_DOUBLES consecutive doubles in this order.
enum LayerField {
  F_KIND = 0,      // 0 = full-frame plane, 1 = disk
  F_RADIUS,        // disk radius in pixels
  F_DEPTH0,        // depth at keyframe 0 (scene units, > 0)
  F_DEPTH_RATE,    // depth change per keyframe
  F_CX0, F_CY0,    // centre at keyframe 0 (pixels)
  F_VX, F_VY,      // centre velocity (pixels per keyframe)
  F_ANGLE0,        // angle at keyframe 0 (radians)
  F_OMEGA,         // angular velocity (radians per keyframe)
  F_TEX_KIND,      // 0 = value noise, 1 = constant (mu only), 2 = horizontal ramp in log10
  F_SEED,          // texture seed (integer < 2^53)
  F_CELL,          // lattice spacing of the first octave (pixels)
  F_MU, F_SIGMA,   // log10 radiance = clip(mu + sigma * z + bright_rate * k, lo, hi)
  F_LO, F_HI,
  F_BRIGHT_RATE,   // log10 radiance added per keyframe (temporal brightness ramp)
  F_TINT_R, F_TINT_G, F_TINT_B,  // RGB radiance = tint * linear radiance
  SCENE_LAYER_DOUBLES
};

inline uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// Standard normal lattice value at integer lattice point (i, j) (Box-Muller on a hash).
inline double lattice(uint64_t seed, int64_t i, int64_t j) {
  uint64_t h = splitmix64(seed ^ splitmix64(static_cast<uint64_t>(i) * 0xD1B54A32D192ED03ull ^
                                            static_cast<uint64_t>(j)));
  double u1 = (static_cast<double>(h >> 11) + 1.0) * (1.0 / 9007199254740992.0);  // (0, 1]
  uint64_t h2 = splitmix64(h);
  double u2 = static_cast<double>(h2 >> 11) * (1.0 / 9007199254740992.0);          // [0, 1)
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

inline double smooth(double t) { return t * t * (3.0 - 2.0 * t); }

// Lattice values of one octave of one layer over a rectangle of lattice points, filled once
// per render job: a table entry is the very double lattice() returns, so the output does not
// depend on the table (points outside it are computed directly).
struct LatticeTable {
  uint64_t seed = 0;
  int64_t i0 = 0, j0 = 0;
  int64_t ni = 0, nj = 0;
  std::vector<double> v;
  void fill(uint64_t s, int64_t ilo, int64_t ihi, int64_t jlo, int64_t jhi) {
    seed = s;
    i0 = ilo;
    j0 = jlo;
    ni = std::max<int64_t>(0, ihi - ilo + 1);
    nj = std::max<int64_t>(0, jhi - jlo + 1);
    if (ni * nj > (int64_t(1) << 22)) ni = nj = 0;  // too large: compute every point
    v.resize(static_cast<size_t>(ni * nj));
    for (int64_t j = 0; j < nj; ++j)
      for (int64_t i = 0; i < ni; ++i) v[static_cast<size_t>(j * ni + i)] = lattice(s, i0 + i, j0 + j);
  }
  double get(int64_t i, int64_t j) const {
    const int64_t a = i - i0, b = j - j0;
    if (a >= 0 && a < ni && b >= 0 && b < nj) return v[static_cast<size_t>(b * ni + a)];
    return lattice(seed, i, j);
  }
};

inline double value_noise(const LatticeTable& m, double x, double y) {
  double fx = std::floor(x), fy = std::floor(y);
  int64_t i = static_cast<int64_t>(fx), j = static_cast<int64_t>(fy);
  double sx = smooth(x - fx), sy = smooth(y - fy);
  double a = m.get(i, j), b = m.get(i + 1, j);
  double c = m.get(i, j + 1), d = m.get(i + 1, j + 1);
  double top = a + (b - a) * sx, bot = c + (d - c) * sx;
  return top + (bot - top) * sy;
}

struct LayerAt {  // a layer evaluated at one keyframe
  const double* p;
  double depth, cx, cy, ca, sa;         // at keyframe k
  double pcx, pcy, pca, psa;            // at keyframe k-1
  LatticeTable oct[2];                  // value-noise lattice of both octaves over this job
};

// Lattice points that texture coordinates (u / cell) * scale of the job's pixels can reach:
// the layer-local images of the rectangle's corners, widened by two points on each side.
void lattice_range(const LayerAt& a, double scale, int W, int row0, int row1, int64_t* ilo,
                   int64_t* ihi, int64_t* jlo, int64_t* jhi) {
  double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
  const double xs[2] = {0.0, static_cast<double>(W - 1)};
  const double ys[2] = {static_cast<double>(row0), static_cast<double>(row1 - 1)};
  for (double x : xs)
    for (double y : ys) {
      const double dx = x - a.cx, dy = y - a.cy;
      const double ux = (a.ca * dx + a.sa * dy) * scale, uy = (-a.sa * dx + a.ca * dy) * scale;
      xmin = std::min(xmin, ux);
      xmax = std::max(xmax, ux);
      ymin = std::min(ymin, uy);
      ymax = std::max(ymax, uy);
    }
  *ilo = static_cast<int64_t>(std::floor(xmin)) - 2;
  *ihi = static_cast<int64_t>(std::floor(xmax)) + 2;
  *jlo = static_cast<int64_t>(std::floor(ymin)) - 2;
  *jhi = static_cast<int64_t>(std::floor(ymax)) + 2;
}

void render_env(int W, int H, int n_layers, const double* layers, int32_t k, int row0, int row1,
                float* L, float* I, float* rgb, float* mv, float* Z) {
  std::vector<LayerAt> ls(n_layers);
  for (int l = 0; l < n_layers; ++l) {
    const double* p = layers + static_cast<size_t>(l) * SCENE_LAYER_DOUBLES;
    LayerAt& a = ls[l];
    a.p = p;
    a.depth = p[F_DEPTH0] + p[F_DEPTH_RATE] * k;
    a.cx = p[F_CX0] + p[F_VX] * k;
    a.cy = p[F_CY0] + p[F_VY] * k;
    double ang = p[F_ANGLE0] + p[F_OMEGA] * k;
    a.ca = std::cos(ang);
    a.sa = std::sin(ang);
    a.pcx = p[F_CX0] + p[F_VX] * (k - 1);
    a.pcy = p[F_CY0] + p[F_VY] * (k - 1);
    double pang = p[F_ANGLE0] + p[F_OMEGA] * (k - 1);
    a.pca = std::cos(pang);
    a.psa = std::sin(pang);
    if (p[F_TEX_KIND] == 0.0) {
      const uint64_t seed = static_cast<uint64_t>(p[F_SEED]);
      for (int o = 0; o < 2; ++o) {
        int64_t ilo, ihi, jlo, jhi;
        lattice_range(a, (o ? 2.0 : 1.0) / p[F_CELL], W, row0, row1, &ilo, &ihi, &jlo, &jhi);
        a.oct[o].fill(o ? splitmix64(seed ^ 0xA5A5A5A5ull) : splitmix64(seed), ilo, ihi, jlo, jhi);
      }
    }
  }
  // nearest layer first; equal depths keep layer order
  std::vector<int> order(n_layers);
  for (int l = 0; l < n_layers; ++l) order[l] = l;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return ls[x].depth < ls[y].depth; });
  const double ln10 = 2.302585092994046;
  for (int y = row0; y < row1; ++y) {
    for (int x = 0; x < W; ++x) {
      const LayerAt* hit = nullptr;
      for (int oi = 0; oi < n_layers; ++oi) {
        const LayerAt& a = ls[order[oi]];
        if (a.p[F_KIND] == 1.0) {
          double dx = x - a.cx, dy = y - a.cy, r = a.p[F_RADIUS];
          if (dx * dx + dy * dy >= r * r) continue;
        }
        hit = &a;
        break;
      }
      size_t px = static_cast<size_t>(y) * W + x;
      if (!hit) {  // no layer covers the pixel: black at infinite depth, no motion
        if (L) L[px] = static_cast<float>(-2.0 * ln10);
        if (I) I[px] = 0.01f;
        if (rgb) rgb[3 * px] = rgb[3 * px + 1] = rgb[3 * px + 2] = 0.01f;
        if (mv) mv[2 * px] = mv[2 * px + 1] = 0.0f;
        if (Z) Z[px] = INFINITY;
        continue;
      }
      const double* p = hit->p;
      double dx = x - hit->cx, dy = y - hit->cy;
      double ux = hit->ca * dx + hit->sa * dy;   // u = R(-a) (p - c)
      double uy = -hit->sa * dx + hit->ca * dy;
      double z;
      if (p[F_TEX_KIND] == 0.0) {
        double cell = p[F_CELL];
        double n1 = value_noise(hit->oct[0], ux / cell, uy / cell);
        double n2 = value_noise(hit->oct[1], 2.0 * ux / cell, 2.0 * uy / cell);
        z = (n1 + 0.5 * n2) * 1.35;  // ~unit variance for smoothstep value noise
      } else if (p[F_TEX_KIND] == 2.0) {
        z = ux;
      } else {
        z = 0.0;
      }
      double l10 = p[F_MU] + p[F_SIGMA] * z + p[F_BRIGHT_RATE] * k;
      l10 = std::min(std::max(l10, p[F_LO]), p[F_HI]);
      const double inten = (I || rgb) ? std::pow(10.0, l10) : 0.0;
      if (L) L[px] = static_cast<float>(ln10 * l10);
      if (I) I[px] = static_cast<float>(inten);
      if (rgb) {
        rgb[3 * px] = static_cast<float>(inten * p[F_TINT_R]);
        rgb[3 * px + 1] = static_cast<float>(inten * p[F_TINT_G]);
        rgb[3 * px + 2] = static_cast<float>(inten * p[F_TINT_B]);
      }
      if (mv) {
        // position of the same layer point at keyframe k-1: c' + R(a') u
        double qx = hit->pcx + hit->pca * ux - hit->psa * uy;
        double qy = hit->pcy + hit->psa * ux + hit->pca * uy;
        mv[2 * px] = static_cast<float>(qx - x);
        mv[2 * px + 1] = static_cast<float>(qy - y);
      }
      if (Z) Z[px] = static_cast<float>(hit->depth);
    }
  }
}

}  // namespace

extern "C" {

int scenes_layer_doubles() { return SCENE_LAYER_DOUBLES; }

// Render keyframe k of n_envs environments into packed arrays.  Environment e occupies
// pixels [pix_off[e], pix_off[e] + W[e]*H[e]) of L, I, Z, and 2x / 3x that of mv / rgb.
// Its layers are layers[layer_off[e] .. layer_off[e] + n_layers[e]) (each
// SCENE_LAYER_DOUBLES doubles).  Any output pointer may be null.  Returns 0, or -1 on bad
// sizes.
int scenes_render(int32_t n_envs, const int32_t* W, const int32_t* H, const int64_t* pix_off,
                  const int32_t* layer_off, const int32_t* n_layers, const double* layers,
                  int32_t k, float* L, float* I, float* rgb, float* mv, float* Z,
                  int32_t n_threads) {
  if (n_envs < 0) return -1;
  struct Job { int e, r0, r1; };
  std::vector<Job> jobs;
  for (int e = 0; e < n_envs; ++e) {
    if (W[e] <= 0 || H[e] <= 0 || n_layers[e] < 0) return -1;
    const int rows = n_envs >= 4 * std::max(1, n_threads) ? 64 : 16;  // fewer lattice fills
    for (int r = 0; r < H[e]; r += rows) jobs.push_back({e, r, std::min(H[e], r + rows)});
  }
  auto run = [&](size_t j) {
    const Job& jb = jobs[j];
    int e = jb.e;
    size_t o = static_cast<size_t>(pix_off[e]);
    render_env(W[e], H[e], n_layers[e], layers + static_cast<size_t>(layer_off[e]) * SCENE_LAYER_DOUBLES,
               k, jb.r0, jb.r1, L ? L + o : nullptr, I ? I + o : nullptr,
               rgb ? rgb + 3 * o : nullptr, mv ? mv + 2 * o : nullptr, Z ? Z + o : nullptr);
  };
  int nt = std::max(1, n_threads);
  if (nt == 1 || jobs.size() < 2) {
    for (size_t j = 0; j < jobs.size(); ++j) run(j);
    return 0;
  }
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t]() {
      for (size_t j = t; j < jobs.size(); j += nt) run(j);
    });
  for (auto& x : th) x.join();
  return 0;
}

}  // extern "C"
