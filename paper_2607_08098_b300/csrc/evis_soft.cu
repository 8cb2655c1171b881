// Differentiable soft event-count surrogate of one keyframe gap (forward and hand-written
// backward).  The paper has no backward pass; the surrogate keeps the event path's discrete
// decisions frozen and makes the rest smooth:
//   * z-buffer winners (Eqs. 5-7), hole flags and the reference trajectory L_ref^(i) of the
//     event model (Eq. 4 with the environment's c_on / c_off) are taken exactly as in the
//     event path; the differentiable threshold C enters only the sigmoids;
//   * per direction X, sub-frame i and target t, the winner surface W_X(t) holds the
//     footprint sources whose interpolated depth is <= Z*(t) (1 + delta);
//   * S_X(t) = sum_W w L_X / sum_W w with w the bilinear weight of the source's target q;
//   * L_i = (1-f) S_A + f S_B (one present: that one);
//   * N_on(t) = sum_i sig((L_i - L_ref^(i-1) - C)/tau), N_off(t) = sum_i sig((L_ref^(i-1) - L_i - C)/tau).
// Gradients flow to L_A, L_B, m_A, m_B (through q) and C.  The forward splats with global
// atomics (atomicMin for the winners, fixed-point atomicAdd for the sums); the backward is in
// gather form: every source revisits its footprint cells and owns its gradient (no atomics).
#include <cstring>
#include <vector>

#include "evis_device.cuh"
#include "evis_internal.h"

namespace {

using evis::other_depth;
using evis::valid_depth;

constexpr unsigned long long kEmpty = ~0ull;

struct SoftEnv {
  int32_t W, H, K;
  float c_on, c_off;  // thresholds of the frozen discrete trajectory (the event model's)
  int32_t pad;
  int64_t pix_off;  // packed pixel offset
  int64_t uo;       // first pixel-substep (i = 1) of this environment
};

// Workspace layout (byte offsets, each 256-aligned).
struct Layout {
  size_t env, keys, sw, swl, gx, lsoft, lrefp, flags, total;
  int64_t U;        // total pixel-substeps
};

size_t al(size_t x) { return (x + 255) / 256 * 256; }

Layout layout_for(const evis_env_desc *envs, int n, std::vector<SoftEnv> *tab) {
  Layout L{};
  int64_t px = 0, u = 0;
  if (tab) tab->resize(n);
  for (int e = 0; e < n; ++e) {
    const int64_t hw = int64_t(envs[e].width) * envs[e].height;
    if (tab)
      (*tab)[e] = SoftEnv{envs[e].width, envs[e].height, envs[e].K, envs[e].c_on, envs[e].c_off, 0,
                          px, u};
    px += (hw + 3) / 4 * 4;
    u += hw * envs[e].K;
  }
  L.U = u;
  size_t o = 0;
  L.env = o;   o = al(o + sizeof(SoftEnv) * n);
  L.keys = o;  o = al(o + 8 * 2 * size_t(u));
  L.sw = o;    o = al(o + 8 * 2 * size_t(u));
  L.swl = o;   o = al(o + 8 * 2 * size_t(u));
  L.gx = o;    o = al(o + 4 * 2 * size_t(u));
  L.lsoft = o; o = al(o + 4 * size_t(u));
  L.lrefp = o; o = al(o + 4 * size_t(u));
  L.flags = o; o = al(o + size_t(u));
  L.total = o;
  return L;
}

struct SoftArgs {
  const SoftEnv *envs;
  const float *LA, *LB;
  const float2 *mvA, *mvB;
  const float *ZA, *ZB, *Lref0, *C;
  float tau, delta;
  int64_t U;
  unsigned long long *keys;   // [2][U]
  long long *sw, *swl;        // [2][U]: surface sums of w and w L, fixed point (2^-40 units)
  float *gx;                  // [2][U]
  float *lsoft, *lrefp;       // [U]
  unsigned char *flags;       // [U]: bit 0 A present, bit 1 B present
  float *counts;              // packed [2][H][W] per environment
  const float *gcounts;
  float *dLA, *dLB;
  float2 *dmvA, *dmvB;
  float *dC;
};

// Geometry of source (x, y) of direction dir at sub-frame fraction f (binary32, the event
// path's operations): target q, interpolated depth, footprint origin and fractions.
struct Geo {
  bool ok;
  float zt, ax, ay, s;  // s: dq/dm (-f for A, 1-f for B)
  int cx, cy;
};

__device__ __forceinline__ Geo geometry(int dir, int x, int y, int W, int H, float f, float g,
                                        const float2 *mvA, const float *ZA, const float2 *mvB,
                                        const float *ZB) {
  Geo r{};
  const int p = y * W + x;
  const float zs = dir ? ZB[p] : ZA[p];
  if (!valid_depth(zs)) return r;
  const float2 m = dir ? mvB[p] : mvA[p];
  const float fx = static_cast<float>(x), fy = static_cast<float>(y);
  float qx, qy, zo;
  if (dir == 0) {
    qx = __fsub_rn(fx, __fmul_rn(f, m.x));
    qy = __fsub_rn(fy, __fmul_rn(f, m.y));
  } else {
    qx = __fadd_rn(fx, __fmul_rn(g, m.x));
    qy = __fadd_rn(fy, __fmul_rn(g, m.y));
  }
  if (!(qx > -1.0f && qx < static_cast<float>(W) && qy > -1.0f && qy < static_cast<float>(H)))
    return r;
  if (dir == 0) {
    zo = other_depth(ZB, W, H, __fsub_rn(fx, m.x), __fsub_rn(fy, m.y), zs);
    r.zt = __fadd_rn(__fmul_rn(g, zs), __fmul_rn(f, zo));
  } else {
    zo = other_depth(ZA, W, H, __fadd_rn(fx, m.x), __fadd_rn(fy, m.y), zs);
    r.zt = __fadd_rn(__fmul_rn(g, zo), __fmul_rn(f, zs));
  }
  const float fx0 = floorf(qx), fy0 = floorf(qy);
  r.cx = static_cast<int>(fx0);
  r.cy = static_cast<int>(fy0);
  r.ax = __fsub_rn(qx, fx0);
  r.ay = __fsub_rn(qy, fy0);
  r.s = dir == 0 ? -f : g;
  r.ok = true;
  return r;
}

// Weight of footprint cell (dx, dy) (0 when excluded) and its slopes d w / d m.
__device__ __forceinline__ float cell_weight(const Geo &q, int dx, int dy, int W, int H,
                                             float *dwx, float *dwy) {
  const int cx = q.cx + dx, cy = q.cy + dy;
  const float wx = dx ? q.ax : __fsub_rn(1.0f, q.ax);
  const float wy = dy ? q.ay : __fsub_rn(1.0f, q.ay);
  const float w = __fmul_rn(wx, wy);
  if (!(w > 0.0f) || cx < 0 || cx >= W || cy < 0 || cy >= H) return 0.0f;
  *dwx = (dx ? 1.0f : -1.0f) * wy * q.s;
  *dwy = (dy ? 1.0f : -1.0f) * wx * q.s;
  return w;
}

__device__ __forceinline__ unsigned long long key_of(const Geo &q, float w, int p) {
  const unsigned wq = min(__float2uint_rz(__fmul_rn(__fsub_rn(1.0f, w), 256.0f)), 255u);
  return (static_cast<unsigned long long>(__float_as_uint(q.zt)) << 32) |
         (static_cast<unsigned long long>(wq) << 24) | static_cast<unsigned>(p);
}

// Membership of the winner surface: Z~ <= Z* (1 + delta), binary32.
__device__ __forceinline__ bool on_surface(float zt, unsigned long long key, float delta) {
  const float zstar = __uint_as_float(static_cast<unsigned>(key >> 32));
  return zt <= __fmul_rn(zstar, __fadd_rn(1.0f, delta));
}

// Thread -> (environment, pixel): blockIdx.y is the environment.
#define SOFT_TARGET_PROLOGUE                                                    \
  const SoftEnv E = a.envs[blockIdx.y];                                         \
  const int HW = E.W * E.H;                                                     \
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;                        \
  const int64_t o = E.pix_off;
#define SOFT_PIXEL_PROLOGUE                                                     \
  SOFT_TARGET_PROLOGUE                                                          \
  const float *ZA = a.ZA + o, *ZB = a.ZB + o;                                   \
  const float2 *mvA = a.mvA + o, *mvB = a.mvB + o;

// Pass 1: the z-buffer winners of every sub-frame and direction.
__global__ void soft_winners(const SoftArgs a) {
  SOFT_PIXEL_PROLOGUE
  if (pix >= HW) return;
  const int x = pix % E.W, y = pix / E.W;
  for (int i = 1; i <= E.K; ++i) {
    const float f = __fdiv_rn(static_cast<float>(i), static_cast<float>(E.K)), g = __fsub_rn(1.0f, f);
    const int64_t ub = E.uo + int64_t(i - 1) * HW;
    for (int dir = 0; dir < 2; ++dir) {
      const Geo q = geometry(dir, x, y, E.W, E.H, f, g, mvA, ZA, mvB, ZB);
      if (!q.ok) continue;
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          float dwx, dwy;
          const float w = cell_weight(q, dx, dy, E.W, E.H, &dwx, &dwy);
          if (w > 0.0f) {
            const int t = (q.cy + dy) * E.W + q.cx + dx;
            atomicMin(&a.keys[dir * a.U + ub + t], key_of(q, w, pix));
          }
        }
    }
  }
}

// Fixed point in units of 2^-40.  This part runs binary64 at a small fraction of the
// binary32 rate, so the conversions are integer or binary32 operations that give the same
// integers as rounding the exact binary64 values half to even.

// w in (0, 1]: w 2^40 is exact in binary32 (a power-of-two scaling), then rounded.
__device__ __forceinline__ long long fixed_of_weight(float w) {
  return __float2ll_rn(__fmul_rn(w, 1099511627776.0f));
}

// w L (w in (0, 1], L finite): the exact 48-bit product of the significands, scaled by
// 2^(e_w + e_L + 40) with the shift rounding half to even; saturates at +-2^62.
__device__ __forceinline__ long long fixed_of_product(float w, float L) {
  const unsigned bw = __float_as_uint(w), bl = __float_as_uint(L);
  const int ew = static_cast<int>(bw >> 23), el = static_cast<int>((bl >> 23) & 0xFFu);
  if ((bl & 0x7FFFFFFFu) == 0u || el == 255) return 0;  // zero (or a non-finite L)
  const unsigned long long mw = (bw & 0x7FFFFFu) | 0x800000u;  // w is normal (>= 2^-48)
  const unsigned long long ml = el ? ((bl & 0x7FFFFFu) | 0x800000u) : (bl & 0x7FFFFFu);
  const unsigned long long prod = mw * ml;                       // < 2^48
  const int sh = ew + (el ? el : 1) - 300 + 40;                 // value = prod 2^sh
  unsigned long long q;
  if (sh >= 0) {
    q = sh >= 14 ? (1ull << 62) : min(prod << sh, 1ull << 62);
  } else if (sh <= -64) {
    q = 0;
  } else {
    const int r = -sh;
    q = (prod + ((1ull << (r - 1)) - 1ull) + ((prod >> r) & 1ull)) >> r;
  }
  const long long v = static_cast<long long>(q);
  return (bl >> 31) ? -v : v;
}

__device__ __forceinline__ float fixed_ratio(long long num, long long den) {
  return __fdiv_rn(__ll2float_rn(num), __ll2float_rn(den));
}
__device__ __forceinline__ float from_fixed(long long v) {
  return __fmul_rn(__ll2float_rn(v), 9.094947017729282e-13f);  // 2^-40
}

// Pass 2: sums of w and w L over each target's winner surface.
__global__ void soft_sums(const SoftArgs a) {
  SOFT_PIXEL_PROLOGUE
  if (pix >= HW) return;
  const int x = pix % E.W, y = pix / E.W;
  const float LAp = a.LA[o + pix], LBp = a.LB[o + pix];
  for (int i = 1; i <= E.K; ++i) {
    const float f = __fdiv_rn(static_cast<float>(i), static_cast<float>(E.K)), g = __fsub_rn(1.0f, f);
    const int64_t ub = E.uo + int64_t(i - 1) * HW;
    for (int dir = 0; dir < 2; ++dir) {
      const Geo q = geometry(dir, x, y, E.W, E.H, f, g, mvA, ZA, mvB, ZB);
      if (!q.ok) continue;
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          float dwx, dwy;
          const float w = cell_weight(q, dx, dy, E.W, E.H, &dwx, &dwy);
          if (!(w > 0.0f)) continue;
          const int64_t u = dir * a.U + ub + (q.cy + dy) * E.W + q.cx + dx;
          if (!on_surface(q.zt, a.keys[u], a.delta)) continue;
          // fixed-point sums: integer addition is exact and order-independent, so the
          // forward pass is deterministic (finite differences can resolve single inputs)
          atomicAdd(reinterpret_cast<unsigned long long *>(&a.sw[u]),
                    static_cast<unsigned long long>(fixed_of_weight(w)));
          atomicAdd(reinterpret_cast<unsigned long long *>(&a.swl[u]),
                    static_cast<unsigned long long>(fixed_of_product(w, dir ? LBp : LAp)));
        }
    }
  }
}

__device__ __forceinline__ float sigm(float u) { return 1.0f / (1.0f + __expf(-u)); }

// Pass 3 (per target): soft values, counts, and the frozen discrete reference trajectory.
__global__ void soft_targets(const SoftArgs a) {
  SOFT_TARGET_PROLOGUE
  if (pix >= HW) return;
  const float C = a.C[blockIdx.y];
  float Lref = a.Lref0[o + pix];
  float non = 0.0f, noff = 0.0f;
  for (int i = 1; i <= E.K; ++i) {
    const float f = __fdiv_rn(static_cast<float>(i), static_cast<float>(E.K)), g = __fsub_rn(1.0f, f);
    const int64_t u = E.uo + int64_t(i - 1) * HW + pix;
    const unsigned long long kA = a.keys[u], kB = a.keys[a.U + u];
    const bool hA = kA != kEmpty, hB = kB != kEmpty;
    a.flags[u] = static_cast<unsigned char>((hA ? 1 : 0) | (hB ? 2 : 0));
    a.lrefp[u] = Lref;
    if (!hA && !hB) continue;
    const float SA = hA ? fixed_ratio(a.swl[u], a.sw[u]) : 0.0f;
    const float SB = hB ? fixed_ratio(a.swl[a.U + u], a.sw[a.U + u]) : 0.0f;
    const float Ls = (hA && hB) ? g * SA + f * SB : (hA ? SA : SB);
    a.lsoft[u] = Ls;
    non += sigm((Ls - Lref - C) / a.tau);
    noff += sigm((Lref - Ls - C) / a.tau);
    // discrete trajectory (binary32, the event path's operations)
    const float la = hA ? a.LA[o + (kA & 0xFFFFFFull)] : 0.0f;
    const float lb = hB ? a.LB[o + (kB & 0xFFFFFFull)] : 0.0f;
    const float L = (hA && hB) ? __fadd_rn(__fmul_rn(g, la), __fmul_rn(f, lb)) : (hA ? la : lb);
    const float d = __fsub_rn(L, Lref);
    const int pol = d > 0.0f ? 1 : -1;
    const float th = pol > 0 ? E.c_on : E.c_off;
    const float qn = __fdiv_rn(fabsf(d), th);
    // n of Eq. 4 without bound: the trajectory emits nothing, so no emission limit applies
    const float nf = qn >= 1.0f ? floorf(qn) : 0.0f;
    if (nf > 0.0f) Lref = __fadd_rn(Lref, __fmul_rn(pol > 0 ? nf : -nf, th));
  }
  a.counts[2 * o + pix] = non;
  a.counts[2 * o + HW + pix] = noff;
}

// Backward pass 1 (per target): dN/dL_i, its share per direction divided by the surface
// weight, and the threshold gradient (block sum, one float atomic per block).
__global__ void soft_targets_bwd(const SoftArgs a) {
  SOFT_TARGET_PROLOGUE
  const float C = a.C[blockIdx.y];
  float dc = 0.0f;
  if (pix < HW) {
    const float gon = a.gcounts[2 * o + pix], goff = a.gcounts[2 * o + HW + pix];
    for (int i = 1; i <= E.K; ++i) {
      const float f = __fdiv_rn(static_cast<float>(i), static_cast<float>(E.K)), g = __fsub_rn(1.0f, f);
      const int64_t u = E.uo + int64_t(i - 1) * HW + pix;
      const unsigned char fl = a.flags[u];
      const bool hA = fl & 1, hB = fl & 2;
      a.gx[u] = 0.0f;
      a.gx[a.U + u] = 0.0f;
      if (!hA && !hB) continue;
      const float Ls = a.lsoft[u], Lref = a.lrefp[u];
      const float son = sigm((Ls - Lref - C) / a.tau), soff = sigm((Lref - Ls - C) / a.tau);
      const float don = son * (1.0f - son) / a.tau, doff = soff * (1.0f - soff) / a.tau;
      const float G = gon * don - goff * doff;
      dc -= gon * don + goff * doff;
      if (hA) a.gx[u] = G * (hB ? g : 1.0f) / from_fixed(a.sw[u]);
      if (hB) a.gx[a.U + u] = G * (hA ? f : 1.0f) / from_fixed(a.sw[a.U + u]);
    }
  }
  for (int d = 16; d > 0; d >>= 1) dc += __shfl_xor_sync(0xFFFFFFFFu, dc, d);
  __shared__ float part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = dc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float sum = 0.0f;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) sum += part[w];
    atomicAdd(&a.dC[blockIdx.y], sum);
  }
}

// Backward pass 2 (per source, gather form): each source of A and B revisits its footprint
// cells on the winner surfaces and collects dL and dm; no atomics.
__global__ void soft_sources_bwd(const SoftArgs a) {
  SOFT_PIXEL_PROLOGUE
  if (pix >= HW) return;
  const int x = pix % E.W, y = pix / E.W;
  const float Lp[2] = {a.LA[o + pix], a.LB[o + pix]};
  float gL[2] = {0.0f, 0.0f}, gmx[2] = {0.0f, 0.0f}, gmy[2] = {0.0f, 0.0f};
  for (int i = 1; i <= E.K; ++i) {
    const float f = __fdiv_rn(static_cast<float>(i), static_cast<float>(E.K)), g = __fsub_rn(1.0f, f);
    const int64_t ub = E.uo + int64_t(i - 1) * HW;
    for (int dir = 0; dir < 2; ++dir) {
      const Geo q = geometry(dir, x, y, E.W, E.H, f, g, mvA, ZA, mvB, ZB);
      if (!q.ok) continue;
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          float dwx = 0.0f, dwy = 0.0f;
          const float w = cell_weight(q, dx, dy, E.W, E.H, &dwx, &dwy);
          if (!(w > 0.0f)) continue;
          const int64_t u = dir * a.U + ub + (q.cy + dy) * E.W + q.cx + dx;
          if (!on_surface(q.zt, a.keys[u], a.delta)) continue;
          const float G = a.gx[u];
          if (G == 0.0f) continue;
          const float S = fixed_ratio(a.swl[u], a.sw[u]);
          gL[dir] += G * w;
          gmx[dir] += G * (Lp[dir] - S) * dwx;
          gmy[dir] += G * (Lp[dir] - S) * dwy;
        }
    }
  }
  a.dLA[o + pix] = gL[0];
  a.dLB[o + pix] = gL[1];
  a.dmvA[o + pix] = make_float2(gmx[0], gmy[0]);
  a.dmvB[o + pix] = make_float2(gmx[1], gmy[1]);
}

evis_status soft_prepare(const evis_env_desc *envs, int32_t n, void *ws, int64_t ws_bytes,
                         cudaStream_t st, SoftArgs *a, bool upload, int *max_hw) {
  if (!envs || n < 1 || n > 65535 || !ws) return EVIS_ERR_INVALID_ARG;
  *max_hw = 0;
  for (int e = 0; e < n; ++e) {
    const evis_env_desc &d = envs[e];
    if (d.width < 1 || d.height < 1 || d.width > 65535 || d.height > 65535 ||
        int64_t(d.width) * d.height > (int64_t(1) << 24) || d.K < 1 || d.K > 4096 ||
        !(d.c_on > 0.0f && d.c_on < INFINITY) || !(d.c_off > 0.0f && d.c_off < INFINITY) ||
        d.margin != 0)  // the surrogate counts over the whole rendered frame
      return EVIS_ERR_INVALID_ARG;
    *max_hw = std::max(*max_hw, d.width * d.height);
  }
  std::vector<SoftEnv> tab;
  const Layout L = layout_for(envs, n, &tab);
  if (ws_bytes < static_cast<int64_t>(L.total)) return EVIS_ERR_INVALID_ARG;
  unsigned char *b = static_cast<unsigned char *>(ws);
  a->envs = reinterpret_cast<const SoftEnv *>(b + L.env);
  a->U = L.U;
  a->keys = reinterpret_cast<unsigned long long *>(b + L.keys);
  a->sw = reinterpret_cast<long long *>(b + L.sw);
  a->swl = reinterpret_cast<long long *>(b + L.swl);
  a->gx = reinterpret_cast<float *>(b + L.gx);
  a->lsoft = reinterpret_cast<float *>(b + L.lsoft);
  a->lrefp = reinterpret_cast<float *>(b + L.lrefp);
  a->flags = b + L.flags;
  if (upload) {
    cudaError_t e = cudaMemcpyAsync(b + L.env, tab.data(), sizeof(SoftEnv) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a->keys, 0xFF, 8 * 2 * size_t(L.U), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a->sw, 0, 8 * 2 * size_t(L.U), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a->swl, 0, 8 * 2 * size_t(L.U), st);
    // (a copy from pageable memory returns once the table is staged, so the local may go)
    if (e != cudaSuccess) return EVIS_ERR_CUDA;
  }
  return EVIS_OK;
}

}  // namespace

extern "C" {

evis_status evis_soft_workspace_size(const evis_env_desc *envs, int32_t n_envs, int64_t *bytes) {
  if (!envs || n_envs < 1 || n_envs > 65535 || !bytes) return EVIS_ERR_INVALID_ARG;
  *bytes = static_cast<int64_t>(layout_for(envs, n_envs, nullptr).total);
  return EVIS_OK;
}

evis_status evis_soft_forward(const evis_env_desc *envs, int32_t n_envs, float tau, float delta,
                              const float *LA, const float *LB, const float *mvA,
                              const float *mvB, const float *ZA, const float *ZB,
                              const float *Lref0, const float *C, float *counts,
                              void *workspace, int64_t workspace_bytes, evis_stream_t stream) {
  if (!(tau > 0.0f) || !(delta >= 0.0f) || !LA || !LB || !mvA || !mvB || !ZA || !ZB || !Lref0 ||
      !C || !counts)
    return EVIS_ERR_INVALID_ARG;
  if (!evis::aligned(mvA, 8) || !evis::aligned(mvB, 8) || !evis::aligned(LA, 4) ||
      !evis::aligned(LB, 4) || !evis::aligned(ZA, 4) || !evis::aligned(ZB, 4) ||
      !evis::aligned(Lref0, 4) || !evis::aligned(C, 4) || !evis::aligned(counts, 4) ||
      !evis::aligned(workspace, 16))
    return EVIS_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  SoftArgs a{};
  int max_hw = 0;
  evis_status s = soft_prepare(envs, n_envs, workspace, workspace_bytes, st, &a, true, &max_hw);
  if (s != EVIS_OK) return s;
  a.LA = LA;
  a.LB = LB;
  a.mvA = reinterpret_cast<const float2 *>(mvA);
  a.mvB = reinterpret_cast<const float2 *>(mvB);
  a.ZA = ZA;
  a.ZB = ZB;
  a.Lref0 = Lref0;
  a.C = C;
  a.tau = tau;
  a.delta = delta;
  a.counts = counts;
  const dim3 grid((max_hw + 255) / 256, n_envs);
  soft_winners<<<grid, 256, 0, st>>>(a);
  soft_sums<<<grid, 256, 0, st>>>(a);
  soft_targets<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? EVIS_OK : EVIS_ERR_CUDA;
}

evis_status evis_soft_backward(const evis_env_desc *envs, int32_t n_envs, float tau, float delta,
                               const float *LA, const float *LB, const float *mvA,
                               const float *mvB, const float *ZA, const float *ZB,
                               const float *C, const float *gcounts, float *dLA, float *dLB,
                               float *dmvA, float *dmvB, float *dC, void *workspace,
                               int64_t workspace_bytes, evis_stream_t stream) {
  if (!(tau > 0.0f) || !(delta >= 0.0f) || !LA || !LB || !mvA || !mvB || !ZA || !ZB || !C ||
      !gcounts || !dLA || !dLB || !dmvA || !dmvB || !dC)
    return EVIS_ERR_INVALID_ARG;
  if (!evis::aligned(mvA, 8) || !evis::aligned(mvB, 8) || !evis::aligned(dmvA, 8) ||
      !evis::aligned(dmvB, 8) || !evis::aligned(LA, 4) || !evis::aligned(LB, 4) ||
      !evis::aligned(ZA, 4) || !evis::aligned(ZB, 4) || !evis::aligned(C, 4) ||
      !evis::aligned(gcounts, 4) || !evis::aligned(dLA, 4) || !evis::aligned(dLB, 4) ||
      !evis::aligned(dC, 4) || !evis::aligned(workspace, 16))
    return EVIS_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  SoftArgs a{};
  int max_hw = 0;
  evis_status s = soft_prepare(envs, n_envs, workspace, workspace_bytes, st, &a, false, &max_hw);
  if (s != EVIS_OK) return s;
  a.LA = LA;
  a.LB = LB;
  a.mvA = reinterpret_cast<const float2 *>(mvA);
  a.mvB = reinterpret_cast<const float2 *>(mvB);
  a.ZA = ZA;
  a.ZB = ZB;
  a.C = C;
  a.tau = tau;
  a.delta = delta;
  a.gcounts = gcounts;
  a.dLA = dLA;
  a.dLB = dLB;
  a.dmvA = reinterpret_cast<float2 *>(dmvA);
  a.dmvB = reinterpret_cast<float2 *>(dmvB);
  a.dC = dC;
  if (cudaMemsetAsync(dC, 0, sizeof(float) * n_envs, st) != cudaSuccess) return EVIS_ERR_CUDA;
  const dim3 grid((max_hw + 255) / 256, n_envs);
  soft_targets_bwd<<<grid, 256, 0, st>>>(a);
  soft_sources_bwd<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? EVIS_OK : EVIS_ERR_CUDA;
}

}  // extern "C"
