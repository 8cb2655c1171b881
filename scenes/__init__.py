"""Seeded synthetic scenes: the one input generator shared by the CUDA path and the oracle.

The paper renders keyframes with a physics engine and a ray-traced renderer (Sec. 3.1,
Eqs. 1-2) and reads the renderer's backward motion vectors and depth (Sec. 3.3).  Neither is
available here, so this module renders analytic layered scenes with the same three buffers
per keyframe: log-radiance (or linear / RGB radiance), motion vectors pointing from each pixel
to its position in the previous keyframe, and depth.  It contains none of the event-synthesis
arithmetic; both sides receive its arrays as inputs.

Packed layout (shared by every consumer): environment e owns pixels
``[pix_off[e], pix_off[e] + H*W)`` where ``pix_off`` is the prefix sum of ``H*W`` rounded up
to a multiple of 4, so each environment starts on a 16-byte boundary.  ``mv`` uses twice
those offsets (interleaved dx, dy) and RGB three times.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libevis_scenes.so")
_SRC = os.path.join(_HERE, "evis_scenes.cpp")
_lib = None

LN10 = 2.302585092994046

# layer field order, mirrors the enum in evis_scenes.cpp
_FIELDS = ["kind", "radius", "depth0", "depth_rate", "cx0", "cy0", "vx", "vy", "angle0",
           "omega", "tex_kind", "seed", "cell", "mu", "sigma", "lo", "hi", "bright_rate",
           "tint_r", "tint_g", "tint_b"]


def build(force: bool = False) -> str:
    """Compile the generator library in place (g++, host only)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
                               _SRC, "-o", _SO])
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        lib.scenes_layer_doubles.restype = ctypes.c_int
        lib.scenes_render.restype = ctypes.c_int
        lib.scenes_render.argtypes = [ctypes.c_int32] + [ctypes.c_void_p] * 6 + [ctypes.c_int32] + \
            [ctypes.c_void_p] * 5 + [ctypes.c_int32]
        assert lib.scenes_layer_doubles() == len(_FIELDS)
        _lib = lib
    return _lib


@dataclass
class Layer:
    kind: int = 0            # 0 plane, 1 disk
    radius: float = 0.0
    depth0: float = 5.0
    depth_rate: float = 0.0
    cx0: float = 0.0
    cy0: float = 0.0
    vx: float = 0.0
    vy: float = 0.0
    angle0: float = 0.0
    omega: float = 0.0
    tex_kind: int = 0        # 0 value noise, 1 constant, 2 ramp along local x
    seed: int = 0
    cell: float = 16.0
    mu: float = 0.5
    sigma: float = 1.25
    lo: float = -2.0
    hi: float = 3.0
    bright_rate: float = 0.0
    tint_r: float = 1.0
    tint_g: float = 1.0
    tint_b: float = 1.0

    def as_array(self) -> np.ndarray:
        return np.array([float(getattr(self, f)) for f in _FIELDS], dtype=np.float64)


@dataclass
class EnvScene:
    """One environment: sensor geometry, event parameters and its layers."""
    W: int
    H: int
    K: int
    c_on: float
    c_off: float
    refractory_ns: int = 0
    t0_ns: int = 0
    layers: list = field(default_factory=list)
    c_on_map: np.ndarray | None = None   # optional per-pixel thresholds [H*W] float32
    c_off_map: np.ndarray | None = None
    margin: int = 0                      # over-render margin per side (W, H include it)


def pixel_offsets(envs) -> tuple[np.ndarray, int]:
    """Packed pixel offsets (each rounded up to a multiple of 4) and the padded total."""
    off = np.zeros(len(envs), dtype=np.int64)
    acc = 0
    for i, e in enumerate(envs):
        off[i] = acc
        acc += (e.H * e.W + 3) // 4 * 4
    return off, acc


@dataclass
class Keyframe:
    L: np.ndarray | None     # [npx] float32 log-radiance (natural log)
    I: np.ndarray | None     # [npx] float32 linear radiance
    rgb: np.ndarray | None   # [npx, 3] float32
    mv: np.ndarray           # [npx, 2] float32 backward motion vectors (pixels)
    Z: np.ndarray            # [npx] float32 depth


def render(envs, k: int, want=("L", "I", "mv", "Z"), threads: int | None = None) -> Keyframe:
    """Render keyframe ``k`` of every environment into packed arrays."""
    lib = _load()
    off, total = pixel_offsets(envs)
    n = len(envs)
    W = np.array([e.W for e in envs], dtype=np.int32)
    H = np.array([e.H for e in envs], dtype=np.int32)
    nl = np.array([len(e.layers) for e in envs], dtype=np.int32)
    lo = np.zeros(n, dtype=np.int32)
    if n:
        lo[1:] = np.cumsum(nl)[:-1]
    lay = np.concatenate([l.as_array() for e in envs for l in e.layers]) if nl.sum() else \
        np.zeros(len(_FIELDS))
    out = {}
    # padding pixels between environments (each environment's H*W rounded up to 4): zero
    # motion, unit depth and linear radiance, zero log-radiance; the renderer's threads write
    # every other pixel (and so touch the pages of the large arrays in parallel)
    pads = [np.arange(o + e.H * e.W, o + (e.H * e.W + 3) // 4 * 4) for e, o in zip(envs, off)]
    pads = np.concatenate(pads) if pads else np.zeros(0, np.int64)
    for name, width in (("L", 1), ("I", 1), ("rgb", 3), ("mv", 2), ("Z", 1)):
        if name in want:
            a = np.empty(total * width, dtype=np.float32)
            v = a.reshape(total, width)
            v[pads] = 1.0 if name in ("Z", "I") else 0.0
            out[name] = a
        else:
            out[name] = None
    p = lambda a: a.ctypes.data if a is not None else None  # noqa: E731
    if threads is None:
        threads = min(32, os.cpu_count() or 1)
    rc = lib.scenes_render(n, W.ctypes.data, H.ctypes.data, off.ctypes.data, lo.ctypes.data,
                           nl.ctypes.data, lay.ctypes.data, int(k), p(out["L"]), p(out["I"]),
                           p(out["rgb"]), p(out["mv"]), p(out["Z"]), int(threads))
    if rc != 0:
        raise ValueError("scenes_render rejected the environment table")
    return Keyframe(L=out["L"], I=out["I"],
                    rgb=None if out["rgb"] is None else out["rgb"].reshape(-1, 3),
                    mv=out["mv"].reshape(-1, 2), Z=out["Z"])


def threshold_maps(envs, offsets=None, total=None):
    """Packed per-pixel ON/OFF threshold maps, or (None, None) if no env has one."""
    if not any(e.c_on_map is not None for e in envs):
        return None, None
    if offsets is None:
        offsets, total = pixel_offsets(envs)
    con = np.zeros(total, dtype=np.float32)
    coff = np.zeros(total, dtype=np.float32)
    for e, o in zip(envs, offsets):
        n = e.H * e.W
        con[o:o + n] = e.c_on_map if e.c_on_map is not None else e.c_on
        coff[o:o + n] = e.c_off_map if e.c_off_map is not None else e.c_off
    return con, coff


# --------------------------------------------------------------------------------------
# Workloads.  Seeds: splitmix64(config_seed ^ env) with config_seed = 0xE7150000 + number.
# --------------------------------------------------------------------------------------

def splitmix64(x: int) -> int:
    m = (1 << 64) - 1
    x = (x + 0x9E3779B97F4A7C15) & m
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & m
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & m
    return x ^ (x >> 31)


def _rng(config_no: int, env: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(splitmix64((0xE7150000 + config_no) ^ env)))


def _tex_seed(rng) -> int:
    return int(rng.integers(0, 1 << 52))


def _random_layers(rng, W, H, n_layers, vmax, wmax, rmin=0.15, rmax=0.3, dmin=1.0, dmax=10.0):
    """A plane (farthest) plus ``n_layers - 1`` disks with random rigid 2D motions."""
    depths = np.sort(rng.uniform(dmin, dmax, size=n_layers))[::-1]
    layers = []
    for l in range(n_layers):
        speed = rng.uniform(0.0, vmax)
        ang = rng.uniform(0.0, 2.0 * np.pi)
        omega = rng.uniform(-wmax, wmax)
        common = dict(depth0=float(depths[l]), vx=float(speed * np.cos(ang)),
                      vy=float(speed * np.sin(ang)), omega=float(omega), seed=_tex_seed(rng),
                      angle0=float(rng.uniform(0, 2 * np.pi)))
        if l == 0:
            layers.append(Layer(kind=0, cx0=W / 2.0, cy0=H / 2.0, cell=16.0, **common))
        else:
            r = rng.uniform(rmin, rmax) * min(W, H)
            layers.append(Layer(kind=1, radius=float(r), cx0=float(rng.uniform(0, W)),
                                cy0=float(rng.uniform(0, H)), cell=float(rng.choice([8.0, 16.0])),
                                **common))
    return layers


@dataclass
class Workload:
    name: str
    envs: list
    dt_ns: int
    n_pairs: int

    @property
    def offsets(self):
        return pixel_offsets(self.envs)

    @property
    def pixel_substeps(self) -> int:
        return int(sum(e.H * e.W * e.K for e in self.envs))

    @property
    def pixels(self) -> int:
        return int(sum(e.H * e.W for e in self.envs))


def config1() -> Workload:
    """Plain single env: 128x128, 10 pairs, K=8, C=0.2, background plane + rotating disk."""
    c30, s30 = np.cos(np.pi / 6), np.sin(np.pi / 6)
    bg = Layer(kind=0, depth0=5.0, cx0=64.0, cy0=64.0, vx=3.0, vy=0.0, cell=16.0,
               seed=0xE7150001)
    disk = Layer(kind=1, radius=30.0, depth0=2.0, cx0=40.0, cy0=50.0, vx=6 * c30, vy=6 * s30,
                 omega=0.05, cell=8.0, seed=0xE7150101)
    env = EnvScene(W=128, H=128, K=8, c_on=0.2, c_off=0.2, layers=[bg, disk])
    return Workload("plain single env 128x128, K=8, C=0.2, 10 frame pairs", [env],
                    33_333_333, 10)


def config2(n_envs: int = 64, W: int = 346, H: int = 260, first_env: int = 0) -> Workload:
    """64 envs at 346x260, 32 pairs, K=16, C=0.25, refractory 100 us, three depth layers.
    ``first_env`` shifts the seeds (environment e uses seed index first_env + e)."""
    envs = []
    for e in range(first_env, first_env + n_envs):
        rng = _rng(2, e)
        envs.append(EnvScene(W=W, H=H, K=16, c_on=0.25, c_off=0.25, refractory_ns=100_000,
                             layers=_random_layers(rng, W, H, 3, vmax=10.0, wmax=0.1)))
    return Workload(f"{n_envs} envs at {W}x{H}, K=16, C=0.25, refractory 100us, 3 layers",
                    envs, 16_666_667, 32)


def config3(n_envs: int = 256, scale: float = 1.0) -> Workload:
    """Batched uneven: mixed resolutions 4:2:1:1, K ~ U{4..32}, per-pixel thresholds."""
    sizes = [(128, 128)] * 4 + [(346, 260)] * 2 + [(640, 480), (1280, 720)]
    order = _rng(3, 1 << 40).permutation(n_envs)
    envs = []
    for e in range(n_envs):
        rng = _rng(3, e)
        W, H = sizes[int(order[e]) % 8]
        W, H = max(8, int(W * scale)), max(8, int(H * scale))
        K = int(rng.integers(4, 33))
        con = np.maximum(rng.normal(0.2, 0.03, size=H * W), 0.01).astype(np.float32)
        coff = np.maximum(rng.normal(0.2, 0.03, size=H * W), 0.01).astype(np.float32)
        envs.append(EnvScene(W=W, H=H, K=K, c_on=0.2, c_off=0.2, c_on_map=con, c_off_map=coff,
                             layers=_random_layers(rng, W, H, 3, vmax=10.0, wmax=0.1)))
    return Workload(f"{n_envs} envs mixed resolution, K~U(4..32), per-pixel C", envs,
                    16_666_667, 8)


def config4(n_envs: int = 1024, W: int = 640, H: int = 480, first_env: int = 0) -> Workload:
    """High-speed: 640x480, K=32, flows up to 40 px/frame, five depth layers, C=0.15.

    Disks of radius 0.2-0.4 x 480 moving up to 40 px/frame leave about 10 % of the
    pixel-substeps without a source in one warp direction or the other (5-8 % in each,
    measured on environments 0, 511 and 1023: disocclusion holes); textures are
    smoother (64 px cells, sigma 0.3) so that the output stays event-dense but bounded
    (about 0.11 events per pixel-substep).  ``first_env`` shifts the seeds (environment e
    uses seed index first_env + e)."""
    envs = []
    for e in range(first_env, first_env + n_envs):
        rng = _rng(4, e)
        lay = _random_layers(rng, W, H, 5, vmax=40.0, wmax=0.1, rmin=0.2, rmax=0.4)
        for layer in lay:
            layer.sigma, layer.cell = 0.3, 64.0
        envs.append(EnvScene(W=W, H=H, K=32, c_on=0.15, c_off=0.15, layers=lay))
    return Workload(f"{n_envs} envs at {W}x{H}, K=32, C=0.15, 5 layers, flow<=40px", envs,
                    8_000_000, 4)


def config5(n_envs: int = 16, W: int = 346, H: int = 260) -> Workload:
    """Differentiable: 16 envs at 346x260, K=8 (soft event-count surrogate, tau=0.02)."""
    envs = []
    for e in range(n_envs):
        rng = _rng(5, e)
        envs.append(EnvScene(W=W, H=H, K=8, c_on=0.2, c_off=0.2,
                             layers=_random_layers(rng, W, H, 3, vmax=10.0, wmax=0.1)))
    return Workload(f"{n_envs} envs at {W}x{H}, K=8, soft counts tau=0.02", envs,
                    16_666_667, 1)


CONFIGS = {1: config1, 2: config2, 3: config3, 4: config4, 5: config5}
