"""EVIS event synthesis on B300: a thin ctypes binding of libevis.so.

Every step of the path runs in the library's CUDA kernels; this module only marshals
arguments (torch CUDA tensors -> device pointers, the current torch stream -> the context's
stream).  There is no CPU fallback: importing the binding without the built library raises.
The C entry points are documented in ``include/evis.h``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libevis.so")

IN_LOG, IN_LUM, IN_RGB = 0x0, 0x1, 0x2
MODE_BLEND, MODE_B_PRIMARY, MODE_JOINT = 0x0, 0x10, 0x40
TIE_WEIGHT, TIE_INDEX = 0x0, 0x20
KEEP_INPUTS = 0x100
COLOR = 0x200   # R, G, B events (Sec. 3.2); polarity field +-(1 + channel)
STATS = 0x400   # collect holes, ON / OFF and noise counts for env_stats()

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_OVERFLOW, ERR_STATE, ERR_TIMEOUT, ERR_RANGE = range(8)
MAX_CROSSINGS = 4096   # crossings one pixel may emit per sub-frame (EVIS_MAX_CROSSINGS)

ENV_STATS_DTYPE = np.dtype([("target_subframes", "<u8"), ("holes_a", "<u8"), ("holes_b", "<u8"),
                            ("holes_both", "<u8"), ("events_on", "<u8"), ("events_off", "<u8"),
                            ("noise_events", "<u8"), ("over_limit", "<u8")])

EVENT_DTYPE = np.dtype([("t", "<i8"), ("x", "<u2"), ("y", "<u2"), ("env", "<u2"), ("p", "<i2")])


class EnvDesc(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("K", ctypes.c_int32),
                ("c_on", ctypes.c_float), ("c_off", ctypes.c_float), ("margin", ctypes.c_int32),
                ("c_on_map", ctypes.c_void_p), ("c_off_map", ctypes.c_void_p),
                ("refractory_ns", ctypes.c_int64), ("t0_ns", ctypes.c_int64)]


class Config(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_float), ("flags", ctypes.c_uint32),
                ("event_capacity", ctypes.c_int64)]


class NoiseDesc(ctypes.Structure):
    _fields_ = [("leak_hz", ctypes.c_float), ("shot_hz", ctypes.c_float),
                ("hot_hz", ctypes.c_float), ("hot_fraction", ctypes.c_float),
                ("lo", ctypes.c_float), ("hi", ctypes.c_float), ("seed", ctypes.c_uint64)]


class VoxelEnv(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("t0_ns", ctypes.c_int64), ("t1_ns", ctypes.c_int64)]


class EvisError(RuntimeError):
    def __init__(self, status: int, msg: str = "", events=None):
        self.status = status
        self.events = events   # what a read delivered before reporting the status
        super().__init__(f"{status_string(status)} ({status}){': ' + msg if msg else ''}")


_lib = None

_SIGS = {
    "evis_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p]),
    "evis_step": (ctypes.c_int, [ctypes.c_void_p] * 4 + [ctypes.c_int64]),
    "evis_step_host": (ctypes.c_int, [ctypes.c_void_p] * 4 + [ctypes.c_int64]),
    "evis_step_trace": (ctypes.c_int, [ctypes.c_void_p] * 4 + [ctypes.c_int64] +
                        [ctypes.c_void_p] * 2),
    "evis_read_events": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                        ctypes.c_void_p]),
    "evis_read_events_async": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                              ctypes.c_void_p]),
    "evis_read_wait": (ctypes.c_int, [ctypes.c_void_p]),
    "evis_event_count": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "evis_events_device": (ctypes.c_int, [ctypes.c_void_p] * 3),
    "evis_clear_events": (ctypes.c_int, [ctypes.c_void_p]),
    "evis_get_state": (ctypes.c_int, [ctypes.c_void_p] * 4),
    "evis_get_gaps": (ctypes.c_int, [ctypes.c_void_p] * 2),
    "evis_get_stats": (ctypes.c_int, [ctypes.c_void_p] * 4),
    "evis_get_env_stats": (ctypes.c_int, [ctypes.c_void_p] * 2),
    "evis_set_state": (ctypes.c_int, [ctypes.c_void_p] * 5),
    "evis_log_intensity": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32,
                                          ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]),
    "evis_set_noise": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "evis_voxel_workspace_size": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                                 ctypes.c_int64, ctypes.c_void_p]),
    "evis_voxel_grid": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                       ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "evis_set_defocus": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "evis_defocus": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_uint32, ctypes.c_float, ctypes.c_void_p,
                                    ctypes.c_void_p]),
    "evis_set_tile_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32]),
    "evis_set_env_tile_shapes": (ctypes.c_int, [ctypes.c_void_p] * 3),
    "evis_get_tile_shapes": (ctypes.c_int, [ctypes.c_void_p] * 3),
    "evis_autotune": (ctypes.c_int, [ctypes.c_void_p] * 4 + [ctypes.c_int64, ctypes.c_int32,
                                                             ctypes.c_void_p]),
    "evis_input_buffers": (ctypes.c_int, [ctypes.c_void_p] * 4),
    "evis_capture": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "evis_replay": (ctypes.c_int, [ctypes.c_void_p]),
    "evis_soft_workspace_size": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "evis_soft_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_float,
                                         ctypes.c_float] + [ctypes.c_void_p] * 10 +
                          [ctypes.c_int64, ctypes.c_void_p]),
    "evis_soft_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_float,
                                          ctypes.c_float] + [ctypes.c_void_p] * 14 +
                           [ctypes.c_int64, ctypes.c_void_p]),
    "evis_profile_enable": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "evis_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                         ctypes.c_void_p]),
    "evis_step_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32] + [ctypes.c_void_p] * 8 +
                          [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                           ctypes.c_int64, ctypes.c_void_p]),
    "evis_total_pixels": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "evis_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "evis_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "evis_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
}


def lib():
    """The loaded libevis.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with `python -m paper_2607_08098_b300.build` "
                "(the event-synthesis path has no CPU fallback)")
        h = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(h, name)
            fn.restype = res
            fn.argtypes = args
        _lib = h
    return _lib


def status_string(status: int) -> str:
    return lib().evis_status_string(int(status)).decode()


def _check(status: int, handle=None):
    if status != OK:
        msg = lib().evis_last_error(handle).decode() if handle is not None else ""
        raise EvisError(status, msg)


def _ptr(t) -> int:
    """Device pointer of a contiguous torch CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class Context:
    """An event-synthesis context over a list of environments.

    ``envs`` items need ``W, H, K, c_on, c_off`` and may have ``refractory_ns``, ``t0_ns``
    and per-pixel ``c_on_map`` / ``c_off_map`` (CUDA float32 tensors of H*W, kept alive by
    this object).  Inputs to :meth:`step` are CUDA float32 tensors in the packed layout.
    """

    def __init__(self, envs, eps: float = 1e-4, flags: int = 0, capacity: int = 1 << 22,
                 stream=None):
        import torch
        L = lib()
        self.envs = list(envs)
        self.flags = int(flags)
        self.capacity = int(capacity)
        self._keep = []
        arr = (EnvDesc * len(self.envs))()
        for i, e in enumerate(self.envs):
            con = getattr(e, "c_on_map", None)
            coff = getattr(e, "c_off_map", None)
            if con is not None:
                con = torch.as_tensor(con, dtype=torch.float32).cuda().contiguous()
                coff = torch.as_tensor(coff, dtype=torch.float32).cuda().contiguous()
                self._keep += [con, coff]
            arr[i] = EnvDesc(int(e.W), int(e.H), int(e.K), float(e.c_on), float(e.c_off),
                             int(getattr(e, "margin", 0)), _ptr(con), _ptr(coff),
                             int(getattr(e, "refractory_ns", 0)),
                             int(getattr(e, "t0_ns", 0)))
        cfg = Config(float(eps), self.flags, self.capacity)
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        st = L.evis_create(ctypes.addressof(arr), len(self.envs), ctypes.addressof(cfg),
                           _stream_handle(self._stream), ctypes.byref(h))
        if st != OK:
            raise EvisError(st, L.evis_last_error(None).decode())
        self._h = h
        n = ctypes.c_int64()
        _check(L.evis_total_pixels(self._h, ctypes.byref(n)), self._h)
        self.total = n.value
        self.nc = 3 if self.flags & COLOR else 1
        self.n_frame = self.total * (3 if ((self.flags & 0x3) == IN_RGB or self.nc == 3) else 1)

    @property
    def handle(self):
        return self._h

    @property
    def stream(self):
        return self._stream

    def close(self):
        if getattr(self, "_h", None):
            lib().evis_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check_inputs(self, frames, mv, depth):
        for name, t, n in (("frames", frames, self.n_frame), ("mv", mv, 2 * self.total),
                           ("depth", depth, self.total)):
            if not t.is_cuda or t.dtype.itemsize != 4 or t.numel() != n:
                raise ValueError(f"{name}: expected a CUDA float32 tensor of {n} elements")

    def step(self, frames, mv, depth, dt_ns: int):
        self._check_inputs(frames, mv, depth)
        _check(lib().evis_step(self._h, _ptr(frames), _ptr(mv), _ptr(depth), int(dt_ns)), self._h)

    def step_trace(self, frames, mv, depth, dt_ns: int):
        """Step and return (keys [sum K*2*H*W] uint64 as int64, Lint [sum K*H*W]) tensors."""
        import torch
        self._check_inputs(frames, mv, depth)
        nk = sum(e.K * 2 * e.H * e.W for e in self.envs)
        nl = sum(e.K * self.nc * e.H * e.W for e in self.envs)
        keys = torch.empty(nk, dtype=torch.int64, device=frames.device)
        lint = torch.empty(nl, dtype=torch.float32, device=frames.device)
        _check(lib().evis_step_trace(self._h, _ptr(frames), _ptr(mv), _ptr(depth), int(dt_ns),
                                     _ptr(keys), _ptr(lint)), self._h)
        return keys, lint

    def step_host(self, frames: np.ndarray, mv: np.ndarray, depth: np.ndarray, dt_ns: int):
        """Step from host arrays (numpy or pinned torch CPU tensors)."""
        def hp(a, n):
            if hasattr(a, "data_ptr"):
                if a.numel() != n:
                    raise ValueError("host input has the wrong size")
                return a.data_ptr()
            a = np.ascontiguousarray(a, dtype=np.float32)
            if a.size != n:
                raise ValueError("host input has the wrong size")
            return a.ctypes.data
        _check(lib().evis_step_host(self._h, hp(frames, self.n_frame), hp(mv, 2 * self.total),
                                    hp(depth, self.total), int(dt_ns)), self._h)

    def read_events(self, cap: int | None = None, allow_overflow: bool = False,
                    allow_over_limit: bool = False):
        """Drain the event buffer to a numpy structured array (EVENT_DTYPE).

        A pixel-sub-frame beyond the crossing limit since the last read raises EvisError
        (ERR_RANGE, the delivered events in .events) unless allow_over_limit is set; its
        count per environment is in env_stats()."""
        n = ctypes.c_int64()
        cnt = self.event_count()
        if cap is None:
            cap = min(cnt, self.capacity)
        out = np.empty(max(cap, 0), dtype=EVENT_DTYPE)
        st = lib().evis_read_events(self._h, out.ctypes.data if cap else None, int(cap),
                                    ctypes.byref(n))
        got = out[:min(n.value, cap)]
        over = n.value > min(cap, self.capacity)
        if st == ERR_RANGE:
            if not allow_over_limit:
                raise EvisError(st, "a pixel-sub-frame exceeded the crossing limit", events=got)
            st = ERR_OVERFLOW if over else OK
        if st == ERR_OVERFLOW and allow_overflow:
            return got, n.value
        _check(st, self._h)
        return (got, n.value) if allow_overflow else got

    def read_events_async(self, dst_ptr: int, cap: int) -> int:
        """Start copying the buffered events to dst_ptr (pinned host or device memory, room
        for cap records) while the next steps fill the context's other buffer; returns the
        number of events produced since the last read.  dst is complete once the next
        read_events_async or read_wait returns."""
        n = ctypes.c_int64()
        _check(lib().evis_read_events_async(self._h, dst_ptr, int(cap), ctypes.byref(n)), self._h)
        return n.value

    def read_wait(self):
        """Wait for the copy started by the last read_events_async."""
        _check(lib().evis_read_wait(self._h), self._h)

    def event_count(self) -> int:
        n = ctypes.c_int64()
        st = lib().evis_event_count(self._h, ctypes.byref(n))
        if st not in (OK, ERR_OVERFLOW, ERR_RANGE):
            _check(st, self._h)
        return n.value

    def clear_events(self):
        _check(lib().evis_clear_events(self._h), self._h)

    def events_device(self):
        ev = ctypes.c_void_p()
        cnt = ctypes.c_void_p()
        _check(lib().evis_events_device(self._h, ctypes.byref(ev), ctypes.byref(cnt)), self._h)
        return ev.value, cnt.value

    def set_noise(self, specs):
        """Sensor noise per environment (Sec. 3.4): a list of dicts with leak_hz, shot_hz,
        hot_hz, hot_fraction, lo, hi, seed (missing keys off / defaults), or None for off."""
        if specs is None:
            _check(lib().evis_set_noise(self._h, None), self._h)
            return
        if len(specs) != len(self.envs):
            raise ValueError("one noise spec per environment")
        arr = (NoiseDesc * len(specs))()
        for i, sp in enumerate(specs):
            arr[i] = NoiseDesc(sp.get("leak_hz", 0.0), sp.get("shot_hz", 0.0), sp.get("hot_hz", 0.0),
                               sp.get("hot_fraction", 0.0), sp.get("lo", -5.0), sp.get("hi", 5.0),
                               int(sp.get("seed", 0)))
        _check(lib().evis_set_noise(self._h, ctypes.addressof(arr)), self._h)

    def set_defocus(self, sigmas):
        """Per-environment defocus sigma in pixels (Sec. 3.4), or None for none."""
        if sigmas is None:
            _check(lib().evis_set_defocus(self._h, None), self._h)
            return
        sg = np.ascontiguousarray(sigmas, dtype=np.float32)
        if sg.size != len(self.envs):
            raise ValueError("one sigma per environment")
        _check(lib().evis_set_defocus(self._h, sg.ctypes.data), self._h)

    def voxel_grid(self, segments, bins: int = 128, workspace=None):
        """Voxel grid of the events currently in the device buffer (read in place, count
        taken on the device): segments as for the module-level voxel_grid, one per
        environment; sensor sizes are the environments' minus their margins."""
        ev, cnt = self.events_device()
        return voxel_grid(ev, cnt, self.capacity, segments, bins, workspace, self._stream)

    TILE_SHAPES = ((32, 8), (32, 16), (32, 32), (64, 16), (64, 32), (128, 16))

    def set_tile_shape(self, tile_w: int, tile_h: int):
        """Target tile of the synthesis kernel (speed only; results are identical)."""
        _check(lib().evis_set_tile_shape(self._h, int(tile_w), int(tile_h)), self._h)

    def set_env_tile_shapes(self, shapes):
        """Per-environment (tile_w, tile_h) pairs."""
        tw = np.array([t[0] for t in shapes], dtype=np.int32)
        th = np.array([t[1] for t in shapes], dtype=np.int32)
        _check(lib().evis_set_env_tile_shapes(self._h, tw.ctypes.data, th.ctypes.data), self._h)

    def tile_shapes(self):
        tw = np.zeros(len(self.envs), dtype=np.int32)
        th = np.zeros(len(self.envs), dtype=np.int32)
        _check(lib().evis_get_tile_shapes(self._h, tw.ctypes.data, th.ctypes.data), self._h)
        return list(zip(tw.tolist(), th.tolist()))

    def autotune(self, frames, mv, depth, dt_ns: int, reps: int = 3) -> float:
        """Pick the fastest tile shape per resolution class on the gap to this keyframe (the
        state is left unchanged); returns the summed best time in ms."""
        self._check_inputs(frames, mv, depth)
        best = ctypes.c_float()
        _check(lib().evis_autotune(self._h, _ptr(frames), _ptr(mv), _ptr(depth), int(dt_ns),
                                   int(reps), ctypes.byref(best)), self._h)
        return best.value

    def input_buffers(self):
        """(frames, mv, depth) device pointers of the library's current input buffers."""
        f, m, d = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib().evis_input_buffers(self._h, ctypes.byref(f), ctypes.byref(m), ctypes.byref(d)),
               self._h)
        return f.value, m.value, d.value

    def write_inputs(self, frames, mv, depth):
        """Copy CUDA tensors into the current input buffers (stream-ordered, device to device)."""
        from cuda.bindings import runtime as rt
        self._check_inputs(frames, mv, depth)
        dst = self.input_buffers()
        strm = _stream_handle(self._stream)
        for d, t in zip(dst, (frames, mv, depth)):
            err, = rt.cudaMemcpyAsync(d, _ptr(t), t.numel() * 4,
                                      rt.cudaMemcpyKind.cudaMemcpyDeviceToDevice, strm)
            if err != rt.cudaError_t.cudaSuccess:
                raise EvisError(ERR_CUDA, f"cudaMemcpyAsync: {err}")

    def capture(self, dt_ns: int):
        _check(lib().evis_capture(self._h, int(dt_ns)), self._h)

    def replay(self):
        _check(lib().evis_replay(self._h), self._h)

    def profile(self, max_steps: int):
        """Record per-phase CUDA events for the next ``max_steps`` steps (0 disables)."""
        _check(lib().evis_profile_enable(self._h, int(max_steps)), self._h)

    def profile_read(self) -> np.ndarray:
        """[steps, 2] milliseconds: (input preparation, synthesis kernel) per profiled step."""
        buf = np.zeros(2 * 4096, dtype=np.float32)
        n = ctypes.c_int32()
        _check(lib().evis_profile_read(self._h, buf.ctypes.data, 4096, ctypes.byref(n)), self._h)
        return buf[:2 * n.value].reshape(-1, 2)

    def stats(self):
        """{'keyframes', 'gaps', 'invalid_sources' [n_envs]} since creation."""
        kf = ctypes.c_uint64()
        gp = ctypes.c_uint64()
        inv = np.zeros(len(self.envs), dtype=np.uint64)
        _check(lib().evis_get_stats(self._h, ctypes.byref(kf), ctypes.byref(gp), inv.ctypes.data),
               self._h)
        return {"keyframes": kf.value, "gaps": gp.value, "invalid_sources": inv}

    def env_stats(self) -> np.ndarray:
        """Per-environment statistics since creation (ENV_STATS_DTYPE): target-sub-frames,
        holes of each warp direction and of both, ON / OFF events, noise events and
        pixel-sub-frames beyond the crossing limit."""
        out = np.zeros(len(self.envs), dtype=ENV_STATS_DTYPE)
        _check(lib().evis_get_env_stats(self._h, out.ctypes.data), self._h)
        return out

    def gaps(self):
        """Keyframe gaps processed per environment (the noise generator's gap counter)."""
        g = np.empty(len(self.envs), dtype=np.uint32)
        _check(lib().evis_get_gaps(self._h, g.ctypes.data), self._h)
        return g

    def set_state(self, Lref=None, t_last=None, clocks=None, gaps=None):
        """Restore a checkpoint (host arrays as returned by state() and gaps()); feed the
        last keyframe before the checkpoint first."""
        def arr(a, dt):
            return None if a is None else np.ascontiguousarray(a, dtype=dt)
        keep = [arr(Lref, np.float32), arr(t_last, np.int64), arr(clocks, np.int64),
                arr(gaps, np.uint32)]
        ptrs = [None if a is None else a.ctypes.data for a in keep]
        _check(lib().evis_set_state(self._h, *ptrs), self._h)

    def state(self):
        """(Lref, t_last, clocks); Lref and t_last hold nc planes of total pixels."""
        Lref = np.empty(self.nc * self.total, dtype=np.float32)
        tl = np.empty(self.nc * self.total, dtype=np.int64)
        clk = np.empty(len(self.envs), dtype=np.int64)
        _check(lib().evis_get_state(self._h, Lref.ctypes.data, tl.ctypes.data, clk.ctypes.data),
               self._h)
        return Lref, tl, clk


def log_intensity(x, mode: int = IN_LUM, eps: float = 1e-4):
    """log(I + eps) of a CUDA tensor (I, or Rec. 709 luminance of [..., 3] RGB) on the GPU."""
    import torch
    x = x.contiguous()
    n = x.numel() // 3 if mode == IN_RGB else x.numel()
    out = torch.empty(n, dtype=torch.float32, device=x.device)
    _check(lib().evis_log_intensity(_ptr(x), n, int(mode), float(eps), _ptr(out),
                                    torch.cuda.current_stream().cuda_stream))
    return out


def defocus(image, sigma: float, stream=None):
    """Blurred luminance [H, W] of a CUDA float32 image [H, W] (luminance) or [H, W, 3]
    (linear RGB), by the library's defocus kernel (Sec. 3.4)."""
    import torch
    if image.dim() not in (2, 3) or (image.dim() == 3 and image.shape[2] != 3):
        raise ValueError("image must be [H, W] or [H, W, 3]")
    img = image.contiguous()
    H, W = img.shape[0], img.shape[1]
    out = torch.empty((H, W), dtype=torch.float32, device=img.device)
    mode = IN_RGB if img.dim() == 3 else IN_LUM
    _check(lib().evis_defocus(_ptr(img), W, H, mode, float(sigma), _ptr(out), _stream_handle(stream)))
    return out


def _voxel_envs(segments):
    arr = (VoxelEnv * len(segments))()
    for i, (W, H, t0, t1) in enumerate(segments):
        arr[i] = VoxelEnv(int(W), int(H), int(t0), int(t1))
    return arr


def voxel_workspace_size(segments, bins: int = 128, max_events: int = 0) -> int:
    """Device workspace bytes of voxel_grid for up to max_events records."""
    n = ctypes.c_int64()
    arr = _voxel_envs(segments)
    _check(lib().evis_voxel_workspace_size(ctypes.addressof(arr), len(segments), int(bins),
                                           int(max_events), ctypes.byref(n)))
    return n.value


def voxel_grid(events_ptr: int, count_ptr, max_events: int, segments, bins: int = 128,
               workspace=None, stream=None):
    """Event voxel grid (per polarity, linear interpolation in time, per-bin max
    normalisation) of device event records: segments is a list of (width, height, t0_ns,
    t1_ns) per environment; count_ptr a device uint64 pointer or None.  Returns a CUDA float
    tensor, per environment [2][bins][H][W] concatenated."""
    import torch
    arr = _voxel_envs(segments)
    wsb = voxel_workspace_size(segments, bins, max_events)
    if workspace is None or workspace.numel() < wsb:
        workspace = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    n_vox = sum(2 * bins * int(W) * int(H) for W, H, _, _ in segments)
    out = torch.empty(n_vox, dtype=torch.float32, device="cuda")
    _check(lib().evis_voxel_grid(events_ptr, count_ptr, int(max_events), ctypes.addressof(arr),
                                 len(segments), int(bins), workspace.data_ptr(), int(workspace.numel()),
                                 out.data_ptr(), _stream_handle(stream)))
    return out


def sort_events(ev: np.ndarray) -> np.ndarray:
    """Order (env, t, y, x, p): the buffer order is arbitrary, this one is canonical."""
    return ev[np.lexsort((ev["p"], ev["x"], ev["y"], ev["t"], ev["env"]))]


def _descs(envs):
    arr = (EnvDesc * len(envs))()
    for i, e in enumerate(envs):
        arr[i] = EnvDesc(int(e.W), int(e.H), int(e.K), float(e.c_on), float(e.c_off),
                         int(getattr(e, "margin", 0)), None, None, 0, 0)
    return arr


def soft_workspace_bytes(envs) -> int:
    n = ctypes.c_int64()
    arr = _descs(envs)
    _check(lib().evis_soft_workspace_size(ctypes.addressof(arr), len(envs), ctypes.byref(n)))
    return n.value


def _soft_forward(envs, tau, delta, LA, LB, mvA, mvB, ZA, ZB, Lref0, C, ws=None):
    import torch
    arr = _descs(envs)
    if ws is None:
        ws = torch.empty(soft_workspace_bytes(envs), dtype=torch.uint8, device=LA.device)
    counts = torch.empty(2 * LA.numel(), dtype=torch.float32, device=LA.device)
    _check(lib().evis_soft_forward(ctypes.addressof(arr), len(envs), float(tau), float(delta),
                                   *[_ptr(t) for t in (LA, LB, mvA, mvB, ZA, ZB, Lref0, C, counts,
                                                        ws)],
                                   ws.numel(), torch.cuda.current_stream().cuda_stream))
    return counts, ws


def _soft_backward(envs, tau, delta, LA, LB, mvA, mvB, ZA, ZB, C, ws, gcounts):
    import torch
    arr = _descs(envs)
    out = [torch.empty_like(LA), torch.empty_like(LB), torch.empty_like(mvA),
           torch.empty_like(mvB), torch.empty_like(C)]
    _check(lib().evis_soft_backward(ctypes.addressof(arr), len(envs), float(tau), float(delta),
                                    *[_ptr(t) for t in (LA, LB, mvA, mvB, ZA, ZB, C,
                                                         gcounts.contiguous(), *out, ws)],
                                    ws.numel(), torch.cuda.current_stream().cuda_stream))
    return out


def _make_soft_function():
    import torch

    class SoftEventCount(torch.autograd.Function):
        """Soft ON/OFF event counts of one keyframe gap (include/evis.h, evis_soft_forward),
        differentiable in L_A, L_B, mv_A, mv_B and C; depth and Lref0 are constants."""

        @staticmethod
        def forward(ctx, LA, LB, mvA, mvB, ZA, ZB, Lref0, C, envs, tau, delta):
            ts = [t.contiguous().float() for t in (LA, LB, mvA, mvB, ZA, ZB, Lref0, C)]
            counts, ws = _soft_forward(envs, tau, delta, *ts)
            ctx.save_for_backward(*ts[:6], ts[7], ws)
            ctx.envs, ctx.tau, ctx.delta = envs, tau, delta
            return counts

        @staticmethod
        def backward(ctx, gcounts):
            LA, LB, mvA, mvB, ZA, ZB, C, ws = ctx.saved_tensors
            dLA, dLB, dmvA, dmvB, dC = _soft_backward(ctx.envs, ctx.tau, ctx.delta, LA, LB, mvA,
                                                      mvB, ZA, ZB, C, ws, gcounts.float())
            return dLA, dLB, dmvA, dmvB, None, None, None, dC, None, None, None

    return SoftEventCount


_soft_fn = None


def soft_event_counts(LA, LB, mvA, mvB, ZA, ZB, Lref0, C, envs, tau=0.02, delta=1e-3):
    """Differentiable soft event counts (packed [2][H][W] per environment) of one gap."""
    global _soft_fn
    if _soft_fn is None:
        _soft_fn = _make_soft_function()
    return _soft_fn.apply(LA, LB, mvA, mvB, ZA, ZB, Lref0, C, envs, tau, delta)
