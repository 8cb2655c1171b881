"""The C-ABI library builds, loads and exports every symbol include/evis.h declares, and its
host-side validation rejects bad arguments before touching CUDA (CPU only)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def evis():
    from paper_2607_08098_b300 import build
    build.build()
    import paper_2607_08098_b300 as ev
    return ev


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(evis_\w+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(evis):
    names = _declared()
    assert {"evis_create", "evis_step", "evis_read_events", "evis_destroy"} <= names
    out = subprocess.check_output(["nm", "-D", "--defined-only", evis.LIB_PATH], text=True)
    exported = set(re.findall(r"\bT (evis_\w+)", out))
    missing = names - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    h = ctypes.CDLL(evis.LIB_PATH)
    for n in names:
        getattr(h, n)


def test_binding_covers_the_abi(evis):
    names = _declared()
    bound = set(evis._SIGS)
    assert names <= bound, names - bound


def _desc(ev, **kw):
    d = dict(width=64, height=32, K=8, c_on=0.2, c_off=0.2, c_on_map=None, c_off_map=None,
             refractory_ns=0, t0_ns=0)
    d.update(kw)
    return ev.EnvDesc(**d)


@pytest.mark.parametrize("bad", [
    dict(width=0), dict(height=70000), dict(width=8192, height=4096), dict(K=0), dict(K=5000),
    dict(c_on=0.0), dict(c_off=-1.0), dict(c_on=float("nan")), dict(c_off=float("inf")),
    dict(refractory_ns=-1), dict(c_on_map=1234), dict(margin=-1), dict(margin=16),
    dict(width=8, margin=4), dict(c_on_map=0x100002, c_off_map=0x200000),
    dict(c_on_map=0x100000, c_off_map=0x200001),
])
def test_create_rejects_bad_descriptors_before_cuda(evis, bad):
    L = evis.lib()
    arr = (evis.EnvDesc * 1)(_desc(evis, **bad))
    cfg = evis.Config(1e-4, 0, 1024)
    h = ctypes.c_void_p()
    st = L.evis_create(ctypes.addressof(arr), 1, ctypes.addressof(cfg), None, ctypes.byref(h))
    assert st == evis.ERR_INVALID_ARG
    assert h.value is None
    assert L.evis_last_error(None).decode() != ""


@pytest.mark.parametrize("cfg", [(-1.0, 0, 10), (float("nan"), 0, 10), (1e-4, 0x3, 10), (1e-4, 0x50, 10),
                                 (1e-4, 0x8000, 10), (1e-4, 0, 0), (1e-4, 0, 1 << 41)])
def test_create_rejects_bad_config(evis, cfg):
    L = evis.lib()
    arr = (evis.EnvDesc * 1)(_desc(evis))
    c = evis.Config(*cfg)
    h = ctypes.c_void_p()
    st = L.evis_create(ctypes.addressof(arr), 1, ctypes.addressof(c), None, ctypes.byref(h))
    assert st == evis.ERR_INVALID_ARG


def test_create_rejects_bad_counts_and_nulls(evis):
    L = evis.lib()
    arr = (evis.EnvDesc * 1)(_desc(evis))
    c = evis.Config(1e-4, 0, 16)
    h = ctypes.c_void_p()
    assert L.evis_create(ctypes.addressof(arr), 0, ctypes.addressof(c), None, ctypes.byref(h)) == 1
    assert L.evis_create(None, 1, ctypes.addressof(c), None, ctypes.byref(h)) == 1
    assert L.evis_create(ctypes.addressof(arr), 1, None, None, ctypes.byref(h)) == 1
    assert L.evis_create(ctypes.addressof(arr), 1, ctypes.addressof(c), None, None) == 1


def test_null_context_calls_are_rejected(evis):
    L = evis.lib()
    n = ctypes.c_int64()
    assert L.evis_step(None, None, None, None, 1) == evis.ERR_INVALID_ARG
    assert L.evis_read_events(None, None, 0, ctypes.byref(n)) == evis.ERR_INVALID_ARG
    assert L.evis_destroy(None) == evis.ERR_INVALID_ARG
    assert L.evis_log_intensity(None, 4, 0, 1e-4, None, None) == evis.ERR_INVALID_ARG
    assert L.evis_log_intensity(None, 4, 7, 1e-4, None, None) == evis.ERR_INVALID_ARG
    assert evis.status_string(evis.ERR_OVERFLOW) == "event buffer overflow"


def test_binding_fails_loudly_without_library(evis, monkeypatch):
    monkeypatch.setattr(evis, "_lib", None)
    monkeypatch.setattr(evis, "LIB_PATH", "/nonexistent/libevis.so")
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        evis.lib()


@pytest.mark.parametrize("seg,bins", [((0, 4, 0, 10), 8), ((4, 4, 10, 10), 8), ((4, 4, 0, 1 << 32), 8),
                                      ((4, 4, 0, 10), 0), ((4, 4, 0, 10), 1025), ((70000, 1, 0, 10), 8)])
def test_voxel_arguments_checked_without_a_gpu(evis, seg, bins):
    with pytest.raises(evis.EvisError):
        evis.voxel_workspace_size([seg], bins)


def test_voxel_grid_rejects_misaligned_pointers_without_a_gpu(evis):
    """Alignment is checked on the host before any CUDA call (the pointers here are never
    dereferenced): events and workspace 16 bytes, count 8, grid 4."""
    import ctypes
    segs = [(8, 8, 0, 1000)]
    arr = evis._voxel_envs(segs)
    L = evis.lib()
    ok = dict(events=0x10000, count=0x20000, ws=0x30000, grid=0x40000)
    for key, bad in (("events", 0x10008), ("count", 0x20004), ("ws", 0x30008), ("grid", 0x40002)):
        p = dict(ok, **{key: bad})
        st = L.evis_voxel_grid(p["events"], p["count"], 10, ctypes.addressof(arr), 1, 4, p["ws"],
                               1 << 30, p["grid"], None)
        assert st == evis.ERR_INVALID_ARG, key


def test_misaligned_inputs_rejected_without_a_gpu(evis):
    """Motion vectors are read as float pairs and event records as 16-byte pairs: the
    allocation-free step and the soft surrogate reject misaligned device pointers on the host,
    before any CUDA call (the fake addresses here are never dereferenced)."""
    import ctypes
    L = evis.lib()
    env = evis.EnvDesc(16, 8, 4, 0.2, 0.2, 0, None, None, 0, 0)
    b = 0x100000
    na = dict(L_A=b, mv_A=b, Z_A=b, L_B=b, mv_B=b, Z_B=b, Lref=b, t_last=b, events=b, count=b)
    for key, off in (("mv_A", 4), ("mv_B", 4), ("L_A", 2), ("t_last", 4), ("count", 4), ("events", 8)):
        p = dict(na, **{key: b + off})
        st = L.evis_step_noalloc(ctypes.byref(env), 0, p["L_A"], p["mv_A"], p["Z_A"], p["L_B"],
                                 p["mv_B"], p["Z_B"], p["Lref"], p["t_last"], 0, 1000, p["events"],
                                 p["count"], 10, None)
        assert st == evis.ERR_INVALID_ARG, key
    sf = dict(LA=b, LB=b, mvA=b, mvB=b, ZA=b, ZB=b, Lref0=b, C=b, counts=b, ws=b)
    for key, off in (("mvA", 4), ("mvB", 4), ("ZB", 2), ("ws", 8)):
        p = dict(sf, **{key: b + off})
        st = L.evis_soft_forward(ctypes.byref(env), 1, 0.02, 1e-3, p["LA"], p["LB"], p["mvA"], p["mvB"],
                                 p["ZA"], p["ZB"], p["Lref0"], p["C"], p["counts"], p["ws"], 1 << 30, None)
        assert st == evis.ERR_INVALID_ARG, key


def test_voxel_workspace_size(evis):
    """Two uint64 per region (a row segment of 32 pixels across 256 planes), one uint32 entry
    per record, two once the planes of an environment span two groups (bins > 128)."""
    segs = [(640, 480, 0, 500_000_000), (3, 2, 5, 9)]
    regions = 480 * 20 + 2 * 1
    n0 = evis.voxel_workspace_size(segs, 128)
    assert 16 * regions <= n0 < 16 * regions + 4096 + 4 * 2 * 128 * 2
    assert evis.voxel_workspace_size(segs, 128, 1_000_000) - n0 == 4 * 1_000_000
    m0 = evis.voxel_workspace_size(segs, 129)
    assert 32 * regions <= m0 < 32 * regions + 4096 + 4 * 2 * 129 * 2
    assert evis.voxel_workspace_size(segs, 129, 1_000_000) - m0 == 8 * 1_000_000


def test_state_calls_reject_a_null_context_without_a_gpu(evis):
    L = evis.lib()
    assert L.evis_set_state(None, None, None, None, None) == evis.ERR_INVALID_ARG
    assert L.evis_get_gaps(None, None) == evis.ERR_INVALID_ARG
    assert L.evis_get_stats(None, None, None, None) == evis.ERR_INVALID_ARG


def test_pipelined_readback_rejects_a_null_context_without_a_gpu(evis):
    L = evis.lib()
    n = ctypes.c_int64()
    assert L.evis_read_events_async(None, None, 0, ctypes.byref(n)) == evis.ERR_INVALID_ARG
    assert L.evis_read_wait(None) == evis.ERR_INVALID_ARG


def test_build_relinks_when_the_units_change(evis, monkeypatch, tmp_path):
    """The library counts as out of date when a translation unit is added or removed since
    its link, even when it is newer than every source (a removed unit's kernels must not
    stay in it)."""
    from paper_2607_08098_b300 import build
    assert not build._stale()                       # just built by the fixture
    real = build.sources()
    extra = tmp_path / "evis_extra.cu"
    extra.write_text("")
    monkeypatch.setattr(build, "sources", lambda: sorted(real + [str(extra)]))
    assert build._stale()                           # a unit added
    monkeypatch.setattr(build, "sources", lambda: real[:-1])
    assert build._stale()                           # a unit removed
    monkeypatch.setattr(build, "sources", lambda: real)
    assert not build._stale()
