"""Python binding of the C ABI in include/rt.h (ctypes).

Argument marshalling only: every step of the render and the cross-correlation
runs in the CUDA library.  Device buffers are torch tensors (their data
pointers are passed); the stream defaults to torch's current stream.  If the
library has not been built this module raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("GRATINGRT_LIB") or os.path.join(PKG, "libgratingrt.so")

RT_OK, RT_PENDING = 0, 1
RT_EINVAL, RT_ENOMEM, RT_ENODEV, RT_EBUSY, RT_ETIMEDOUT, RT_ECUDA = -22, -12, -19, -16, -110, -5
RT_FP32, RT_FP64 = 0, 1


class RtError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rt error {code}: {msg}")
        self.code = code


class SceneDesc(C.Structure):
    _fields_ = [
        ("Lambda", C.c_double), ("A", C.c_double), ("H", C.c_double), ("E", C.c_double),
        ("cam_dist", C.c_double), ("elev_deg", C.c_double), ("azim_deg", C.c_double), ("hfov_deg", C.c_double),
        ("bg_cell", C.c_double), ("tex_texel", C.c_double),
        ("colour0", C.c_double * 3), ("colour1", C.c_double * 3),
        ("h", C.c_double), ("rtol", C.c_double), ("atol", C.c_double), ("h_max", C.c_double),
        ("gauss_w", C.c_double),
        ("seed", C.c_uint64), ("scene_id", C.c_uint64),
        ("max_steps", C.c_int64),
        ("tex", C.POINTER(C.c_float)),
        ("mirror", C.c_int32), ("cloak", C.c_int32), ("width", C.c_int32), ("height", C.c_int32),
        ("spp", C.c_int32), ("centre_line", C.c_int32), ("background", C.c_int32), ("tex_size", C.c_int32),
        ("integrator", C.c_int32), ("precision", C.c_int32), ("max_bounces", C.c_int32), ("flags", C.c_int32),
    ]


class RayRecord(C.Structure):
    _fields_ = [
        ("pos", C.c_double * 3), ("dir", C.c_double * 3), ("rgb", C.c_float * 3),
        ("status", C.c_int32), ("bounces", C.c_int32), ("events", C.c_int32), ("steps", C.c_int64),
    ]


RECORD_DTYPE = np.dtype({
    "names": ["pos", "dir", "rgb", "status", "bounces", "events", "steps"],
    "formats": [("<f8", 3), ("<f8", 3), ("<f4", 3), "<i4", "<i4", "<i4", "<i8"],
    "offsets": [0, 24, 48, 60, 64, 68, 72],
    "itemsize": 80,
})
assert C.sizeof(RayRecord) == RECORD_DTYPE.itemsize


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("latency_ms", C.c_float), ("queue_ms", C.c_float), ("rays", C.c_uint64)]


class ServerInfo(C.Structure):
    _fields_ = [("queued", C.c_uint64), ("in_flight", C.c_uint64), ("completed", C.c_uint64),
                ("failed", C.c_uint64), ("bytes_in_use", C.c_uint64), ("budget", C.c_uint64)]


class Stats(C.Structure):
    _fields_ = [("rays", C.c_uint64), ("steps", C.c_uint64), ("evals", C.c_uint64), ("newton", C.c_uint64),
                ("events", C.c_uint64), ("fp64_refine", C.c_uint64), ("status", C.c_uint64 * 5),
                ("profile", C.c_uint64 * 4), ("sched_timeouts", C.c_uint64)]


_lib = None

EXPORTS = ["rt_create_scene", "rt_destroy_scene", "rt_render", "rt_render_pixels", "rt_render_host",
           "rt_scene_stats", "rt_scene_set_launch", "rt_scene_get_launch", "rt_scene_set_wait_limit",
           "rt_scene_autotune",
           "rt_batch_create", "rt_batch_destroy", "rt_batch_render", "rt_batch_stats", "rt_batch_set_launch",
           "rt_batch_get_launch", "rt_batch_autotune", "rt_batch_update",
           "rt_validate_desc", "rt_request_bytes", "rt_server_create", "rt_server_destroy", "rt_submit", "rt_poll",
           "rt_server_stats",
           "rt_xcorr", "rt_xcorr_noalloc", "rt_xcorr_map", "rt_eval_medium", "rt_last_error", "rt_version"]


def lib() -> C.CDLL:
    """Load libgratingrt.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    L = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    L.rt_create_scene.argtypes = [C.POINTER(SceneDesc), C.POINTER(vp)]
    L.rt_destroy_scene.argtypes = [vp]
    L.rt_destroy_scene.restype = None
    L.rt_render.argtypes = [vp, vp, vp, vp, vp]
    L.rt_render_pixels.argtypes = [vp, vp, C.c_int64, vp, vp, vp]
    L.rt_render_host.argtypes = [vp, vp, vp, vp]
    L.rt_scene_stats.argtypes = [vp, C.POINTER(Stats)]
    L.rt_scene_set_launch.argtypes = [vp, C.c_int32, C.c_int32]
    L.rt_scene_get_launch.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    L.rt_scene_set_wait_limit.argtypes = [vp, C.c_int32, C.c_int32]
    L.rt_scene_autotune.argtypes = [vp, vp, C.c_int32, vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    L.rt_batch_create.argtypes = [C.POINTER(vp), C.c_int32, C.POINTER(vp)]
    L.rt_batch_destroy.argtypes = [vp]
    L.rt_batch_destroy.restype = None
    L.rt_batch_render.argtypes = [vp, C.POINTER(vp), vp]
    L.rt_batch_stats.argtypes = [vp, C.POINTER(Stats)]
    L.rt_batch_set_launch.argtypes = [vp, C.c_int32]
    L.rt_batch_get_launch.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int64)]
    L.rt_batch_autotune.argtypes = [vp, C.POINTER(vp), C.c_int32, vp, C.POINTER(C.c_int32)]
    L.rt_batch_update.argtypes = [vp, C.POINTER(SceneDesc), C.c_int32, vp, C.POINTER(C.c_uint64)]
    L.rt_xcorr.argtypes = [vp, vp, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_double), C.c_int32,
                           C.c_double, vp, vp]
    L.rt_xcorr_noalloc.argtypes = [vp, vp, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_double), C.c_int32,
                                   C.c_double, vp, vp]
    L.rt_xcorr_map.argtypes = [C.POINTER(vp), C.POINTER(vp), C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                               C.c_double, C.c_double, C.c_int32, C.c_int32, vp, vp, vp]
    L.rt_eval_medium.argtypes = [C.c_int32, C.c_double, C.c_double, vp, C.c_int64, vp, vp]
    L.rt_validate_desc.argtypes = [C.POINTER(SceneDesc)]
    L.rt_request_bytes.argtypes = [C.POINTER(SceneDesc), C.POINTER(C.c_uint64)]
    L.rt_server_create.argtypes = [C.c_size_t, C.c_int32, C.POINTER(vp)]
    L.rt_server_destroy.argtypes = [vp]
    L.rt_server_destroy.restype = None
    L.rt_submit.argtypes = [vp, C.POINTER(SceneDesc), vp, C.POINTER(C.c_uint64)]
    L.rt_poll.argtypes = [vp, C.c_uint64, C.c_int32, C.POINTER(Result)]
    L.rt_server_stats.argtypes = [vp, C.POINTER(ServerInfo)]
    L.rt_last_error.restype = C.c_char_p
    L.rt_version.restype = C.c_char_p
    _lib = L
    return L


def _check(rc: int):
    if rc < 0:
        raise RtError(rc, lib().rt_last_error().decode())
    return rc


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t) -> int | None:
    if t is None:
        return None
    return t.data_ptr()


def make_desc(params: dict, tex: np.ndarray | None = None) -> tuple[SceneDesc, np.ndarray | None]:
    d = SceneDesc()
    for name, _ in SceneDesc._fields_:
        if name in ("tex", "colour0", "colour1"):
            continue
        if name in params:
            setattr(d, name, params[name])
    for name in ("colour0", "colour1"):
        getattr(d, name)[:] = [float(v) for v in params.get(name, (0.0, 0.0, 0.0))]
    keep = None
    if tex is not None:
        keep = np.ascontiguousarray(tex, dtype=np.float32)
        d.tex = keep.ctypes.data_as(C.POINTER(C.c_float))
        d.tex_size = int(keep.shape[0])
    return d, keep


class Scene:
    """A scene on the current CUDA device (rt_create_scene)."""

    def __init__(self, params: dict, tex: np.ndarray | None = None):
        self.params = dict(params)
        desc, _keep = make_desc(params, tex)
        h = C.c_void_p()
        _check(lib().rt_create_scene(C.byref(desc), C.byref(h)))
        self._h = h
        self.width = int(params["width"])
        self.height = int(params["height"])
        self.spp = int(params["spp"])
        self.wout = 1 if params.get("centre_line", 0) else self.width

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().rt_destroy_scene(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self) -> tuple[int, int, int]:
        return (self.height, self.wout, 3)

    def render(self, rgb, rgb8=None, rec=None, stream=None):
        """rgb: float32 (H, Wout, 3) CUDA tensor; rgb8: uint8 same shape; rec: uint8 tensor of
        H*Wout*spp*80 bytes (view with RECORD_DTYPE after copying to host)."""
        _check(lib().rt_render(self._h, _ptr(rgb), _ptr(rgb8), _ptr(rec), _stream(stream)))

    def render_pixels(self, pix, rgb, rec=None, stream=None):
        _check(lib().rt_render_pixels(self._h, _ptr(pix), int(pix.numel()), _ptr(rgb), _ptr(rec), _stream(stream)))

    def render_host(self, h_rgb: np.ndarray, h_rgb8: np.ndarray | None = None, stream=None):
        _check(lib().rt_render_host(self._h, h_rgb.ctypes.data, None if h_rgb8 is None else h_rgb8.ctypes.data,
                                    _stream(stream)))

    def set_launch(self, variant: int = -1, min_active: int = 0):
        _check(lib().rt_scene_set_launch(self._h, variant, min_active))

    def set_wait_limit(self, spin_limit: int = 0, hold_lock: bool = False):
        """rt_scene_set_wait_limit: attempts per wait of the wavefront loop's queues
        (0: the default) and, with hold_lock, make every wait of the next renders
        run out (failure-detection tests)."""
        _check(lib().rt_scene_set_wait_limit(self._h, int(spin_limit), 1 if hold_lock else 0))

    def get_launch(self) -> dict:
        v, m, g = C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib().rt_scene_get_launch(self._h, C.byref(v), C.byref(m), C.byref(g)))
        return {"variant": v.value, "min_active": m.value, "grid": g.value}

    def autotune(self, rgb, trials: int = 3, stream=None) -> dict:
        """rt_scene_autotune: time the launch configurations on this scene (rendering into rgb)."""
        v, m = C.c_int32(), C.c_int32()
        _check(lib().rt_scene_autotune(self._h, _ptr(rgb), trials, _stream(stream), C.byref(v), C.byref(m)))
        return {"variant": v.value, "min_active": m.value}

    def stats(self, check: bool = True) -> dict:
        """Counters of the last render (rt_scene_stats).  With check=False a
        render that gave up bounded waits (RT_ETIMEDOUT) still returns its
        counters, with the return code under "rc", instead of raising."""
        s = Stats()
        rc = lib().rt_scene_stats(self._h, C.byref(s))
        if check or rc not in (RT_OK, RT_ETIMEDOUT):
            _check(rc)
        return dict(_stats_dict(s), rc=rc)


def _stats_dict(s: Stats) -> dict:
    return {"rays": s.rays, "steps": s.steps, "evals": s.evals, "newton": s.newton, "events": s.events,
            "fp64_refine": s.fp64_refine, "status": list(s.status), "profile": list(s.profile),
            "sched_timeouts": s.sched_timeouts}


class Batch:
    """Several scenes rendered by one persistent launch (rt_batch_*); the scenes
    must stay alive while the batch is used."""

    def __init__(self, scenes: list):
        self.scenes = list(scenes)
        arr = (C.c_void_p * len(self.scenes))(*[sc._h.value for sc in self.scenes])
        h = C.c_void_p()
        _check(lib().rt_batch_create(arr, len(self.scenes), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().rt_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _outs(self, outs):
        assert len(outs) == len(self.scenes)
        return (C.c_void_p * len(outs))(*[_ptr(t) for t in outs])

    def render(self, outs, stream=None):
        _check(lib().rt_batch_render(self._h, self._outs(outs), _stream(stream)))

    def update(self, params: list, stream=None) -> int:
        """New parameters for every scene (rt_batch_update): the table is copied
        to the device on `stream` before the next render; returns the bytes copied."""
        assert len(params) == len(self.scenes)
        arr = (SceneDesc * len(params))()
        for q, p in enumerate(params):
            arr[q], _ = make_desc(p, None)
        b = C.c_uint64()
        _check(lib().rt_batch_update(self._h, arr, len(params), _stream(stream), C.byref(b)))
        return b.value

    def stats(self) -> dict:
        s = Stats()
        _check(lib().rt_batch_stats(self._h, C.byref(s)))
        return _stats_dict(s)

    def set_launch(self, min_active: int):
        _check(lib().rt_batch_set_launch(self._h, min_active))

    def get_launch(self) -> dict:
        m, g, t = C.c_int32(), C.c_int32(), C.c_int64()
        _check(lib().rt_batch_get_launch(self._h, C.byref(m), C.byref(g), C.byref(t)))
        return {"min_active": m.value, "grid": g.value, "pixels": t.value}

    def autotune(self, outs, trials: int = 3, stream=None) -> int:
        m = C.c_int32()
        _check(lib().rt_batch_autotune(self._h, self._outs(outs), trials, _stream(stream), C.byref(m)))
        return m.value


def records_to_numpy(rec_bytes) -> np.ndarray:
    """View a uint8 CUDA/CPU tensor of records as a numpy structured array."""
    a = rec_bytes.cpu().numpy() if hasattr(rec_bytes, "cpu") else np.asarray(rec_bytes)
    return a.view(RECORD_DTYPE)


def xcorr(f, g, fov_deg, hfov_deg: float, out=None, stream=None):
    """C(0,0) of Eqs. 14-15 per field of view: returns a float64 CUDA tensor (n_fov, C+1)."""
    import torch
    if f.dim() == 2:
        f = f.unsqueeze(-1)
        g = g.unsqueeze(-1)
    H, W, Cc = f.shape
    fov = (C.c_double * len(fov_deg))(*[float(x) for x in fov_deg])
    if out is None:
        out = torch.empty((len(fov_deg), Cc + 1), dtype=torch.float64, device=f.device)
    _check(lib().rt_xcorr(_ptr(f), _ptr(g), H, W, Cc, fov, len(fov_deg), float(hfov_deg), _ptr(out),
                          _stream(stream)))
    return out


def xcorr_map(pairs, fov_deg: float, hfov_deg: float, max_di: int, max_dj: int, out=None, peak=None,
              stream=None):
    """C(di, dj) of Eq. 15 over pixel shifts, averaged over the (f, g) image
    pairs (rt_xcorr_map): returns the float64 CUDA map (2 max_di + 1,
    2 max_dj + 1, C + 1) and the peak tensor (value, di, dj) of its stacked
    channels."""
    import torch
    fs, gs = [], []
    for f, g in pairs:
        if f.dim() == 2:
            f = f.unsqueeze(-1)
            g = g.unsqueeze(-1)
        fs.append(f)
        gs.append(g)
    H, W, Cc = fs[0].shape
    n = len(fs)
    fp = (C.c_void_p * n)(*[_ptr(t) for t in fs])
    gp = (C.c_void_p * n)(*[_ptr(t) for t in gs])
    if out is None:
        out = torch.empty((2 * max_di + 1, 2 * max_dj + 1, Cc + 1), dtype=torch.float64, device=fs[0].device)
    if peak is None:
        peak = torch.empty(3, dtype=torch.float64, device=fs[0].device)
    _check(lib().rt_xcorr_map(fp, gp, n, H, W, Cc, float(fov_deg), float(hfov_deg), int(max_di), int(max_dj),
                              _ptr(out), _ptr(peak), _stream(stream)))
    return out, peak


def xcorr_noalloc(f, g, fov_deg, hfov_deg: float, out=None, stream=None):
    """xcorr through rt_xcorr_noalloc: the same results without any device
    allocation by the library (its scratch is a fixed array; see include/rt.h)."""
    import torch
    if f.dim() == 2:
        f = f.unsqueeze(-1)
        g = g.unsqueeze(-1)
    H, W, Cc = f.shape
    fov = (C.c_double * len(fov_deg))(*[float(x) for x in fov_deg])
    if out is None:
        out = torch.empty((len(fov_deg), Cc + 1), dtype=torch.float64, device=f.device)
    _check(lib().rt_xcorr_noalloc(_ptr(f), _ptr(g), H, W, Cc, fov, len(fov_deg), float(hfov_deg), _ptr(out),
                                  _stream(stream)))
    return out


def eval_medium(precision: int, Lambda: float, A: float, xy, out=None, stream=None):
    """(Re W0, Im W0, n, F_x, F_y) at the points xy (float64 CUDA tensor (n, 2))."""
    import torch
    n = xy.shape[0]
    if out is None:
        out = torch.empty((n, 5), dtype=torch.float64, device=xy.device)
    _check(lib().rt_eval_medium(precision, float(Lambda), float(A), _ptr(xy), n, _ptr(out), _stream(stream)))
    return out


def version() -> str:
    return lib().rt_version().decode()


def validate(params: dict, tex: np.ndarray | None = None) -> None:
    """rt_validate_desc: raise RtError for an invalid scene descriptor (host only)."""
    desc, _keep = make_desc(params, tex)
    _check(lib().rt_validate_desc(C.byref(desc)))


def request_bytes(params: dict) -> int:
    """Ray-state footprint of a request in a server's budget (rt_request_bytes)."""
    desc, _keep = make_desc(params, None)
    b = C.c_uint64()
    _check(lib().rt_request_bytes(C.byref(desc), C.byref(b)))
    return b.value


class Server:
    """Render server with continuous batching (rt_server_*, rt_submit, rt_poll)."""

    def __init__(self, budget_bytes: int, max_inflight: int = 2):
        h = C.c_void_p()
        _check(lib().rt_server_create(int(budget_bytes), int(max_inflight), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().rt_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, params: dict, out, tex: np.ndarray | None = None) -> int:
        desc, _keep = make_desc(params, tex)
        t = C.c_uint64()
        _check(lib().rt_submit(self._h, C.byref(desc), _ptr(out), C.byref(t)))
        return t.value

    def poll(self, ticket: int, timeout_us: int = 0):
        """The result dict when done; None while pending."""
        r = Result()
        rc = lib().rt_poll(self._h, ticket, int(timeout_us), C.byref(r))
        if rc in (RT_PENDING, RT_ETIMEDOUT):
            return None
        _check(rc)
        return {"status": r.status, "latency_ms": r.latency_ms, "queue_ms": r.queue_ms, "rays": r.rays}

    def stats(self) -> dict:
        i = ServerInfo()
        _check(lib().rt_server_stats(self._h, C.byref(i)))
        return {k: getattr(i, k) for k, _ in ServerInfo._fields_}
