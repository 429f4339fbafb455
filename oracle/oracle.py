"""ctypes wrapper around the FP64 CPU oracle (oracle.c).

Test infrastructure: only the test suite, the package smoke check and the
CPU-baseline leg of bench.py use this module.  It imports nothing from the
product package; scenes arrive as plain dictionaries (see
``paper_1012_5107_gb300.inputs``) and arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, -O2, OpenMP)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


class OrScene(C.Structure):
    _fields_ = [
        ("Lambda", C.c_double), ("A", C.c_double),
        ("H", C.c_double), ("E", C.c_double),
        ("cam_dist", C.c_double), ("elev_deg", C.c_double), ("azim_deg", C.c_double), ("hfov_deg", C.c_double),
        ("bg_cell", C.c_double), ("tex_texel", C.c_double),
        ("colour0", C.c_double * 3), ("colour1", C.c_double * 3),
        ("h", C.c_double), ("rtol", C.c_double), ("atol", C.c_double), ("h_max", C.c_double),
        ("gauss_w", C.c_double),
        ("seed", C.c_uint64), ("scene_id", C.c_uint64),
        ("max_steps", C.c_int64),
        ("tex", C.POINTER(C.c_float)),
        ("mirror", C.c_int32), ("cloak", C.c_int32),
        ("width", C.c_int32), ("height", C.c_int32), ("spp", C.c_int32), ("centre_line", C.c_int32),
        ("background", C.c_int32),
        ("tex_size", C.c_int32), ("integrator", C.c_int32),
        ("max_bounces", C.c_int32), ("flags", C.c_int32),
    ]


class OrRecord(C.Structure):
    _fields_ = [
        ("pos", C.c_double * 3), ("dir", C.c_double * 3), ("rgb", C.c_double * 3),
        ("steps", C.c_int64), ("halley", C.c_int64), ("evals", C.c_int64),
        ("bounces", C.c_int32), ("status", C.c_int32), ("events", C.c_int32), ("pad", C.c_int32),
    ]


RECORD_DTYPE = np.dtype([
    ("pos", "<f8", 3), ("dir", "<f8", 3), ("rgb", "<f8", 3),
    ("steps", "<i8"), ("halley", "<i8"), ("evals", "<i8"),
    ("bounces", "<i4"), ("status", "<i4"), ("events", "<i4"), ("pad", "<i4"),
])
assert RECORD_DTYPE.itemsize == C.sizeof(OrRecord)

_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        dp = C.POINTER(C.c_double)
        L.or_lambertw0.argtypes = [dp, C.c_int64, dp, C.POINTER(C.c_int32)]
        L.or_index.argtypes = [C.POINTER(OrScene), dp, C.c_int64, dp]
        L.or_trochoid.argtypes = [C.POINTER(OrScene), dp, C.c_int64, dp]
        L.or_integrate_fixed.argtypes = [C.POINTER(OrScene), dp, C.c_double, C.c_int64, C.c_int32, dp]
        L.or_camera_dir.argtypes = [C.POINTER(OrScene), C.c_int32, C.c_int32, C.c_int32, dp, dp]
        L.or_splitmix64_out.argtypes = [C.c_uint64, C.c_uint64]
        L.or_splitmix64_out.restype = C.c_uint64
        L.or_trace_from.argtypes = [C.POINTER(OrScene), dp, dp, C.c_int32, C.c_int32, C.c_void_p, dp,
                                    C.c_int32, C.POINTER(C.c_int32)]
        L.or_render_pixels.argtypes = [C.POINTER(OrScene), C.POINTER(C.c_int64), C.c_int64,
                                       C.POINTER(C.c_float), C.c_void_p, C.c_int32]
        L.or_render.argtypes = [C.POINTER(OrScene), C.POINTER(C.c_float), C.c_void_p, C.c_int32]
        L.or_quantize.argtypes = [C.POINTER(C.c_float), C.c_int64, C.POINTER(C.c_uint8)]
        L.or_xcorr.argtypes = [C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_int32, C.c_int32, C.c_int32,
                               C.c_int32, C.c_int32, dp]
        L.or_xcorr_map.argtypes = [C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_int32, C.c_int32, C.c_int32,
                                   C.c_int32, C.c_int32, C.c_int32, C.c_int32, dp]
        L.or_fov_columns.argtypes = [C.c_int32, C.c_double, C.c_double, C.POINTER(C.c_int32),
                                     C.POINTER(C.c_int32)]
        L.or_max_threads.restype = C.c_int
        L.or_fresnel.argtypes = [C.c_double, C.c_double, C.c_double]
        L.or_fresnel.restype = C.c_double
        L.or_trace_paths.argtypes = [C.POINTER(OrScene), dp, dp, C.c_int32, C.c_int32, C.c_void_p, dp, C.c_int32,
                                     C.POINTER(C.c_int32)]
        L.or_faddeeva_eval.argtypes = [dp, C.c_int64, dp]
        L.or_gauss_map.argtypes = [C.POINTER(OrScene), dp, C.c_int64, dp]
        L.or_surface.argtypes = [C.POINTER(OrScene), dp, C.c_int64, dp]
        L.or_surface_line_hit.argtypes = [C.POINTER(OrScene), dp, dp, C.c_int32]
        L.or_surface_line_hit.restype = C.c_double
        L.or_init()                   # coefficient table of the Faddeeva function
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Scene:
    """An oracle scene built from a plain parameter dictionary.  Keeps the
    texture array alive for as long as the scene is used."""

    def __init__(self, params: dict, tex: np.ndarray | None = None):
        s = OrScene()
        for name, _ in OrScene._fields_:
            if name in ("tex", "colour0", "colour1"):
                continue
            if name in params:
                setattr(s, name, params[name])
        for name in ("colour0", "colour1"):
            v = params.get(name, (0.0, 0.0, 0.0))
            getattr(s, name)[:] = [float(x) for x in v]
        self._tex = None
        if tex is not None:
            self._tex = np.ascontiguousarray(tex, dtype=np.float32)
            s.tex = self._tex.ctypes.data_as(C.POINTER(C.c_float))
            s.tex_size = int(self._tex.shape[0])
        self.c = s
        self.params = dict(params)

    @property
    def ref(self):
        return C.byref(self.c)

    @property
    def out_width(self) -> int:
        return 1 if self.c.centre_line else self.c.width


def lambertw0(z) -> tuple[np.ndarray, np.ndarray]:
    z = np.ascontiguousarray(np.atleast_1d(np.asarray(z, dtype=np.complex128)))
    zz = np.ascontiguousarray(np.stack([z.real, z.imag], -1).reshape(-1))
    out = np.zeros_like(zz)
    it = np.zeros(z.size, dtype=np.int32)
    lib().or_lambertw0(_dp(zz), z.size, _dp(out), it.ctypes.data_as(C.POINTER(C.c_int32)))
    return out[0::2] + 1j * out[1::2], it


def index(sc: Scene, x, y) -> np.ndarray:
    """Rows (Re W, Im W, n, dn/dx, dn/dy, dn/dz) at the points (x, y): W = W0
    for the grating cloak, the virtual coordinate w for the Gaussian cloak."""
    x, y = np.broadcast_arrays(np.asarray(x, float), np.asarray(y, float))
    xy = np.ascontiguousarray(np.stack([x.ravel(), y.ravel()], -1).reshape(-1))
    out = np.zeros((x.size, 6))
    lib().or_index(sc.ref, _dp(xy), x.size, _dp(out))
    return out.reshape(x.shape + (6,))


def trochoid(sc: Scene, x) -> np.ndarray:
    """Rows (xi, y_s, N_x, N_y) of the grating at abscissae x (Eq. 2)."""
    x = np.ascontiguousarray(np.atleast_1d(np.asarray(x, float)))
    out = np.zeros((x.size, 4))
    lib().or_trochoid(sc.ref, _dp(x), x.size, _dp(out))
    return out


def integrate_fixed(sc: Scene, s0, h: float, nsteps: int, method: int = 0) -> np.ndarray:
    s0 = np.ascontiguousarray(np.asarray(s0, float))
    out = np.zeros((nsteps, 6))
    lib().or_integrate_fixed(sc.ref, _dp(s0), h, nsteps, method, _dp(out))
    return out


def camera_dir(sc: Scene, i: int, j: int, s: int):
    o = np.zeros(3)
    d = np.zeros(3)
    lib().or_camera_dir(sc.ref, i, j, s, _dp(o), _dp(d))
    return o, d


def splitmix64(seed: int, m: int) -> int:
    return int(lib().or_splitmix64_out(seed, m))


def trace_from(sc: Scene, X, p, medium: int = 0, surface: int = -1, traj_cap: int = 0):
    X = np.ascontiguousarray(np.asarray(X, float))
    p = np.ascontiguousarray(np.asarray(p, float))
    rec = np.zeros(1, dtype=RECORD_DTYPE)
    traj = np.zeros((max(traj_cap, 1), 6))
    n = C.c_int32(0)
    if lib().or_trace_from(sc.ref, _dp(X), _dp(p), medium, surface, rec.ctypes.data,
                           _dp(traj) if traj_cap else None, traj_cap, C.byref(n)):
        raise ValueError("oracle: texture background without a texture")
    return rec[0], traj[: n.value]


FLAG_REFERENCED, FLAG_PLATE, FLAG_FRESNEL = 1, 2, 4


def fresnel(n1: float, n2: float, cos_i: float) -> float:
    """Unpolarised Fresnel reflectance from index n1 into n2 at incidence cosine cos_i."""
    return float(lib().or_fresnel(n1, n2, cos_i))


def trace_paths(sc: Scene, X, p, medium: int = 0, surface: int = -1, cap: int = 9):
    """Records and weights of every path of one sample: the first path, then
    its Fresnel branches in the order they were started."""
    X = np.ascontiguousarray(np.asarray(X, float))
    p = np.ascontiguousarray(np.asarray(p, float))
    rec = np.zeros(cap, dtype=RECORD_DTYPE)
    w = np.zeros(cap)
    n = C.c_int32(0)
    if lib().or_trace_paths(sc.ref, _dp(X), _dp(p), medium, surface, rec.ctypes.data, _dp(w), cap, C.byref(n)):
        raise ValueError("oracle: invalid scene")
    return rec[: n.value], w[: n.value]


def render_pixels(sc: Scene, pix, nthreads: int = 0, records: bool = False):
    pix = np.ascontiguousarray(np.asarray(pix, dtype=np.int64))
    rgb = np.zeros((pix.size, 3), dtype=np.float32)
    rec = np.zeros(pix.size * sc.c.spp, dtype=RECORD_DTYPE) if records else None
    if lib().or_render_pixels(sc.ref, pix.ctypes.data_as(C.POINTER(C.c_int64)), pix.size,
                              rgb.ctypes.data_as(C.POINTER(C.c_float)),
                              rec.ctypes.data if records else None, nthreads):
        raise ValueError("oracle: invalid scene (texture background without a texture, or a plate "
                         "without the flat mirror alone)")
    return (rgb, rec) if records else rgb


def render(sc: Scene, nthreads: int = 0, records: bool = False):
    H, W = sc.c.height, sc.out_width
    out = render_pixels(sc, np.arange(H * W), nthreads, records)
    if records:
        rgb, rec = out
        return rgb.reshape(H, W, 3), rec.reshape(H, W, sc.c.spp)
    return out.reshape(H, W, 3)


def quantize(c) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(c, dtype=np.float32))
    q = np.zeros(c.shape, dtype=np.uint8)
    lib().or_quantize(c.ctypes.data_as(C.POINTER(C.c_float)), c.size, q.ctypes.data_as(C.POINTER(C.c_uint8)))
    return q


def fov_columns(W: int, hfov_deg: float, fov_deg: float) -> tuple[int, int]:
    j0, j1 = C.c_int32(0), C.c_int32(0)
    lib().or_fov_columns(W, hfov_deg, fov_deg, C.byref(j0), C.byref(j1))
    return j0.value, j1.value


def xcorr(f, g, j0: int, j1: int) -> np.ndarray:
    """C(0,0) (Eqs. 14-15) per channel and for the stacked channels, over columns j0..j1-1."""
    f = np.ascontiguousarray(np.asarray(f, dtype=np.float32))
    g = np.ascontiguousarray(np.asarray(g, dtype=np.float32))
    if f.ndim == 2:
        f = f[..., None]
        g = g[..., None]
    H, W, Cc = f.shape
    out = np.zeros(Cc + 1)
    lib().or_xcorr(f.ctypes.data_as(C.POINTER(C.c_float)), g.ctypes.data_as(C.POINTER(C.c_float)),
                   H, W, Cc, j0, j1, _dp(out))
    return out


def xcorr_map(f, g, j0: int, j1: int, max_di: int, max_dj: int) -> np.ndarray:
    """C(di, dj) of Eq. 15 for |di| <= max_di, |dj| <= max_dj over columns j0..j1-1:
    array (2 max_di + 1, 2 max_dj + 1, channels + 1), the last entry the stacked channels."""
    f = np.ascontiguousarray(np.asarray(f, dtype=np.float32))
    g = np.ascontiguousarray(np.asarray(g, dtype=np.float32))
    if f.ndim == 2:
        f = f[..., None]
        g = g[..., None]
    H, W, Cc = f.shape
    out = np.zeros((2 * max_di + 1, 2 * max_dj + 1, Cc + 1))
    if lib().or_xcorr_map(f.ctypes.data_as(C.POINTER(C.c_float)), g.ctypes.data_as(C.POINTER(C.c_float)),
                          H, W, Cc, j0, j1, max_di, max_dj, _dp(out)):
        raise MemoryError("oracle: allocation failed")
    return out


def max_threads() -> int:
    return int(lib().or_max_threads())


if __name__ == "__main__":  # pragma: no cover
    build(force="--force" in sys.argv)
    print(LIB)


def faddeeva(s) -> np.ndarray:
    """The oracle's Faddeeva function F(s) = exp(-s^2) erfc(-i s)."""
    s = np.asarray(s, dtype=np.complex128)
    ss = np.ascontiguousarray(np.stack([s.real.ravel(), s.imag.ravel()], -1).reshape(-1))
    out = np.zeros_like(ss)
    lib().or_faddeeva_eval(_dp(ss), s.size, _dp(out))
    return (out[0::2] + 1j * out[1::2]).reshape(s.shape)


def gauss_map(sc: Scene, w) -> tuple[np.ndarray, np.ndarray]:
    """z(w) and z'(w) of the Gaussian conformal map at virtual points w."""
    w = np.asarray(w, dtype=np.complex128)
    ww = np.ascontiguousarray(np.stack([w.real.ravel(), w.imag.ravel()], -1).reshape(-1))
    out = np.zeros(4 * w.size)
    lib().or_gauss_map(sc.ref, _dp(ww), w.size, _dp(out))
    out = out.reshape(-1, 4)
    return (out[:, 0] + 1j * out[:, 1]).reshape(w.shape), (out[:, 2] + 1j * out[:, 3]).reshape(w.shape)


def surface(sc: Scene, x) -> np.ndarray:
    """Rows (y_s, dy_s/dx, N_x, N_y) of the mirror surface (trochoid or bump) at abscissae x."""
    x = np.ascontiguousarray(np.atleast_1d(np.asarray(x, float)))
    out = np.zeros((x.size, 4))
    lib().or_surface(sc.ref, _dp(x), x.size, _dp(out))
    return out


def surface_line_hit(sc: Scene, X, p, on_surface: bool = False) -> float:
    """First t > 0 at which X + t p meets the mirror surface (inf if none)."""
    X = np.ascontiguousarray(np.asarray(X, float))
    p = np.ascontiguousarray(np.asarray(p, float))
    return float(lib().or_surface_line_hit(sc.ref, _dp(X), _dp(p), int(on_surface)))
