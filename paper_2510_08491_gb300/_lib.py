"""ctypes binding of libsnp (include/snp.h): argument marshalling only.

Every stage of the renderer runs in the CUDA library; this module converts
Python objects to the C structs and raw device pointers.  Importing it does not
touch the GPU; loading fails loudly when libsnp.so has not been built.
"""
from __future__ import annotations

import ctypes as C
import os
import re

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsnp.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "snp.h")

SNP_OK, SNP_ERR_INVALID_ARG, SNP_ERR_CUDA, SNP_ERR_CAPACITY, SNP_ERR_TIMEOUT, SNP_ERR_UNSUPPORTED = range(6)
STATUS_NAMES = {0: "SNP_OK", 1: "SNP_ERR_INVALID_ARG", 2: "SNP_ERR_CUDA", 3: "SNP_ERR_CAPACITY",
                4: "SNP_ERR_TIMEOUT", 5: "SNP_ERR_UNSUPPORTED"}
COLOR_CONST, COLOR_MLP, COLOR_SH = 0, 1, 2
F32, BF16 = 0, 1
FORM_STABLE, FORM_NAIVE = 0, 1
FEAT_DIM = 8
GEOM_STRIDE = 16


class SnpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Camera(C.Structure):
    _fields_ = [("R_wc", C.c_float * 9), ("eye", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("z_near", C.c_float), ("width", C.c_int32),
                ("height", C.c_int32), ("time", C.c_float)]


class SceneDesc(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_sigma", C.c_int32), ("color_mode", C.c_int32), ("n_c", C.c_int32),
                ("weight_dtype", C.c_int32), ("omega0", C.c_float), ("dynamic", C.c_int32)]


class NetLayout(C.Structure):
    _fields_ = [("off", C.c_int32 * 14), ("stride", C.c_int32)]


class ScenePtrs(C.Structure):
    _fields_ = [("geom", C.c_void_p), ("net", C.c_void_p)]


class GradPtrs(C.Structure):
    _fields_ = [("geom", C.c_void_p), ("net", C.c_void_p)]


class Config(C.Structure):
    _fields_ = [("tile_size", C.c_int32), ("chunk", C.c_int32), ("integral_form", C.c_int32),
                ("t_min", C.c_float), ("bg", C.c_float * 3), ("flags", C.c_int32), ("bwd_chunk", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("n_keys", C.c_int64), ("n_tiles", C.c_int64), ("n_pixels", C.c_int64),
                ("n_candidates", C.c_int64), ("n_hits", C.c_int64), ("n_composited", C.c_int64),
                ("fwd_ctas_per_sm", C.c_int32), ("bwd_ctas_per_sm", C.c_int32)]


class PopctlConfig(C.Structure):
    _fields_ = [("grad_threshold", C.c_float), ("prune_threshold", C.c_float), ("grow_scale", C.c_float),
                ("prune_scale", C.c_float), ("extent", C.c_float), ("reserved_", C.c_int32)]


class AdamConfig(C.Structure):
    _fields_ = [("lr_geom", C.c_float * 4), ("lr_net", C.c_float * 14), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("step", C.c_int32)]


POP_PRUNE, POP_KEEP, POP_CLONE, POP_SPLIT = 0, 1, 2, 3

_lib = None

_SIGS = {
    "snp_get_net_layout": [C.POINTER(SceneDesc), C.POINTER(NetLayout)],
    "snp_default_chunks": [C.POINTER(SceneDesc), C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)],
    "snp_create": [C.c_int32, C.POINTER(C.c_void_p)],
    "snp_destroy": [C.c_void_p],
    "snp_last_error": [C.c_void_p],
    "snp_reserve": [C.c_void_p, C.POINTER(SceneDesc), C.POINTER(Camera), C.c_int32, C.POINTER(Config), C.c_int64],
    "snp_render_forward": [C.c_void_p, C.POINTER(SceneDesc), C.POINTER(ScenePtrs), C.POINTER(Camera), C.c_int32,
                           C.POINTER(Config), C.c_void_p, C.POINTER(C.c_int64), C.c_void_p],
    "snp_render_backward": [C.c_void_p, C.c_int64, C.POINTER(SceneDesc), C.POINTER(ScenePtrs), C.c_void_p,
                            C.POINTER(GradPtrs), C.c_void_p],
    "snp_get_stats": [C.c_void_p, C.c_int64, C.POINTER(Stats), C.c_void_p],
    "snp_debug_keys": [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64),
                       C.c_void_p],
    "snp_stage_times": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32],
    "snp_autotune": [C.c_void_p, C.POINTER(SceneDesc), C.POINTER(ScenePtrs), C.POINTER(Camera), C.c_int32,
                     C.POINTER(Config), C.c_int32, C.POINTER(Config), C.POINTER(C.c_float), C.c_void_p],
    "snp_mse_loss": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p],
    "snp_popctl_accumulate": [C.c_void_p, C.POINTER(SceneDesc), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "snp_popctl_plan": [C.c_void_p, C.POINTER(SceneDesc), C.c_void_p, C.c_void_p, C.c_void_p,
                        C.POINTER(PopctlConfig), C.c_void_p, C.c_void_p, C.POINTER(C.c_int64), C.c_void_p],
    "snp_popctl_apply": [C.c_void_p, C.POINTER(SceneDesc), C.POINTER(ScenePtrs), C.c_void_p, C.c_void_p,
                         C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "snp_geom_reg": [C.c_void_p, C.POINTER(SceneDesc), C.c_void_p, C.c_float, C.c_void_p, C.c_void_p, C.c_void_p],
    "snp_adam_step": [C.c_void_p, C.POINTER(SceneDesc), C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(GradPtrs),
                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(AdamConfig), C.c_void_p],
}
FLAG_STAGE_TIMING = 1
FLAG_LENGTH_QUEUE = 2
FLAG_REPLAY_COLOR = 4
STAGES = ("project", "scan", "emit", "sort", "ranges", "raster_fwd", "raster_bwd", "post_bwd")


def header_symbols():
    """Names of the functions declared in include/snp.h."""
    txt = open(HEADER).read()
    pat = r"^\s*(?:snp_status|void|int64_t|const char \*)\s*(snp_\w+)\s*\("
    return sorted(set(re.findall(pat, txt, re.M)))


def lib():
    """Load libsnp.so (built by paper_2510_08491_gb300.build); raise if missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libsnp.so is not built ({LIB_PATH}); run paper_2510_08491_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int32
        L.snp_destroy.restype = None
        L.snp_last_error.restype = C.c_char_p
        L.snp_kernel_launches.argtypes = []
        L.snp_kernel_launches.restype = C.c_int64
        _lib = L
    return _lib


def net_layout(n_sigma: int, color_mode: int, n_c: int, dynamic: bool = False):
    d = SceneDesc(0, n_sigma, color_mode, n_c if color_mode == COLOR_MLP else 0, F32, 1.0, int(bool(dynamic)))
    L = NetLayout()
    st = lib().snp_get_net_layout(C.byref(d), C.byref(L))
    if st != SNP_OK:
        raise SnpError(st, "bad scene description")
    return list(L.off), L.stride


def default_chunks(n_sigma: int, color_mode: int, n_c: int, tile_size: int = 16, dynamic: bool = False):
    """(forward chunk, backward chunk) the library picks for this scene shape (snp_default_chunks)."""
    d = SceneDesc(0, n_sigma, color_mode, n_c if color_mode == COLOR_MLP else 0, F32, 1.0, int(bool(dynamic)))
    f, b = C.c_int32(), C.c_int32()
    st = lib().snp_default_chunks(C.byref(d), int(tile_size), C.byref(f), C.byref(b))
    if st != SNP_OK:
        raise SnpError(st, "bad scene description or tile size")
    return f.value, b.value


def make_camera(cam) -> Camera:
    c = Camera()
    c.R_wc[:] = [float(v) for v in cam.R_wc.reshape(-1)]
    c.eye[:] = [float(v) for v in cam.eye]
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.z_near = float(cam.z_near)
    c.width, c.height = int(cam.width), int(cam.height)
    c.time = float(getattr(cam, "time", 0.0))
    return c


def make_cameras(cams):
    arr = (Camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i] = make_camera(c)
    return arr


def make_config(tile_size=16, chunk=0, form=FORM_STABLE, t_min=1e-4, bg=(0.0, 0.0, 0.0), timing=False,
                length_queue=False, replay_color=False, bwd_chunk=0) -> Config:
    cfg = Config()
    cfg.tile_size, cfg.chunk, cfg.integral_form = int(tile_size), int(chunk), int(form)
    cfg.bwd_chunk = int(bwd_chunk)
    cfg.flags = (FLAG_STAGE_TIMING if timing else 0) | (FLAG_LENGTH_QUEUE if length_queue else 0) | \
        (FLAG_REPLAY_COLOR if replay_color else 0)
    cfg.t_min = float(t_min)
    cfg.bg[:] = [float(b) for b in bg]
    return cfg


class Context:
    """Owns one snp_context (one CUDA device)."""

    def __init__(self, device: int = 0):
        self._p = C.c_void_p()
        st = lib().snp_create(int(device), C.byref(self._p))
        if st != SNP_OK:
            raise SnpError(st, f"snp_create(device={device}) failed")

    @property
    def handle(self):
        return self._p

    def check(self, st: int):
        if st != SNP_OK:
            raise SnpError(st, lib().snp_last_error(self._p).decode())

    def stage_times(self, reset: bool = True):
        import numpy as np
        ms = np.zeros(len(STAGES), np.float64)
        calls = np.zeros(len(STAGES), np.int64)
        self.check(lib().snp_stage_times(self._p, ms.ctypes.data_as(C.c_void_p), calls.ctypes.data_as(C.c_void_p),
                                         1 if reset else 0))
        return {k: (float(ms[i]), int(calls[i])) for i, k in enumerate(STAGES)}

    def close(self):
        if self._p:
            lib().snp_destroy(self._p)
            self._p = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kernel_launches() -> int:
    """Kernels libsnp has launched in this process."""
    return int(lib().snp_kernel_launches())
