"""ctypes front end of the C oracle (snp_oracle.c) plus its tile lists.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

What lives here:
  * build()/lib(): compile snp_oracle.c with gcc (-O2 -fopenmp -ffp-contract=off).
  * key_project(): the FP32 key specification per camera (visible, pixel rect, depth).
  * tile_keys(): emission of (tile << 32 | depth bits, record index) in
    (view, primitive, tile row, tile column) order followed by a stable sort --
    the "primitive sorting/tiling" stage of App. A; ties in tile and depth keep
    emission order, i.e. ascending primitive index.
  * render(): the FP64 renderer of Sec. 3.2 / Eq. 4 over tile lists (tiled) or
    over all visible primitives (brute force, no tiling).
  * mse_loss(): the squared-error image loss of the differentiation workload.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "snp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libsnp_oracle.so")

FORM_STABLE, FORM_NAIVE = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-Wall", "-Wno-unknown-pragmas", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Geom32(C.Structure):
    _fields_ = [("n", C.c_int64), ("centers", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p)]


class _Scene(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_sigma", C.c_int32), ("color_mode", C.c_int32),
                ("n_c", C.c_int32), ("pad_", C.c_int32), ("omega0", C.c_double)] + \
               [(f, C.c_void_p) for f in ("centers", "log_scales", "quats", "W1", "b1", "w2", "b2",
                                          "rgb", "feat", "Wc1", "bc1", "Wc2", "bc2", "Wc3", "bc3", "sh")] + \
               [("time", C.c_double), ("wt", C.c_void_p), ("sh_t", C.c_void_p)]


class _Camera(C.Structure):
    _fields_ = [("R_wc", C.c_float * 9), ("eye", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("z_near", C.c_float), ("width", C.c_int32),
                ("height", C.c_int32), ("time", C.c_float)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.POINTER
        L.ora_key_project.argtypes = [P(_Geom32), P(_Camera), C.c_void_p, C.c_void_p, C.c_void_p]
        L.ora_key_exp.argtypes = [C.c_float]
        L.ora_key_exp.restype = C.c_float
        L.ora_render.argtypes = [P(_Scene), P(_Camera), C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_double, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p]
        L.ora_render.restype = C.c_int64
        L.ora_pair.argtypes = [P(_Scene), C.c_int64, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]
        L.ora_integral.argtypes = [P(_Scene), C.c_int64, C.c_void_p, C.c_void_p, C.c_double, C.c_double,
                                   C.c_int32]
        L.ora_integral.restype = C.c_double
        L.ora_color.argtypes = [P(_Scene), C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
        L.ora_sh_basis.argtypes = [C.c_void_p, C.c_void_p]
        L.ora_pixel_ray.argtypes = [P(_Camera), C.c_int32, C.c_int32, C.c_void_p]
        _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class CScene:
    """float64 copies of the scene arrays (exact for float32 inputs) for the FP64
    renderer, plus the float32 geometry for the key specification."""

    def __init__(self, scene):
        self.keep = {}
        s = _Scene()
        s.n = scene.n
        s.n_sigma = scene.n_sigma
        s.color_mode = {"const": 0, "mlp": 1, "sh": 2}[scene.color]
        s.n_c = scene.n_c if scene.color == "mlp" else 0
        s.omega0 = float(scene.omega0)
        for f in ("centers", "log_scales", "quats", "W1", "b1", "w2", "b2", "rgb", "feat", "Wc1", "bc1",
                  "Wc2", "bc2", "Wc3", "bc3", "sh", "wt", "sh_t"):
            a = getattr(scene, f, None)
            if a is not None:
                a = np.ascontiguousarray(a, dtype=np.float64)
                self.keep[f] = a
                setattr(s, f, a.ctypes.data)
        self.s = s
        g = _Geom32()
        g.n = scene.n
        for f in ("centers", "log_scales", "quats"):
            a = np.ascontiguousarray(getattr(scene, f), dtype=np.float32)
            self.keep[f + "32"] = a
            setattr(g, f, a.ctypes.data)
        self.g = g

    def ref(self, time: float = 0.0):
        """The C scene; `time` is the timestamp xi_t used by the single-pair calls
        (pair, integral, color) of a dynamic scene (renders take the camera's)."""
        self.s.time = float(time)
        return C.byref(self.s)

    def gref(self):
        return C.byref(self.g)


def c_camera(cam) -> _Camera:
    c = _Camera()
    c.R_wc[:] = [float(v) for v in np.asarray(cam.R_wc, dtype=np.float32).reshape(-1)]
    c.eye[:] = [float(v) for v in np.asarray(cam.eye, dtype=np.float32)]
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.z_near = float(cam.z_near)
    c.width, c.height = int(cam.width), int(cam.height)
    c.time = float(getattr(cam, "time", 0.0))
    return c


# ----------------------------------------------------------------------------- keys


@dataclass
class KeyRecords:
    visible: np.ndarray  # int32 [n]
    rect: np.ndarray  # int32 [n, 4]  px0, py0, px1, py1 (inclusive)
    depth: np.ndarray  # float32 [n]


def key_project(scene, cam, cs: Optional[CScene] = None) -> KeyRecords:
    cs = cs or CScene(scene)
    n = scene.n
    vis = np.zeros(n, np.int32)
    rect = np.zeros((n, 4), np.int32)
    depth = np.zeros(n, np.float32)
    cc = c_camera(cam)
    lib().ora_key_project(cs.gref(), C.byref(cc), _ptr(vis), _ptr(rect), _ptr(depth))
    return KeyRecords(vis, rect, depth)


def key_exp(x: float) -> np.float32:
    return np.float32(lib().ora_key_exp(float(np.float32(x))))


def tiles_xy(cam, ts: int):
    return (cam.width + ts - 1) // ts, (cam.height + ts - 1) // ts


@dataclass
class TileLists:
    keys: np.ndarray  # uint64 [K] sorted
    vals: np.ndarray  # uint32 [K] record index v * n + i
    tile_off: np.ndarray  # int64 [T_total + 1]
    view_tile_off: np.ndarray  # int64 [V + 1]
    records: List[KeyRecords]


def emission_keys(scene, cams: Sequence, ts: int, cs: Optional[CScene] = None):
    """Tile keys and values in emission order (view, primitive, tile row, tile column),
    before sorting; also returns the per-view key records and view tile offsets."""
    cs = cs or CScene(scene)
    n = scene.n
    keys_all, vals_all, recs = [], [], []
    vto = [0]
    for v, cam in enumerate(cams):
        r = key_project(scene, cam, cs)
        recs.append(r)
        tx_n, ty_n = tiles_xy(cam, ts)
        idx = np.nonzero(r.visible)[0]
        tx0 = r.rect[idx, 0] // ts
        ty0 = r.rect[idx, 1] // ts
        tx1 = r.rect[idx, 2] // ts
        ty1 = r.rect[idx, 3] // ts
        w = (tx1 - tx0 + 1).astype(np.int64)
        cnt = w * (ty1 - ty0 + 1)
        tot = int(cnt.sum())
        owner = np.repeat(np.arange(len(idx)), cnt)
        start = np.concatenate([[0], np.cumsum(cnt)[:-1]])
        j = np.arange(tot, dtype=np.int64) - np.repeat(start, cnt)
        ty = ty0[owner] + j // w[owner]
        tx = tx0[owner] + j % w[owner]
        gt = vto[-1] + ty * tx_n + tx
        dbits = r.depth.view(np.uint32)[idx][owner].astype(np.uint64)
        keys_all.append((gt.astype(np.uint64) << np.uint64(32)) | dbits)
        vals_all.append((v * n + idx[owner]).astype(np.uint32))
        vto.append(vto[-1] + tx_n * ty_n)
    keys = np.concatenate(keys_all) if keys_all else np.zeros(0, np.uint64)
    vals = np.concatenate(vals_all) if vals_all else np.zeros(0, np.uint32)
    return keys, vals, recs, vto


def tile_keys(scene, cams: Sequence, ts: int, cs: Optional[CScene] = None) -> TileLists:
    keys, vals, recs, vto = emission_keys(scene, cams, ts, cs)
    order = np.argsort(keys, kind="stable")
    keys = keys[order]
    vals = vals[order]
    t_total = vto[-1]
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    tile_off = np.searchsorted(tiles, np.arange(t_total + 1), side="left").astype(np.int64)
    return TileLists(keys, vals, tile_off, np.asarray(vto, np.int64), recs)


def brute_force_list(rec: KeyRecords) -> np.ndarray:
    """All visible primitives of one view in compositing order (depth key, then index)."""
    idx = np.nonzero(rec.visible)[0]
    order = np.argsort(rec.depth.view(np.uint32)[idx], kind="stable")
    return idx[order].astype(np.int32)


# ----------------------------------------------------------------------------- render


@dataclass
class RenderOut:
    rgb: np.ndarray  # float64 [P, 3]
    tau: np.ndarray  # float64 [P]
    n_walk: np.ndarray  # int32 [P]
    flags: np.ndarray  # int32 [P]
    n_comp: int


def render_pixels(scene, cam, pix: np.ndarray, pix_list: np.ndarray, list_off: np.ndarray,
                  list_prim: np.ndarray, t_min: float = 1e-4, bg=(0.0, 0.0, 0.0),
                  form: int = FORM_STABLE, cs: Optional[CScene] = None) -> RenderOut:
    cs = cs or CScene(scene)
    pix = np.ascontiguousarray(pix, np.int32)
    pix_list = np.ascontiguousarray(pix_list, np.int32)
    list_off = np.ascontiguousarray(list_off, np.int64)
    list_prim = np.ascontiguousarray(list_prim, np.int32)
    P = len(pix)
    rgb = np.zeros((P, 3), np.float64)
    tau = np.zeros(P, np.float64)
    nw = np.zeros(P, np.int32)
    fl = np.zeros(P, np.int32)
    bgv = np.asarray(bg, np.float64)
    cc = c_camera(cam)
    n_comp = lib().ora_render(cs.ref(), C.byref(cc), _ptr(pix), P, _ptr(pix_list), _ptr(list_off),
                              _ptr(list_prim), float(t_min), _ptr(bgv), int(form), _ptr(rgb), _ptr(tau),
                              _ptr(nw), _ptr(fl))
    return RenderOut(rgb, tau, nw, fl, int(n_comp))


def pixel_tile(cam, ts: int, pix: np.ndarray) -> np.ndarray:
    tx_n, _ = tiles_xy(cam, ts)
    px = pix % cam.width
    py = pix // cam.width
    return (py // ts) * tx_n + (px // ts)


def render_view_tiled(scene, cams, v: int, tl: TileLists, ts: int, pix: Optional[np.ndarray] = None,
                      t_min: float = 1e-4, bg=(0.0, 0.0, 0.0), form: int = FORM_STABLE,
                      cs: Optional[CScene] = None) -> RenderOut:
    """Render view v (all pixels, or the given linear pixel indices) through the tile lists."""
    cam = cams[v]
    if pix is None:
        pix = np.arange(cam.n_pixels, dtype=np.int32)
    gtile = tl.view_tile_off[v] + pixel_tile(cam, ts, pix)
    list_prim = (tl.vals.astype(np.int64) % scene.n).astype(np.int32)
    return render_pixels(scene, cam, pix, gtile, tl.tile_off, list_prim, t_min, bg, form, cs)


def render_view_brute(scene, cam, pix: Optional[np.ndarray] = None, t_min: float = 1e-4, bg=(0.0, 0.0, 0.0),
                      form: int = FORM_STABLE, cs: Optional[CScene] = None) -> RenderOut:
    """Brute force: every pixel walks every visible primitive (no tiling)."""
    cs = cs or CScene(scene)
    if pix is None:
        pix = np.arange(cam.n_pixels, dtype=np.int32)
    rec = key_project(scene, cam, cs)
    lst = brute_force_list(rec)
    off = np.asarray([0, len(lst)], np.int64)
    return render_pixels(scene, cam, pix, np.zeros(len(pix), np.int32), off, lst, t_min, bg, form, cs)


def render_image(scene, cams, ts: int = 16, t_min: float = 1e-4, bg=(0.0, 0.0, 0.0),
                 form: int = FORM_STABLE):
    """Full tiled render of every view; returns ([H, W, 3] float64 images, TileLists, outs)."""
    cs = CScene(scene)
    tl = tile_keys(scene, cams, ts, cs)
    imgs, outs = [], []
    for v, cam in enumerate(cams):
        o = render_view_tiled(scene, cams, v, tl, ts, None, t_min, bg, form, cs)
        imgs.append(o.rgb.reshape(cam.height, cam.width, 3))
        outs.append(o)
    return imgs, tl, outs


def pair(scene, i: int, o, d, form: int = FORM_STABLE, cs: Optional[CScene] = None, time: float = 0.0):
    cs = cs or CScene(scene)
    o = np.ascontiguousarray(o, np.float64)
    d = np.ascontiguousarray(d, np.float64)
    out = np.zeros(4, np.float64)
    lib().ora_pair(cs.ref(time), int(i), _ptr(o), _ptr(d), int(form), _ptr(out))
    return bool(out[0]), out[1], out[2], out[3]


def integral(scene, i: int, o, d, t0: float, t1: float, form: int = FORM_STABLE,
             cs: Optional[CScene] = None, time: float = 0.0) -> float:
    cs = cs or CScene(scene)
    o = np.ascontiguousarray(o, np.float64)
    d = np.ascontiguousarray(d, np.float64)
    return float(lib().ora_integral(cs.ref(time), int(i), _ptr(o), _ptr(d), float(t0), float(t1), int(form)))


def color(scene, i: int, d, cs: Optional[CScene] = None, eye=(0.0, 0.0, 0.0), time: float = 0.0) -> np.ndarray:
    """Colour of primitive i seen from a camera at `eye` along the unit pixel ray d."""
    cs = cs or CScene(scene)
    d = np.ascontiguousarray(d, np.float64)
    o = np.ascontiguousarray(eye, np.float64)
    out = np.zeros(3, np.float64)
    lib().ora_color(cs.ref(time), int(i), _ptr(o), _ptr(d), _ptr(out))
    return out


def sh_basis(v) -> np.ndarray:
    """The 16 real spherical harmonics of degrees 0..3 at the unit vector v."""
    v = np.ascontiguousarray(v, np.float64)
    out = np.zeros(16, np.float64)
    lib().ora_sh_basis(_ptr(v), _ptr(out))
    return out


def pixel_ray(cam, px: int, py: int) -> np.ndarray:
    cc = c_camera(cam)
    d = np.zeros(3, np.float64)
    lib().ora_pixel_ray(C.byref(cc), int(px), int(py), _ptr(d))
    return d


def mse_loss(image: np.ndarray, target: np.ndarray):
    """Mean squared error over all n values, L = (1/n) sum (image - target)^2, and
    dL/dimage = 2 (image - target) / n, in FP64.  (The paper trains with the
    photometric loss of 3D Gaussian splatting, Sec. 3.3 Training; the squared
    error is the loss of the 300k-primitive 1280 x 720 differentiation workload.)"""
    e = np.asarray(image, np.float64).ravel() - np.asarray(target, np.float64).ravel()
    n = e.size
    if n == 0:
        return 0.0, e
    return float(np.dot(e, e) / n), 2.0 * e / n
