"""Seeded synthetic scenes and cameras for the splattable-neural-primitive renderer.

This module only draws inputs: primitive parameters, network weights and pinhole
cameras.  It holds none of the renderer's arithmetic (no projection, no
intersection, no integral, no compositing), so that the FP64 oracle and the CUDA
path can both consume it without sharing any of the method.

Representation (Sec. 3.1): every primitive has an ellipsoid bound (centre, scale,
rotation quaternion), a one-hidden-layer sine density network of width N_sigma
(Eq. 6: W1 [N_sigma x 3], b1 [N_sigma], W2 [1 x N_sigma], b2) and a colour.  The
colour is either a constant RGB or a per-primitive MLP with two hidden ReLU layers
of width N_c and a sigmoid output, whose input is the unit view direction
concatenated with an 8-d per-primitive feature (the neural colour field of
App. D.2, Eq. "color_render", in the ReLU/sigmoid form this workload fixes).

Draw order (fixed, numpy PCG64): centres, log-scales, quaternions, W1, b1, w2, b2,
rgb, then feat, Wc1, bc1, Wc2, bc2, Wc3, bc3.  N(mu, s) means standard deviation s.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional, Sequence

import numpy as np

FEAT_DIM = 8


@dataclass
class Camera:
    """Pinhole camera, OpenCV frame (x right, y down, z forward).

    R_wc maps world offsets to camera coordinates (rows = camera axes in world).
    fx = fy = (H/2)/tan(fov_y/2), cx = W/2, cy = H/2.  All stored as float32;
    both renderers read exactly these float32 values.
    """

    R_wc: np.ndarray  # (3, 3) float32
    eye: np.ndarray  # (3,) float32
    fx: np.float32
    fy: np.float32
    cx: np.float32
    cy: np.float32
    width: int
    height: int
    z_near: np.float32 = np.float32(0.2)
    time: np.float32 = np.float32(0.0)  # timestamp in [0, 1] (dynamic scenes only)

    @property
    def n_pixels(self) -> int:
        return self.width * self.height


@dataclass
class Scene:
    """Structure-of-arrays primitive set (all float32 numpy arrays).

    weight_dtype "bf16" means the density and colour network weights hold values
    that are exactly representable in bfloat16 (rounded to nearest even from the
    float32 draw); geometry and constant colours always stay float32.
    """

    n: int
    n_sigma: int
    omega0: float
    color: str  # "const" | "mlp"
    n_c: int
    centers: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray  # (w, x, y, z), not normalised
    W1: np.ndarray  # (n, Ns, 3)
    b1: np.ndarray  # (n, Ns)
    w2: np.ndarray  # (n, Ns)
    b2: np.ndarray  # (n,)
    rgb: np.ndarray  # (n, 3)
    feat: Optional[np.ndarray] = None  # (n, 8)
    Wc1: Optional[np.ndarray] = None  # (n, Nc, 3 + 8)
    bc1: Optional[np.ndarray] = None  # (n, Nc)
    Wc2: Optional[np.ndarray] = None  # (n, Nc, Nc)
    bc2: Optional[np.ndarray] = None  # (n, Nc)
    Wc3: Optional[np.ndarray] = None  # (n, 3, Nc)
    bc3: Optional[np.ndarray] = None  # (n, 3)
    sh: Optional[np.ndarray] = None  # (n, 16, 3) spherical-harmonic colour coefficients
    # time-conditioned scenes: phase weights W_t per hidden unit and, with SH colour,
    # the degree-0 time series a_1..a_4, b_1..b_4, c_1..c_4 per channel
    dynamic: bool = False
    wt: Optional[np.ndarray] = None  # (n, Ns)
    sh_t: Optional[np.ndarray] = None  # (n, 12, 3)
    weight_dtype: str = "f32"
    extra: dict = field(default_factory=dict)

    NET_FIELDS = ("W1", "b1", "w2", "b2", "feat", "Wc1", "bc1", "Wc2", "bc2", "Wc3", "bc3", "sh", "wt", "sh_t")
    GEOM_FIELDS = ("centers", "log_scales", "quats", "rgb")

    def fields(self):
        names = list(self.GEOM_FIELDS) + ["W1", "b1", "w2", "b2"]
        if self.color == "mlp":
            names += ["feat", "Wc1", "bc1", "Wc2", "bc2", "Wc3", "bc3"]
        if self.color == "sh":
            names += ["sh"]
        if self.dynamic:
            names += ["wt"] + (["sh_t"] if self.color == "sh" else [])
        return names

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        kw = {}
        for f in self.fields():
            kw[f] = np.ascontiguousarray(getattr(self, f)[idx])
        return replace(self, n=int(len(idx)), **kw)

    def copy(self) -> "Scene":
        kw = {f: getattr(self, f).copy() for f in self.fields()}
        return replace(self, **kw)

    def to_bf16(self) -> "Scene":
        """Round every network weight to bfloat16 (nearest even), keep float32 storage."""
        kw = {}
        for f in self.fields():
            if f in self.NET_FIELDS:
                kw[f] = bf16_round(getattr(self, f))
        return replace(self, weight_dtype="bf16", **kw)


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even); return float32.

    On the bit pattern u: add 0x7FFF plus the lowest kept bit, clear the low 16
    bits.  In uint32 this wraps only for negative NaN patterns (>= 0xFFFF8000);
    finite values and infinities round exactly, overflow going to infinity."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty_like(x)
    src, dst = x.reshape(-1).view(np.uint32), out.reshape(-1).view(np.uint32)
    step = 1 << 24  # bounded temporaries for the 500k-primitive scenes
    for a in range(0, src.size, step):
        u = src[a:a + step]
        r = dst[a:a + step]
        np.right_shift(u, 16, out=r)
        r &= np.uint32(1)
        r += np.uint32(0x7FFF)
        r += u
        r &= np.uint32(0xFFFF0000)
    return out


# ----------------------------------------------------------------------------- scene files

_HEADER_KEYS = ("n", "n_sigma", "omega0", "color", "n_c", "weight_dtype", "dynamic")
_CAMERA_KEYS = ("R_wc", "eye", "fx", "fy", "cx", "cy", "width", "height", "z_near", "time")


def save_scene(scene: Scene, path: str, cameras: Optional[Sequence[Camera]] = None) -> None:
    """Write a scene (and optionally its cameras) as one .npz file: the structure-of-
    arrays fields in float32 plus a JSON header with the sizes and modes."""
    import json
    header = {k: getattr(scene, k) for k in _HEADER_KEYS}
    header["fields"] = list(scene.fields())
    arrays = {f: np.ascontiguousarray(getattr(scene, f), dtype=np.float32) for f in scene.fields()}
    if cameras is not None:
        header["cameras"] = [{k: np.asarray(getattr(c, k)).tolist() for k in _CAMERA_KEYS} for c in cameras]
    np.savez(path, __header__=np.frombuffer(json.dumps(header).encode(), dtype=np.uint8), **arrays)


def load_scene(path: str):
    """Read a file written by save_scene: returns (scene, cameras or None)."""
    import json
    z = np.load(path)
    header = json.loads(bytes(z["__header__"]).decode())
    kw = {k: header[k] for k in _HEADER_KEYS}
    arrays = {f: np.ascontiguousarray(z[f], dtype=np.float32) for f in header["fields"]}
    base = {f: arrays.get(f) for f in ("centers", "log_scales", "quats", "W1", "b1", "w2", "b2", "rgb")}
    sc = Scene(n=int(kw["n"]), n_sigma=int(kw["n_sigma"]), omega0=float(kw["omega0"]), color=kw["color"],
               n_c=int(kw["n_c"]), weight_dtype=kw["weight_dtype"], dynamic=bool(kw["dynamic"]), **base)
    for f, a in arrays.items():
        if f not in base:
            setattr(sc, f, a)
    cams = None
    if "cameras" in header:
        cams = []
        for c in header["cameras"]:
            cams.append(Camera(R_wc=np.asarray(c["R_wc"], np.float32), eye=np.asarray(c["eye"], np.float32),
                               fx=np.float32(c["fx"]), fy=np.float32(c["fy"]), cx=np.float32(c["cx"]),
                               cy=np.float32(c["cy"]), width=int(c["width"]), height=int(c["height"]),
                               z_near=np.float32(c["z_near"]), time=np.float32(c["time"])))
    return sc, cams


# ----------------------------------------------------------------------------- cameras


def look_at_camera(eye, target, width: int, height: int, fov_y_deg: float = 60.0,
                   up=(0.0, 1.0, 0.0), z_near: float = 0.2) -> Camera:
    eye = np.asarray(eye, dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    up = np.asarray(up, dtype=np.float64)
    f = target - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    dn = np.cross(f, r)
    R = np.stack([r, dn, f]).astype(np.float32)
    fy = (height / 2.0) / math.tan(math.radians(fov_y_deg) / 2.0)
    return Camera(R_wc=R, eye=eye.astype(np.float32), fx=np.float32(fy), fy=np.float32(fy),
                  cx=np.float32(width / 2.0), cy=np.float32(height / 2.0),
                  width=int(width), height=int(height), z_near=np.float32(z_near))


def ring_cameras(n: int, radius: float, width: int, height: int) -> List[Camera]:
    """eye_k = R (sin t_k, 0, cos t_k), t_k = 2 pi k / n, looking at the origin."""
    cams = []
    for k in range(n):
        t = 2.0 * math.pi * k / n
        cams.append(look_at_camera((radius * math.sin(t), 0.0, radius * math.cos(t)),
                                   (0, 0, 0), width, height))
    return cams


def fibonacci_cameras(n: int, radius: float, resolutions: Sequence) -> List[Camera]:
    """Fibonacci sphere: y_i = 1 - (2i+1)/n, golden-angle azimuth; looking at the origin."""
    ga = math.pi * (3.0 - math.sqrt(5.0))
    cams = []
    for i in range(n):
        y = 1.0 - (2.0 * i + 1.0) / n
        rr = math.sqrt(max(0.0, 1.0 - y * y))
        th = ga * i
        eye = (radius * rr * math.cos(th), radius * y, radius * rr * math.sin(th))
        w, h = resolutions[i]
        cams.append(look_at_camera(eye, (0, 0, 0), w, h))
    return cams


# ----------------------------------------------------------------------------- scenes


def make_scene(n: int, seed: int = 0, *, center_half: float = 1.0, n_sigma: int = 8,
               omega0: float = 5.0, color: str = "const", n_c: int = 32,
               log_scale_mean: float = -2.0, log_scale_std: float = 0.3,
               thin_ratio_max: Optional[float] = None, dynamic: bool = False, rng=None) -> Scene:
    """Draw a scene with the distributions of the benchmark workloads.

    centres ~ U[-h, h]^3, log-scales ~ N(-2, 0.3) per axis, quaternions ~ N(0, I4),
    W1 ~ N(0, 1), b1 ~ U(-pi, pi), w2 ~ N(0, 0.5), b2 = 0.5, rgb ~ U(0, 1);
    colour MLP: feat ~ N(0, 1), Wc_l ~ N(0, 1/sqrt(fan_in)), biases 0.
    spherical harmonics ("sh"): degree-0 coefficients ~ N(0, 0.6), degrees 1..3 ~ N(0, 0.2).
    dynamic: W_t ~ N(0, 2) (phase shift per unit time); with SH colour the degree-0
    time series coefficients ~ N(0, 0.1).  Drawn last, after everything above.
    thin_ratio_max: if set, axis 0 is the major axis ~ N(-2, 0.3) and the other two
    are major - ln r with r ~ logU[1, thin_ratio_max] (independently per axis).
    """
    g = rng if rng is not None else np.random.Generator(np.random.PCG64(seed))
    f32 = np.float32
    centers = g.uniform(-center_half, center_half, size=(n, 3)).astype(f32)
    if thin_ratio_max is None:
        log_scales = g.normal(log_scale_mean, log_scale_std, size=(n, 3)).astype(f32)
    else:
        major = g.normal(log_scale_mean, log_scale_std, size=(n, 1))
        lr = g.uniform(0.0, math.log(thin_ratio_max), size=(n, 2))
        log_scales = np.concatenate([major, major - lr], axis=1).astype(f32)
    quats = g.normal(0.0, 1.0, size=(n, 4)).astype(f32)
    W1 = g.normal(0.0, 1.0, size=(n, n_sigma, 3)).astype(f32)
    b1 = g.uniform(-math.pi, math.pi, size=(n, n_sigma)).astype(f32)
    w2 = g.normal(0.0, 0.5, size=(n, n_sigma)).astype(f32)
    b2 = np.full((n,), 0.5, dtype=f32)
    rgb = g.uniform(0.0, 1.0, size=(n, 3)).astype(f32)
    sc = Scene(n=n, n_sigma=n_sigma, omega0=float(omega0), color=color, n_c=n_c,
               centers=centers, log_scales=log_scales, quats=quats, W1=W1, b1=b1, w2=w2,
               b2=b2, rgb=rgb)
    if color == "mlp":
        # the colour-network weights (up to 2.6 G values at 500k primitives) are drawn
        # directly in float32, without float64 temporaries
        def normal32(std, size):
            out = g.standard_normal(size=size, dtype=f32)
            out *= f32(std)
            return out
        fin1 = 3 + FEAT_DIM
        sc.feat = g.normal(0.0, 1.0, size=(n, FEAT_DIM)).astype(f32)
        sc.Wc1 = normal32(1.0 / math.sqrt(fin1), (n, n_c, fin1))
        sc.bc1 = np.zeros((n, n_c), dtype=f32)
        sc.Wc2 = normal32(1.0 / math.sqrt(n_c), (n, n_c, n_c))
        sc.bc2 = np.zeros((n, n_c), dtype=f32)
        sc.Wc3 = normal32(1.0 / math.sqrt(n_c), (n, 3, n_c))
        sc.bc3 = np.zeros((n, 3), dtype=f32)
    if color == "sh":
        sh = g.normal(0.0, 0.2, size=(n, 16, 3))
        sh[:, 0, :] = g.normal(0.0, 0.6, size=(n, 3))
        sc.sh = sh.astype(f32)
    if dynamic:
        sc.dynamic = True
        sc.wt = g.normal(0.0, 2.0, size=(n, n_sigma)).astype(f32)
        if color == "sh":
            sc.sh_t = g.normal(0.0, 0.1, size=(n, 12, 3)).astype(f32)
    return sc


def perturb(scene: Scene, seed: int, std: float = 0.01) -> Scene:
    """Copy of the scene with every parameter + N(0, std) (the target of the L2 workload)."""
    g = np.random.Generator(np.random.PCG64(seed))
    out = scene.copy()
    for f in scene.fields():
        a = getattr(out, f)
        a += g.normal(0.0, std, size=a.shape).astype(np.float32)
    return out


def orthogonalise_rows(scene: Scene, cam: Camera, seed: int, fraction: float,
                       row_scale_logrange=(-3.0, 0.0)) -> Scene:
    """Near-zero directional frequency stress (w . d -> 0).

    For a seeded `fraction` of primitives, one W1 row is replaced by rho * n_hat,
    where n_hat is the unit normal of the plane through the camera eye that
    contains the primitive's major axis (local axis 0).  Every ray from the eye
    through a point of that axis is orthogonal to n_hat, so w . d is small for
    rays through a thin primitive.  rho = ||w|| * 10^U(lo, hi) shrinks the row
    further.  Half of the chosen primitives instead use the unit normal of the
    plane through the eye spanned by the centre ray and a random direction, so
    the row is exactly orthogonal to the centre ray only.
    """
    g = np.random.Generator(np.random.PCG64(seed))
    out = scene.copy()
    n = scene.n
    pick = np.nonzero(g.uniform(size=n) < fraction)[0]
    k_row = g.integers(0, scene.n_sigma, size=len(pick))
    mode = g.uniform(size=len(pick)) < 0.5
    lo, hi = row_scale_logrange
    expo = g.uniform(lo, hi, size=len(pick))
    rnd = g.normal(size=(len(pick), 3))
    q = scene.quats[pick].astype(np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    # first column of the rotation matrix of q = the local x axis in world space
    axis = np.stack([1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y)], axis=1)
    ray = scene.centers[pick].astype(np.float64) - cam.eye.astype(np.float64)[None]
    other = np.where(mode[:, None], axis, rnd)
    nrm = np.cross(other, ray)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    for j, (i, k) in enumerate(zip(pick, k_row)):
        wnorm = float(np.linalg.norm(out.W1[i, k].astype(np.float64)))
        out.W1[i, k] = (wnorm * 10.0 ** expo[j] * nrm[j]).astype(np.float32)
    out.extra = dict(out.extra, ortho_prims=pick, ortho_rows=k_row)
    return out


# ----------------------------------------------------------------------------- workloads

RESOLUTIONS = ((320, 240), (640, 480), (1280, 720), (1920, 1080))


@dataclass
class Workload:
    name: str
    scene: Scene
    cameras: List[Camera]
    tile_size: int = 16
    t_min: float = 1e-4
    note: str = ""
    # differentiation workload: the loss is the squared error against a render of this scene
    target_scene: Optional[Scene] = None

    @property
    def n_pixels(self) -> int:
        return sum(c.n_pixels for c in self.cameras)


def workload(name: str, seed: int = 0) -> Workload:
    """The benchmark workloads (WORKLOADS) and their profiler cases, by name (all seeded, synthetic)."""
    if name == "tiny64_128px":
        sc = make_scene(64, seed, center_half=1.0, n_sigma=8, omega0=5.0, color="const")
        cam = look_at_camera((0.0, 0.0, 4.0), (0, 0, 0), 128, 128)
        return Workload(name, sc, [cam], 16)
    if name == "fwd100k_1080p_4view":
        sc = make_scene(100_000, seed, center_half=3.0, n_sigma=16, omega0=5.0, color="mlp", n_c=32)
        return Workload(name, sc, ring_cameras(4, 8.0, 1920, 1080), 16)
    if name == "prof100k_1080p_1view":
        # the first view of the 100k / four-view workload, for profiler captures
        wl = workload("fwd100k_1080p_4view", seed)
        return Workload(name, wl.scene, wl.cameras[:1], 16)
    if name == "prof100k_540p_1view":
        # the 100k-primitive scene seen by one ring view at a quarter of the 1080p
        # pixels, for full-set profiler captures of a small case
        wl = workload("fwd100k_1080p_4view", seed)
        return Workload(name, wl.scene, ring_cameras(1, 8.0, 960, 540), 16)
    if name == "batch100k_16view_quarter":
        # the batched workload's primitive (N_sigma = 32, N_c = 64, BF16) at 100k
        # primitives, its 16 view sizes at a quarter of the pixels, for captures
        sc = make_scene(100_000, seed, center_half=3.0, n_sigma=32, omega0=5.0, color="mlp", n_c=64)
        g = np.random.Generator(np.random.PCG64(seed + 7))
        res = [(w // 2, h // 2) for (w, h) in (RESOLUTIONS[i] for i in g.integers(0, 4, size=16))]
        return Workload(name, sc.to_bf16(), fibonacci_cameras(16, 10.0, res), 16)
    if name == "diff300k_720p":
        sc = make_scene(300_000, seed, center_half=3.0, n_sigma=16, omega0=5.0, color="mlp", n_c=32)
        return Workload(name, sc, ring_cameras(1, 8.0, 1280, 720), 16, target_scene=perturb(sc, seed + 11, 0.01))
    if name == "thin50k_1080p":
        sc = make_scene(50_000, seed, center_half=3.0, n_sigma=16, omega0=30.0, color="mlp",
                        n_c=32, thin_ratio_max=50.0)
        cams = ring_cameras(1, 8.0, 1920, 1080)
        sc = orthogonalise_rows(sc, cams[0], seed + 1, fraction=0.5)
        return Workload(name, sc, cams, 16)
    if name == "batch500k_16view":
        sc = make_scene(500_000, seed, center_half=3.0, n_sigma=32, omega0=5.0, color="mlp", n_c=64)
        g = np.random.Generator(np.random.PCG64(seed + 7))
        res = [RESOLUTIONS[i] for i in g.integers(0, 4, size=16)]
        return Workload(name, sc.to_bf16(), fibonacci_cameras(16, 10.0, res), 16)
    if name == "fps100k_800px_sh_1view":
        # the first view of the speed-protocol workload, for full-set profiler captures
        wl = workload("fps100k_800px_sh", seed)
        return Workload(name, wl.scene, wl.cameras[:1], 16)
    if name in ("fps100k_800px_sh", "dyn100k_800px_8t"):
        # The speed protocol of App. A (Integration Cost): 100k random primitives in a
        # volume, the primitive of Sec. 3.3 (Implementation Details: N_sigma = 8, w0 = 30,
        # four SH bands) with its initialisation of the density weights,
        # W1 ~ U(-1/3, 1/3) and w2 ~ U(-sqrt(6/N_sigma)/w0, +), seen by square 800 x 800
        # views at a 39.6 degree field of view on a radius-4 ring at 30 degrees elevation
        # (the camera set-up of the synthetic scenes).  The dynamic variant (the
        # volumetric dynamic scenes of App. Applications) adds the time-conditioned
        # density and degree-0 colour series and gives view k the timestamp k / 7.
        dyn = name.startswith("dyn")
        sc = make_scene(100_000, seed, center_half=1.5, n_sigma=8, omega0=30.0, color="sh",
                        log_scale_mean=-3.0, dynamic=dyn)
        g = np.random.Generator(np.random.PCG64(seed + 3))
        sc.W1 = g.uniform(-1.0 / 3.0, 1.0 / 3.0, size=sc.W1.shape).astype(np.float32)
        lim = math.sqrt(6.0 / sc.n_sigma) / sc.omega0
        sc.w2 = g.uniform(-lim, lim, size=sc.w2.shape).astype(np.float32)
        cams = []
        for k in range(8):
            t = 2.0 * math.pi * k / 8
            eye = (4.0 * math.sin(t) * math.cos(math.radians(30.0)), 4.0 * math.sin(math.radians(30.0)),
                   4.0 * math.cos(t) * math.cos(math.radians(30.0)))
            cam = look_at_camera(eye, (0, 0, 0), 800, 800, fov_y_deg=39.6)
            if dyn:
                cam.time = np.float32(k / 7.0)
            cams.append(cam)
        return Workload(name, sc, cams, 16)
    raise KeyError(name)


WORKLOADS = ("tiny64_128px", "fwd100k_1080p_4view", "diff300k_720p", "thin50k_1080p",
             "batch500k_16view", "fps100k_800px_sh", "dyn100k_800px_8t")
# smaller cases of the same scenes for profiler captures
PROFILE_WORKLOADS = ("prof100k_1080p_1view", "prof100k_540p_1view", "batch100k_16view_quarter",
                     "fps100k_800px_sh_1view")
