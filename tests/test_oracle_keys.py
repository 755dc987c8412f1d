"""Pins for the oracle's FP32 key specification (bounding, culling, depth key, tile lists).

The silhouette rectangle is checked against rays: every pixel whose centre ray hits
a primitive's ellipsoid (independent FP64 intersection with scipy's rotation) must
lie in that primitive's rectangle, and the rectangle must not exceed the exact
FP64 silhouette extent by more than one pixel.  The depth key is checked against
the FP64 camera-frame depth, the sort against its definition.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2510_08491_gb300 import synth


def exact_geometry(sc, cam):
    """FP64 camera-frame centres, covariances and scales, via scipy rotations."""
    q = sc.quats.astype(np.float64)
    R = Rotation.from_quat(np.stack([q[:, 1], q[:, 2], q[:, 3], q[:, 0]], 1)).as_matrix()
    s = np.exp(sc.log_scales.astype(np.float64))
    Rwc = cam.R_wc.astype(np.float64)
    V = np.einsum("ab,nbj->naj", Rwc, R) * s[:, None, :]
    Sig = V @ V.transpose(0, 2, 1)
    mu = (sc.centers.astype(np.float64) - cam.eye.astype(np.float64)) @ Rwc.T
    return mu, Sig, s


def hit_mask(sc, i, cam, px, py):
    """Does the FP64 centre ray of each pixel hit ellipsoid i (raw quadratic, scipy rotation)?"""
    q = sc.quats[i].astype(np.float64)
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    s = np.exp(sc.log_scales[i].astype(np.float64))
    x = (px + 0.5 - float(cam.cx)) / float(cam.fx)
    y = (py + 0.5 - float(cam.cy)) / float(cam.fy)
    Rwc = cam.R_wc.astype(np.float64)
    d = x[:, None] * Rwc[0] + y[:, None] * Rwc[1] + Rwc[2]
    M = R.T / s[:, None]
    a = d @ M.T
    b = M @ (cam.eye.astype(np.float64) - sc.centers[i].astype(np.float64))
    A = (a * a).sum(1)
    B = 2 * a @ b
    Cc = b @ b - 1
    return B * B - 4 * A * Cc > 0


def exact_extent(mu, Sig, f, cc, axis):
    """Exact silhouette interval in image coordinate `axis` (0 = u, 1 = v), FP64."""
    ma, mz = mu[axis], mu[2]
    saa, saz, szz = Sig[axis, axis], Sig[axis, 2], Sig[2, 2]
    a = mz * mz - szz
    b = f * (ma * mz - saz)
    disc = f * f * ((ma * mz - saz) ** 2 - a * (ma * ma - saa))
    r = math.sqrt(max(disc, 0.0))
    return cc - (r - b) / a, cc - (-b - r) / a


@pytest.mark.parametrize("name,thin", [("tiny", None), ("thin", 50.0)])
def test_rect_contains_every_hit_pixel(oracle_lib, name, thin):
    O = oracle_lib
    sc = synth.make_scene(64 if thin is None else 200, seed=0, center_half=1.0, thin_ratio_max=thin)
    cam = synth.look_at_camera((0.0, 0.0, 4.0), (0, 0, 0), 128, 96)
    rec = O.key_project(sc, cam)
    W, H = cam.width, cam.height
    PY, PX = np.mgrid[0:H, 0:W]
    PX, PY = PX.ravel().astype(np.float64), PY.ravel().astype(np.float64)
    n_hits = 0
    for i in range(sc.n):
        hits = hit_mask(sc, i, cam, PX, PY)
        if not rec.visible[i]:
            # culled primitives are either behind the near plane or cover no pixel centre
            continue
        x0, y0, x1, y1 = rec.rect[i]
        inside = (PX >= x0) & (PX <= x1) & (PY >= y0) & (PY <= y1)
        assert not np.any(hits & ~inside), i
        n_hits += hits.sum()
    assert n_hits > 100


def test_culled_primitives_cover_no_pixel(oracle_lib):
    O = oracle_lib
    sc = synth.make_scene(300, seed=1, center_half=3.0)
    cam = synth.look_at_camera((0.0, 0.0, 2.5), (0, 0, 0), 64, 48)
    rec = O.key_project(sc, cam)
    mu, Sig, s = exact_geometry(sc, cam)
    assert (rec.visible == 0).sum() > 30
    PY, PX = np.mgrid[0:cam.height, 0:cam.width]
    PX, PY = PX.ravel().astype(np.float64), PY.ravel().astype(np.float64)
    for i in np.nonzero(rec.visible == 0)[0]:
        near = mu[i, 2] - s[i].max() <= float(cam.z_near) + 1e-6
        if near:
            continue  # behind / across the near plane: culled by definition
        assert not np.any(hit_mask(sc, i, cam, PX, PY))


@pytest.mark.parametrize("thin", [None, 50.0])
def test_rect_is_tight_and_conservative(oracle_lib, thin):
    O = oracle_lib
    sc = synth.make_scene(2000, seed=5, center_half=3.0, thin_ratio_max=thin)
    cam = synth.look_at_camera((0.0, 0.0, 8.0), (0, 0, 0), 1920, 1080)
    rec = O.key_project(sc, cam)
    mu, Sig, s = exact_geometry(sc, cam)
    checked = 0
    for i in np.nonzero(rec.visible)[0]:
        u0, u1 = exact_extent(mu[i], Sig[i], float(cam.fx), float(cam.cx), 0)
        v0, v1 = exact_extent(mu[i], Sig[i], float(cam.fy), float(cam.cy), 1)
        lo_u, hi_u = math.ceil(u0 - 0.5), math.floor(u1 - 0.5)
        lo_v, hi_v = math.ceil(v0 - 0.5), math.floor(v1 - 0.5)
        x0, y0, x1, y1 = rec.rect[i]
        # conservative: contains every pixel centre inside the exact extent
        assert x0 <= max(lo_u, 0) and x1 >= min(hi_u, cam.width - 1)
        assert y0 <= max(lo_v, 0) and y1 >= min(hi_v, cam.height - 1)
        # tight: at most one extra pixel column/row on each side
        assert x0 >= max(lo_u, 0) - 1 and x1 <= min(hi_u, cam.width - 1) + 1
        assert y0 >= max(lo_v, 0) - 1 and y1 <= min(hi_v, cam.height - 1) + 1
        checked += 1
    assert checked > 500


def test_depth_key_is_camera_z(oracle_lib):
    O = oracle_lib
    sc = synth.make_scene(500, seed=6, center_half=3.0)
    cam = synth.ring_cameras(4, 8.0, 320, 240)[1]
    rec = O.key_project(sc, cam)
    mu, _, _ = exact_geometry(sc, cam)
    assert np.allclose(rec.depth.astype(np.float64), mu[:, 2], rtol=1e-6, atol=1e-6)


def test_key_exp_accuracy(oracle_lib):
    O = oracle_lib
    xs = np.linspace(-12.0, 6.0, 20001).astype(np.float32)
    worst = 0.0
    for x in xs[::7]:
        e = O.key_exp(x)
        ref = math.exp(float(x))
        ulp = np.spacing(np.float32(ref))
        worst = max(worst, abs(float(e) - ref) / float(ulp))
    assert worst <= 2.0, worst


def test_tile_lists_are_sorted_and_complete(oracle_lib):
    O = oracle_lib
    sc = synth.make_scene(3000, seed=7, center_half=3.0)
    cams = synth.ring_cameras(3, 8.0, 200, 150)
    ts = 16
    tl = O.tile_keys(sc, cams, ts)
    k = tl.keys
    assert np.all(k[1:] >= k[:-1])
    same = k[1:] == k[:-1]
    # equal keys keep emission order: ascending record index
    assert np.all(tl.vals[1:][same] > tl.vals[:-1][same])
    # every visible primitive appears once in each tile of its rectangle
    for v, cam in enumerate(cams):
        rec = tl.records[v]
        tx_n, _ = O.tiles_xy(cam, ts)
        lo, hi = tl.view_tile_off[v], tl.view_tile_off[v + 1]
        sel = (k >> np.uint64(32)).astype(np.int64)
        sel = (sel >= lo) & (sel < hi)
        prim = tl.vals[sel].astype(np.int64) - v * sc.n
        cnt = np.bincount(prim, minlength=sc.n)
        r = rec.rect // ts
        exp_cnt = np.where(rec.visible == 1, (r[:, 2] - r[:, 0] + 1) * (r[:, 3] - r[:, 1] + 1), 0)
        assert np.array_equal(cnt, exp_cnt)
        tiles = (k[sel] >> np.uint64(32)).astype(np.int64) - lo
        tx, ty = tiles % tx_n, tiles // tx_n
        assert np.all((tx >= r[prim, 0]) & (tx <= r[prim, 2]) & (ty >= r[prim, 1]) & (ty <= r[prim, 3]))
