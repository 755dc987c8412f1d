"""Pins for the oracle's time-conditioned scenes (App. Applications, volumetric
dynamic scenes): the density's cosine argument gains xi_t W_t, and with SH colour
the degree-0 coefficient follows sh_0 + sum_j a_j xi^j + b_j cos(j xi) + c_j sin(j xi).

Checked against (1) adaptive quadrature of the time-conditioned density written
out directly (the closed form must keep its shape, since the time term is constant
along a ray), and (2) the static renderer on an equivalent static scene (the time
phase moved into b1, the series value into sh_0), which exercises a different
code path: the camera's timestamp must reach both integral forms and the colour.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from paper_2510_08491_gb300 import synth

from test_oracle_integral import rays_through


def sigma_t(sc, i, x, xi):
    """sigma(x, xi) = w2 . cos(w0 (W1 u + b1) + xi W_t) + b2, u = (x - c) / max(s)."""
    s = np.exp(sc.log_scales[i].astype(np.float64))
    u = (x - sc.centers[i].astype(np.float64)) / s.max()
    arg = sc.omega0 * (sc.W1[i].astype(np.float64) @ u + sc.b1[i].astype(np.float64)) \
        + xi * sc.wt[i].astype(np.float64)
    return float(sc.w2[i].astype(np.float64) @ np.cos(arg) + float(sc.b2[i]))


@pytest.mark.parametrize("xi", [0.0, 0.37, 1.0])
def test_time_integral_matches_quadrature(oracle_lib, xi):
    O = oracle_lib
    sc = synth.make_scene(10, seed=21, center_half=1.0, n_sigma=8, omega0=5.0, dynamic=True)
    rng = np.random.default_rng(8)
    o = np.array([0.2, 0.1, 4.0])
    cs = O.CScene(sc)
    worst = {O.FORM_STABLE: 0.0, O.FORM_NAIVE: 0.0}
    for i in range(sc.n):
        for d in rays_through(sc, i, rng, 5, o):
            ref = None
            for form in worst:
                hit, t0, t1, ah = O.pair(sc, i, o, d, form, cs, time=xi)
                assert hit
                if ref is None:
                    ref, _ = integrate.quad(lambda t: sigma_t(sc, i, o + t * d, xi), t0, t1,
                                            epsabs=1e-13, epsrel=1e-12, limit=400)
                scale = (t1 - t0) * (abs(float(sc.b2[i])) + np.abs(sc.w2[i]).sum())
                worst[form] = max(worst[form], abs(ah - ref) / scale)
    assert worst[O.FORM_STABLE] < 1e-10, worst
    assert worst[O.FORM_NAIVE] < 1e-7, worst  # well-conditioned rays only (|W1 . d| not tiny)


def _static_equivalent(sc, xi):
    """A static float64 scene rendering the same image as sc at time xi."""
    st = sc.copy()
    for f in st.fields():
        setattr(st, f, getattr(st, f).astype(np.float64))
    st.b1 = st.b1 + xi * st.wt / st.omega0
    if st.color == "sh":
        j = np.arange(1, 5, dtype=np.float64)
        basis = np.concatenate([xi ** j, np.cos(j * xi), np.sin(j * xi)])
        st.sh = st.sh.copy()
        st.sh[:, 0, :] += np.einsum("j,njc->nc", basis, st.sh_t)
    st.dynamic, st.wt, st.sh_t = False, None, None
    return st


@pytest.mark.parametrize("color,xi", [("const", 0.8), ("sh", 0.0), ("sh", 0.45), ("sh", 1.0)])
def test_time_render_equals_static_equivalent(oracle_lib, color, xi):
    O = oracle_lib
    sc = synth.make_scene(300, seed=4, center_half=1.0, n_sigma=8, omega0=5.0, color=color, dynamic=True)
    cam = synth.look_at_camera((0.0, 0.5, 4.0), (0, 0, 0), 64, 48)
    cam.time = np.float32(xi)
    xi32 = float(np.float32(xi))
    pix = np.arange(cam.n_pixels, dtype=np.int32)
    tl = O.tile_keys(sc, [cam], 16)
    st = _static_equivalent(sc, xi32)
    for form in (O.FORM_STABLE, O.FORM_NAIVE):
        a = O.render_view_tiled(sc, [cam], 0, tl, 16, pix, t_min=0.0, form=form)
        b = O.render_view_tiled(st, [cam], 0, tl, 16, pix, t_min=0.0, form=form)
        assert a.n_comp == b.n_comp and a.n_comp > 100
        assert np.abs(a.rgb - b.rgb).max() < 1e-12
    # and the timestamp matters: another time gives another image
    cam.time = np.float32(xi + 0.25)
    c = O.render_view_tiled(sc, [cam], 0, tl, 16, pix, t_min=0.0)
    assert np.abs(c.rgb - a.rgb).max() > 1e-3


def test_time_phase_period(oracle_lib):
    """W_t -> W_t + 2 pi / xi leaves every phase unchanged modulo 2 pi."""
    O = oracle_lib
    sc = synth.make_scene(200, seed=6, center_half=1.0, n_sigma=8, omega0=5.0, dynamic=True)
    cam = synth.look_at_camera((0.0, 0.0, 4.0), (0, 0, 0), 48, 48)
    xi = 0.5
    cam.time = np.float32(xi)
    pix = np.arange(cam.n_pixels, dtype=np.int32)
    tl = O.tile_keys(sc, [cam], 16)
    a = O.render_view_tiled(sc, [cam], 0, tl, 16, pix, t_min=0.0)
    sh = sc.copy()
    sh.wt = sh.wt.astype(np.float64) + 2.0 * math.pi / xi
    b = O.render_view_tiled(sh, [cam], 0, tl, 16, pix, t_min=0.0)
    assert np.abs(a.rgb - b.rgb).max() < 1e-10
