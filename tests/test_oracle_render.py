"""Pins for the oracle's compositing (Eq. 4), kernel alpha (Eq. 9) and colour MLP.

Closed forms for one and two primitives, brute force over all primitives versus
the tiled lists, invariance under input permutation, transmittance/colour bounds,
the early-termination bound, and the colour MLP against torch.nn.functional.
"""
import math

import numpy as np
import pytest
import torch

from paper_2510_08491_gb300 import synth


def test_brute_force_equals_tiled(oracle_lib):
    O = oracle_lib
    wl = synth.workload("tiny64_128px")
    imgs, tl, outs = O.render_image(wl.scene, wl.cameras, 16)
    b = O.render_view_brute(wl.scene, wl.cameras[0])
    assert np.abs(b.rgb.reshape(imgs[0].shape) - imgs[0]).max() <= 1e-15
    assert outs[0].n_comp == b.n_comp > 1000


def test_brute_force_equals_tiled_mlp(oracle_lib):
    O = oracle_lib
    sc = synth.make_scene(300, seed=3, center_half=1.0, n_sigma=16, color="mlp", n_c=32)
    cams = synth.ring_cameras(2, 4.0, 96, 64)
    imgs, tl, outs = O.render_image(sc, cams, 8)
    for v in range(2):
        b = O.render_view_brute(sc, cams[v])
        assert np.abs(b.rgb.reshape(imgs[v].shape) - imgs[v]).max() <= 1e-15


def _one_sphere(center, radius, rgb, sigma0_b2, omega0=5.0):
    sc = synth.make_scene(1, seed=0, n_sigma=8, omega0=omega0)
    sc.centers[0] = np.float32(center)
    sc.log_scales[0] = np.float32(math.log(radius))
    sc.W1[:] = 0.0
    sc.w2[:] = 0.0
    sc.b2[:] = np.float32(sigma0_b2)
    sc.rgb[0] = np.float32(rgb)
    return sc


def _ray_point_distance(o, d, c):
    return np.linalg.norm(np.cross(c - o, d))


def test_single_sphere_closed_form(oracle_lib):
    """One constant-density sphere: C = rgb (1 - exp(-sigma chord)), chord = 2 sqrt(r^2 - p^2)."""
    O = oracle_lib
    sc = _one_sphere([0.05, -0.1, 0.0], 0.4, [0.2, 0.7, 0.9], 1.5)
    cam = synth.look_at_camera((0.0, 0.0, 4.0), (0, 0, 0), 64, 64)
    out = O.render_view_brute(sc, cam, t_min=0.0)
    r = math.exp(float(sc.log_scales[0, 0]))
    c = sc.centers[0].astype(np.float64)
    o = cam.eye.astype(np.float64)
    for p in range(cam.n_pixels):
        d = O.pixel_ray(cam, p % 64, p // 64)
        dist = _ray_point_distance(o, d, c)
        chord = 2 * math.sqrt(r * r - dist * dist) if dist < r else 0.0
        alpha = 1 - math.exp(-float(sc.b2[0]) * chord)
        ref = alpha * sc.rgb[0].astype(np.float64)
        assert np.abs(out.rgb[p] - ref).max() < 1e-13


def test_two_spheres_front_to_back(oracle_lib):
    """C = c1 a1 + c2 a2 (1 - a1) with 1 the nearer primitive (Eq. 4)."""
    O = oracle_lib
    s1 = _one_sphere([0.0, 0.0, 0.5], 0.3, [1.0, 0.0, 0.0], 2.0)
    s2 = _one_sphere([0.1, 0.0, -0.5], 0.35, [0.0, 0.0, 1.0], 3.0)
    sc = s1.copy()
    for f in sc.fields():
        setattr(sc, f, np.concatenate([getattr(s2, f), getattr(s1, f)]))  # far one first in input order
    sc.n = 2
    cam = synth.look_at_camera((0.0, 0.0, 4.0), (0, 0, 0), 48, 48)
    out = O.render_view_brute(sc, cam, t_min=0.0, bg=(0.1, 0.2, 0.3))
    o = cam.eye.astype(np.float64)
    for p in range(cam.n_pixels):
        d = O.pixel_ray(cam, p % 48, p // 48)
        al = []
        for sp in (s1, s2):
            r = math.exp(float(sp.log_scales[0, 0]))
            dist = _ray_point_distance(o, d, sp.centers[0].astype(np.float64))
            chord = 2 * math.sqrt(r * r - dist * dist) if dist < r else 0.0
            al.append(1 - math.exp(-float(sp.b2[0]) * chord))
        c1, c2 = s1.rgb[0].astype(np.float64), s2.rgb[0].astype(np.float64)
        ref = c1 * al[0] + c2 * al[1] * (1 - al[0])
        ref = ref + (1 - al[0]) * (1 - al[1]) * np.array([0.1, 0.2, 0.3])
        assert np.abs(out.rgb[p] - ref).max() < 1e-13


def test_permutation_invariance(oracle_lib):
    O = oracle_lib
    sc = synth.make_scene(150, seed=12, center_half=1.0, n_sigma=8, color="mlp", n_c=32)
    cams = [synth.look_at_camera((0.0, 0.5, 4.0), (0, 0, 0), 80, 60)]
    img, _, _ = O.render_image(sc, cams, 16)
    perm = np.random.default_rng(0).permutation(sc.n)
    img2, _, _ = O.render_image(sc.subset(perm), cams, 16)
    assert np.abs(img[0] - img2[0]).max() < 1e-15


def test_bounds_and_termination(oracle_lib):
    """0 <= C <= max colour; dropping the tail after T < T_min changes C by at most T_min max c."""
    O = oracle_lib
    sc = synth.make_scene(400, seed=13, center_half=0.7, n_sigma=8)
    sc.b2[:] = 3.0  # dense: many pixels terminate
    cams = [synth.look_at_camera((0.0, 0.0, 4.0), (0, 0, 0), 64, 64)]
    a, _, oa = O.render_image(sc, cams, 16, t_min=1e-4)
    b, _, ob = O.render_image(sc, cams, 16, t_min=0.0)
    assert a[0].min() >= 0 and a[0].max() <= sc.rgb.max() + 1e-12
    assert np.all(np.exp(-oa[0].tau) >= 0)
    assert np.abs(a[0] - b[0]).max() <= 1e-4 * sc.rgb.max() + 1e-15
    assert (oa[0].n_walk < ob[0].n_walk).sum() > 20  # termination actually happened


def test_transmittance_monotone(oracle_lib):
    """Rendering growing prefixes of one pixel's list gives non-increasing T (tau non-decreasing)."""
    O = oracle_lib
    sc = synth.make_scene(200, seed=14, center_half=0.5, n_sigma=8)
    cam = synth.look_at_camera((0.0, 0.0, 4.0), (0, 0, 0), 32, 32)
    rec = O.key_project(sc, cam)
    lst = O.brute_force_list(rec)
    pix = np.array([16 * 32 + 16], np.int32)
    taus = []
    for L in range(0, len(lst) + 1, 5):
        out = O.render_pixels(sc, cam, pix, np.zeros(1, np.int32), np.array([0, L], np.int64), lst, t_min=0.0)
        taus.append(out.tau[0])
    assert np.all(np.diff(taus) >= 0) and taus[-1] > 0


def test_color_mlp_matches_torch_functional(oracle_lib):
    O = oracle_lib
    sc = synth.make_scene(10, seed=15, color="mlp", n_c=32)
    rng = np.random.default_rng(0)
    for i in range(sc.n):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        z0 = torch.tensor(np.concatenate([d, sc.feat[i]]), dtype=torch.float64)
        t = lambda a: torch.tensor(a, dtype=torch.float64)
        z1 = torch.nn.functional.relu(torch.nn.functional.linear(z0, t(sc.Wc1[i]), t(sc.bc1[i])))
        z2 = torch.nn.functional.relu(torch.nn.functional.linear(z1, t(sc.Wc2[i]), t(sc.bc2[i])))
        ref = torch.sigmoid(torch.nn.functional.linear(z2, t(sc.Wc3[i]), t(sc.bc3[i]))).numpy()
        got = O.color(sc, i, d)
        assert np.abs(got - ref).max() < 1e-15
        assert np.all((got > 0) & (got < 1))


def test_paper_parameter_counts():
    """App. C: an 8-neuron density MLP has 41 parameters; geometry 10 (3 + 3 + 4)."""
    path = __file__.replace("test_oracle_render.py", "golden/paper_param_counts.txt")
    vals = {}
    for line in open(path):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split("=")
            vals[k.strip()] = int(v)
    sc = synth.make_scene(1, seed=0, n_sigma=vals["n_sigma"])
    n_mlp = sc.W1[0].size + sc.b1[0].size + sc.w2[0].size + 1
    n_geo = sc.centers[0].size + sc.log_scales[0].size + sc.quats[0].size
    assert n_mlp == vals["density_mlp_params"]
    assert n_geo == vals["geometry_params"]
    assert n_mlp + n_geo + vals["sh_params"] == vals["total_params"]
