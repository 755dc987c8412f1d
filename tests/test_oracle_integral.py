"""Pins for the oracle's ray/ellipsoid intersection and closed-form integral (Sec. 3.2).

Each check compares the oracle with something other than itself: adaptive
quadrature of the density of Eq. 5/6 (Eq. 2's discretisation used as a check),
an independent rotation routine (scipy), textbook special cases and the
fundamental theorem of calculus (Eq. 7).
"""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.spatial.transform import Rotation

from paper_2510_08491_gb300 import synth


def sigma_eq56(sc, i, x):
    """Density of Eq. 5/6 evaluated directly at world point x (float64)."""
    s = np.exp(sc.log_scales[i].astype(np.float64))
    u = (x - sc.centers[i].astype(np.float64)) / s.max()
    W1 = sc.W1[i].astype(np.float64)
    h = np.cos(sc.omega0 * (W1 @ u + sc.b1[i].astype(np.float64)))
    return float(sc.w2[i].astype(np.float64) @ h + float(sc.b2[i]))


def ellipsoid_roots(sc, i, o, d):
    """Entry/exit of o + t d with {c + R diag(s) v : |v| <= 1} via the raw quadratic."""
    q = sc.quats[i].astype(np.float64)
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    s = np.exp(sc.log_scales[i].astype(np.float64))
    M = (R.T) / s[:, None]
    a = M @ d
    b = M @ (o - sc.centers[i].astype(np.float64))
    A, B, Cc = a @ a, 2 * a @ b, b @ b - 1.0
    disc = B * B - 4 * A * Cc
    if disc <= 0:
        return None
    r = math.sqrt(disc)
    return (-B - r) / (2 * A), (-B + r) / (2 * A)


def rays_through(sc, i, rng, n, o):
    """Rays from o aimed at random points inside primitive i."""
    q = sc.quats[i].astype(np.float64)
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    s = np.exp(sc.log_scales[i].astype(np.float64))
    out = []
    for _ in range(n):
        v = rng.normal(size=3)
        v *= rng.uniform() ** (1 / 3) / np.linalg.norm(v) * 0.999
        x = sc.centers[i].astype(np.float64) + R @ (s * v)
        d = x - o
        out.append(d / np.linalg.norm(d))
    return out


@pytest.mark.parametrize("omega0,thin,ns", [(5.0, None, 8), (30.0, None, 16), (30.0, 50.0, 16), (5.0, 50.0, 32)])
def test_integral_matches_quadrature(oracle_lib, omega0, thin, ns):
    O = oracle_lib
    sc = synth.make_scene(12, seed=11, center_half=1.0, n_sigma=ns, omega0=omega0, thin_ratio_max=thin)
    rng = np.random.default_rng(5)
    o = np.array([0.3, -0.2, 4.0])
    cs = O.CScene(sc)
    worst = 0.0
    for i in range(sc.n):
        for d in rays_through(sc, i, rng, 6, o):
            hit, t0, t1, ah = O.pair(sc, i, o, d, O.FORM_STABLE, cs)
            roots = ellipsoid_roots(sc, i, o, d)
            assert hit and roots is not None
            assert abs(t0 - roots[0]) < 1e-9 and abs(t1 - roots[1]) < 1e-9
            f = lambda t: sigma_eq56(sc, i, o + t * d)
            ref, err = integrate.quad(f, t0, t1, epsabs=1e-13, epsrel=1e-12, limit=400)
            scale = (t1 - t0) * (abs(float(sc.b2[i])) + np.abs(sc.w2[i]).sum())
            worst = max(worst, abs(ah - ref) / scale)
    assert worst < 1e-10, worst


def test_entry_exit_on_surface(oracle_lib):
    O = oracle_lib
    sc = synth.make_scene(20, seed=3, thin_ratio_max=50.0)
    rng = np.random.default_rng(1)
    o = np.array([0.0, 0.0, 4.0])
    for i in range(sc.n):
        q = sc.quats[i].astype(np.float64)
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        s = np.exp(sc.log_scales[i].astype(np.float64))
        for d in rays_through(sc, i, rng, 4, o):
            hit, t0, t1, _ = O.pair(sc, i, o, d)
            for t in (t0, t1):
                v = (R.T @ (o + t * d - sc.centers[i].astype(np.float64))) / s
                assert abs(np.linalg.norm(v) - 1.0) < 1e-12


def test_sphere_constant_density_chord(oracle_lib):
    """W1 = 0 gives constant sigma = sum w2 cos(w0 b1) + b2; a sphere's chord is 2 sqrt(r^2 - p^2)."""
    O = oracle_lib
    sc = synth.make_scene(1, seed=2, n_sigma=8, omega0=5.0)
    sc.log_scales[:] = np.float32(math.log(0.25))
    sc.centers[:] = np.float32([0.1, -0.05, 0.2])
    sc.W1[:] = 0.0
    r = math.exp(float(sc.log_scales[0, 0]))
    sig = float(np.sum(sc.w2[0].astype(np.float64) * np.cos(5.0 * sc.b1[0].astype(np.float64))) + sc.b2[0])
    o = np.array([0.0, 0.0, 3.0])
    c = sc.centers[0].astype(np.float64)
    rng = np.random.default_rng(0)
    for _ in range(50):
        target = c + rng.uniform(-0.2, 0.2, size=3)
        d = (target - o) / np.linalg.norm(target - o)
        p = np.linalg.norm(np.cross(c - o, d))
        hit, t0, t1, ah = O.pair(sc, 0, o, d)
        if p < r:
            chord = 2 * math.sqrt(r * r - p * p)
            assert hit
            assert abs((t1 - t0) - chord) < 1e-12
            assert abs(ah - sig * chord) < 1e-12
        else:
            assert not hit


def test_zero_amplitudes_give_b2_times_chord(oracle_lib):
    O = oracle_lib
    sc = synth.make_scene(5, seed=4, n_sigma=16, omega0=30.0)
    sc.w2[:] = 0.0
    o = np.array([0.0, 0.2, 4.0])
    rng = np.random.default_rng(2)
    for i in range(sc.n):
        for d in rays_through(sc, i, rng, 3, o):
            hit, t0, t1, ah = O.pair(sc, i, o, d)
            assert abs(ah - float(sc.b2[i]) * (t1 - t0)) < 1e-14


def test_zero_directional_frequency_limit(oracle_lib):
    """W1_k . d = 0 makes Eq. 8's division 0/0; the limit is w2_k cos(phi_k) Delta_t."""
    O = oracle_lib
    sc = synth.make_scene(1, seed=9, n_sigma=4, omega0=30.0)
    o = np.array([0.0, 0.0, 4.0])
    c = sc.centers[0].astype(np.float64)
    d = (c - o) / np.linalg.norm(c - o)
    # make every row orthogonal to d (float32-exact orthogonality is not needed: use the limit bound)
    basis = np.linalg.svd(d[None])[2][1:]
    for k in range(4):
        sc.W1[0, k] = (basis[k % 2] * (1.0 + k)).astype(np.float32)
    hit, t0, t1, ah = O.pair(sc, 0, o, d)
    assert hit
    s = np.exp(sc.log_scales[0].astype(np.float64))
    m = s.max()
    tm = 0.5 * (t0 + t1)
    u = (o + tm * d - c) / m
    W1 = sc.W1[0].astype(np.float64)
    a = 30.0 * (W1 @ d) / m
    assert np.all(np.abs(a) < 1e-5)
    lim = (t1 - t0) * (float(sc.b2[0]) + np.sum(sc.w2[0] * np.cos(30.0 * (W1 @ u + sc.b1[0]))))
    # residual |a| Delta_t is ~1e-6: sinc deviates by (a Delta_t / 2)^2 / 6 at most
    assert abs(ah - lim) < 1e-10
    assert math.isfinite(ah)


def test_stable_equals_naive_when_well_conditioned(oracle_lib):
    O = oracle_lib
    sc = synth.make_scene(30, seed=21, n_sigma=16, omega0=30.0)
    o = np.array([0.5, 0.1, 4.0])
    rng = np.random.default_rng(3)
    cs = O.CScene(sc)
    n_checked = 0
    for i in range(sc.n):
        s = np.exp(sc.log_scales[i].astype(np.float64))
        for d in rays_through(sc, i, rng, 4, o):
            hit, t0, t1, ah_s = O.pair(sc, i, o, d, O.FORM_STABLE, cs)
            a = 30.0 * (sc.W1[i].astype(np.float64) @ d) / s.max()
            if np.min(np.abs(a)) * (t1 - t0) <= 1e-2:
                continue
            _, _, _, ah_n = O.pair(sc, i, o, d, O.FORM_NAIVE, cs)
            scale = (t1 - t0) * (1 + np.abs(sc.w2[i]).sum())
            assert abs(ah_s - ah_n) / scale < 1e-11
            n_checked += 1
    assert n_checked > 50


def test_fundamental_theorem(oracle_lib):
    """d/dt1 of the integral over [t0, t1] is sigma(o + t1 d); d/dt0 is -sigma(o + t0 d) (Eq. 7)."""
    O = oracle_lib
    sc = synth.make_scene(6, seed=8, n_sigma=16, omega0=5.0)
    o = np.array([0.0, 0.0, 4.0])
    rng = np.random.default_rng(4)
    cs = O.CScene(sc)
    for i in range(sc.n):
        for d in rays_through(sc, i, rng, 2, o):
            _, t0, t1, _ = O.pair(sc, i, o, d, O.FORM_STABLE, cs)
            h = 1e-5
            for form in (O.FORM_STABLE, O.FORM_NAIVE):
                g1 = (O.integral(sc, i, o, d, t0, t1 + h, form, cs) - O.integral(sc, i, o, d, t0, t1 - h, form, cs)) / (2 * h)
                g0 = (O.integral(sc, i, o, d, t0 + h, t1, form, cs) - O.integral(sc, i, o, d, t0 - h, t1, form, cs)) / (2 * h)
                assert abs(g1 - sigma_eq56(sc, i, o + t1 * d)) < 1e-6
                assert abs(g0 + sigma_eq56(sc, i, o + t0 * d)) < 1e-6
