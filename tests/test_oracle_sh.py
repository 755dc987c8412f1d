"""Pins of the oracle's spherical-harmonic colour (the view-dependent colour of
Sec. 3.1, four bands): the basis against properties the mathematics fixes, and
the colour against its definition.

* Orthonormality: int_S2 Y_i Y_j = delta_ij, by a product quadrature that is exact
  for these polynomials (Gauss-Legendre in cos(theta) x uniform in phi).
* Addition theorem, per band l: sum_m Y_lm(u) Y_lm(w) = (2l + 1) / (4 pi) P_l(u . w),
  which fixes every constant and sign inside a band up to a common orthogonal map.
* Against scipy's complex harmonics: the real (tesseral) form
  Y_lm = sqrt(2) (-1)^m Re Y_l^m (m > 0), Y_l0, sqrt(2) (-1)^m Im Y_l^|m| (m < 0),
  at index l^2 + l + m; the (-1)^m cancels scipy's Condon-Shortley phase, so every
  constant is positive.  This fixes the order and sign of each function inside a band,
  which the two properties above leave open.
* The C and torch (gradient) oracles evaluate the same basis.
"""
import math

import numpy as np
import pytest
import torch

from paper_2510_08491_gb300 import synth


def _sphere_quadrature(n_t=10, n_p=24):
    x, wx = np.polynomial.legendre.leggauss(n_t)
    ph = 2 * np.pi * np.arange(n_p) / n_p
    ct, phi = np.meshgrid(x, ph, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    v = np.stack([st * np.cos(phi), st * np.sin(phi), ct], -1).reshape(-1, 3)
    w = (wx[:, None] * np.full(n_p, 2 * np.pi / n_p)[None]).reshape(-1)
    return v, w


def test_basis_is_orthonormal(oracle_lib):
    O = oracle_lib
    v, w = _sphere_quadrature()
    Y = np.stack([O.sh_basis(x) for x in v])
    gram = (Y * w[:, None]).T @ Y
    assert np.abs(gram - np.eye(16)).max() < 1e-12


def test_addition_theorem_per_band(oracle_lib):
    O = oracle_lib
    rng = np.random.default_rng(3)
    P = [lambda t: 1.0, lambda t: t, lambda t: 0.5 * (3 * t * t - 1), lambda t: 0.5 * (5 * t ** 3 - 3 * t)]
    for _ in range(20):
        u, w = rng.normal(size=3), rng.normal(size=3)
        u /= np.linalg.norm(u)
        w /= np.linalg.norm(w)
        Yu, Yw = O.sh_basis(u), O.sh_basis(w)
        for l in range(4):
            band = slice(l * l, (l + 1) * (l + 1))
            lhs = float(Yu[band] @ Yw[band])
            rhs = (2 * l + 1) / (4 * math.pi) * P[l](float(u @ w))
            assert abs(lhs - rhs) < 1e-13


def test_basis_is_the_real_form_of_scipys_harmonics(oracle_lib):
    from scipy.special import sph_harm_y
    O = oracle_lib
    rng = np.random.default_rng(7)
    for _ in range(40):
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        theta, phi = math.acos(v[2]), math.atan2(v[1], v[0])
        Y = O.sh_basis(v)
        for l in range(4):
            for m in range(-l, l + 1):
                c = complex(sph_harm_y(l, abs(m), theta, phi))
                if m > 0:
                    ref = math.sqrt(2) * (-1) ** m * c.real
                elif m < 0:
                    ref = math.sqrt(2) * (-1) ** m * c.imag
                else:
                    ref = c.real
                assert abs(Y[l * l + l + m] - ref) < 1e-13, (l, m)


def test_torch_basis_equals_c_basis(oracle_lib):
    O = oracle_lib
    from oracle import grad as G
    rng = np.random.default_rng(5)
    v = rng.normal(size=(50, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    ref = np.stack([O.sh_basis(x) for x in v])
    got = G.sh_basis(torch.tensor(v)).numpy()
    assert np.abs(got - ref).max() < 1e-15


def test_colour_is_clamped_half_plus_expansion(oracle_lib):
    O = oracle_lib
    sc = synth.make_scene(20, seed=9, color="sh")
    eye = np.array([0.3, -0.2, 5.0])
    for i in range(sc.n):
        v = sc.centers[i].astype(np.float64) - eye
        v /= np.linalg.norm(v)
        want = np.maximum(0.0, 0.5 + O.sh_basis(v) @ sc.sh[i].astype(np.float64))
        got = O.color(sc, i, np.array([0.0, 0.0, 1.0]), eye=eye)
        assert np.abs(got - want).max() < 1e-15


def test_zero_coefficients_give_grey(oracle_lib):
    O = oracle_lib
    sc = synth.make_scene(5, seed=1, color="sh")
    sc.sh[:] = 0.0
    for i in range(sc.n):
        assert np.array_equal(O.color(sc, i, np.array([1.0, 0.0, 0.0]), eye=(0, 0, 4)), np.full(3, 0.5))
