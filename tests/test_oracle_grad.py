"""Pins for the FP64 gradient oracle (oracle/grad.py).

Its forward must equal the C oracle's forward, and its reverse-mode gradient must
equal central finite differences of the C oracle's forward, on a
2,000-primitive, 64 x 64 scene with the workload's distributions (N_sigma = 16,
colour MLP N_c = 32, camera on the radius-8 ring), early termination off.
Candidate lists are held fixed (they are the key specification's output, not a
differentiable quantity); a direction whose +h / -h renders change the number of
composited pairs (a hit or a sign of alpha_hat flipped) is skipped, and the
perturbed primitives exclude those with a pair near a kink of the forward (a
grazing ray |h^2| < 1e-3, |alpha_hat| < 1e-4, a colour-MLP pre-activation within
1e-4 of the ReLU kink, or a near-tie in argmax s).  Step: h = 1e-4 for density
weights and constant colours, 1e-6 for colour-MLP weights, 1e-5 for geometry (centres, log-scales,
quaternions), whose chord length has a square-root singularity at grazing rays;
perturbations are exact (float64 scene) and the central differences are
Richardson-extrapolated (h and h/2), so the comparison is at 1e-6.
"""
import numpy as np
import pytest

from paper_2510_08491_gb300 import synth


def _setup(O, n=2000, color="mlp", seed=0, res=64):
    """color "<mode>+t": a time-conditioned scene seen at time 0.6."""
    dyn = color.endswith("+t")
    color = color.split("+")[0]
    sc = synth.make_scene(n, seed=seed, center_half=3.0, n_sigma=16, omega0=5.0, color=color, n_c=32,
                          dynamic=dyn)
    cam = synth.ring_cameras(1, 8.0, res, res)[0]
    if dyn:
        cam.time = np.float32(0.6)
    ts = 16
    tl = O.tile_keys(sc, [cam], ts)
    pix = np.arange(cam.n_pixels, dtype=np.int32)
    gtile = O.pixel_tile(cam, ts, pix)
    lp = (tl.vals.astype(np.int64) % sc.n).astype(np.int32)
    dL = np.random.default_rng(seed + 100).normal(size=(len(pix), 3))
    return sc, cam, pix, gtile, tl.tile_off, lp, dL


GEOM = ("centers", "log_scales", "quats")
COLOR_MLP = ("feat", "Wc1", "bc1", "Wc2", "bc2", "Wc3", "bc3")


def _step(f):
    if f in GEOM:
        return 1e-5
    if f in COLOR_MLP:
        return 1e-6
    return 1e-4


def _safe_prims(sc, cam, pix, gtile, off, lp, g):
    """Composited primitives with no pair near a kink of the forward."""
    from oracle import grad as G
    prim, h2, ah, amin = G.pair_diagnostics(sc, cam, pix, gtile, off, lp)
    bad = (np.abs(h2) < 1e-3) | ((h2 > 0) & (np.abs(ah) < 1e-4)) | ((h2 > 0) & (ah > 0) & (amin < 1e-4))
    badp = np.zeros(sc.n, bool)
    badp[prim[bad]] = True
    s = np.sort(sc.log_scales.astype(np.float64), axis=1)
    badp |= (s[:, 2] - s[:, 1]) < 1e-3
    live = np.abs(g["b2"]) > 0
    return np.nonzero(live & ~badp)[0]


def _loss(O, sc, cam, pix, gtile, off, lp, dL, cs=None):
    out = O.render_pixels(sc, cam, pix, gtile, off, lp, t_min=0.0, cs=cs)
    return float((out.rgb * dL).sum()), out.n_comp


@pytest.mark.parametrize("color", ["const", "mlp", "sh", "sh+t"])
def test_torch_forward_equals_c_forward(oracle_lib, color):
    O = oracle_lib
    from oracle import grad as G
    sc, cam, pix, gtile, off, lp, dL = _setup(O, n=2000, color=color)
    ref = O.render_pixels(sc, cam, pix, gtile, off, lp, t_min=1e-4)
    params = G.scene_tensors(sc, requires_grad=False)
    rgb = G.render(params, sc, cam, pix, gtile, off, lp, t_min=1e-4).numpy()
    ok = ref.flags == 0
    assert np.abs(rgb[ok] - ref.rgb[ok]).max() < 1e-12
    assert ref.n_comp > 500


def _fd(O, sc, f, base, delta, cam, pix, gtile, off, lp, dL):
    """Richardson-extrapolated central difference of L along `delta` (float64, exact
    perturbations): (4 D(h/2) - D(h)) / 3 cancels the h^2 truncation term.  Returns
    (estimate of grad . delta, whether any hit/sign flipped)."""
    vals, ncs = [], []
    for sgn, scl in ((1, 1.0), (-1, 1.0), (1, 0.5), (-1, 0.5)):
        setattr(sc, f, base + sgn * scl * delta)
        l, nc = _loss(O, sc, cam, pix, gtile, off, lp, dL)
        vals.append(l)
        ncs.append(nc)
    setattr(sc, f, base)
    d1 = (vals[0] - vals[1]) / 2.0
    d2 = (vals[2] - vals[3])
    return (4.0 * d2 - d1) / 3.0, len(set(ncs)) > 1


def _fd_group_directions(O, G, color, n_dirs, seed):
    sc, cam, pix, gtile, off, lp, dL = _setup(O, color=color)
    _, g = G.grads(sc, cam, pix, gtile, off, lp, dL, t_min=0.0)
    for f in sc.fields():
        setattr(sc, f, getattr(sc, f).astype(np.float64))
    rng = np.random.default_rng(seed)
    checked = skipped = 0
    worst = 0.0
    live = _safe_prims(sc, cam, pix, gtile, off, lp, g)
    for f in sc.fields():
        base = getattr(sc, f)
        h = _step(f)
        if not np.any(g[f]):
            continue  # e.g. constant colours when the colour MLP is on
        for _ in range(n_dirs):
            # Rademacher direction on every scalar of 40 random composited primitives
            v = np.zeros(base.shape)
            sub = rng.choice(live, size=40, replace=False)
            v[sub] = rng.choice([-1.0, 1.0], size=(40,) + base.shape[1:])
            fd, flipped = _fd(O, sc, f, base, h * v, cam, pix, gtile, off, lp, dL)
            if flipped:
                skipped += 1
                continue
            an = float((g[f] * h * v).sum())
            scale = np.sqrt((g[f] ** 2).mean()) * h * np.abs(v).sum()
            err = abs(fd - an) / (abs(an) + scale + 1e-300)
            worst = max(worst, err)
            checked += 1
    return checked, skipped, worst


@pytest.mark.parametrize("color", ["const", "mlp", "sh", "const+t", "sh+t"])
def test_gradient_matches_fd_directional(oracle_lib, color):
    O = oracle_lib
    from oracle import grad as G
    checked, skipped, worst = _fd_group_directions(O, G, color, 4, 1)
    assert checked >= 3 * skipped
    assert worst < 1e-6, worst


def test_gradient_matches_fd_scalars(oracle_lib):
    O = oracle_lib
    from oracle import grad as G
    sc, cam, pix, gtile, off, lp, dL = _setup(O, color="mlp")
    _, g = G.grads(sc, cam, pix, gtile, off, lp, dL, t_min=0.0)
    for f in sc.fields():
        setattr(sc, f, getattr(sc, f).astype(np.float64))
    rng = np.random.default_rng(7)
    # scalars of primitives that are composited somewhere (others have zero gradient)
    live = _safe_prims(sc, cam, pix, gtile, off, lp, g)
    assert len(live) > 50
    checked = 0
    for _ in range(300):
        f = sc.fields()[rng.integers(len(sc.fields()))]
        if not np.any(g[f]):
            continue
        h = _step(f)
        base = getattr(sc, f)
        i = live[rng.integers(len(live))]
        j = tuple(rng.integers(s) for s in base.shape[1:])
        delta = np.zeros(base.shape)
        delta[(i,) + j] = h
        fd, flipped = _fd(O, sc, f, base, delta, cam, pix, gtile, off, lp, dL)
        if flipped:
            continue
        fd /= h
        an = g[f][(i,) + j]
        rms = np.sqrt((g[f] ** 2).mean())
        assert abs(fd - an) <= 1e-6 * (abs(an) + rms), (f, i, j, fd, an)
        checked += 1
    assert checked > 200
