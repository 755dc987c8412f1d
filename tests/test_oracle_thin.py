"""The precision-stress workload (thin primitives, omega0 = 30) is built so that
at least 10% of the ray/primitive hit pairs have min_k |W1_k . d| < 1e-4 (the
directional frequency Eq. 8 divides by).  Measured with the oracle's geometry on
64 seeded 16 x 16 tiles of the 1920 x 1080 view."""
import numpy as np

from paper_2510_08491_gb300 import synth


def test_thin_workload_hits_near_zero_directional_frequency(oracle_lib):
    from oracle import grad as G
    O = oracle_lib
    wl = synth.workload("thin50k_1080p")
    sc, cam = wl.scene, wl.cameras[0]
    tl = O.tile_keys(sc, [cam], 16)
    lp = (tl.vals.astype(np.int64) % sc.n).astype(np.int32)
    rng = np.random.default_rng(0)
    tx_n, ty_n = O.tiles_xy(cam, 16)
    pix = []
    for t in rng.choice(tx_n * ty_n, size=64, replace=False):
        ty, tx = divmod(int(t), tx_n)
        ys, xs = np.mgrid[ty * 16:min(ty * 16 + 16, cam.height), tx * 16:min(tx * 16 + 16, cam.width)]
        pix.append((ys * cam.width + xs).ravel())
    pix = np.concatenate(pix).astype(np.int32)
    gt = tl.view_tile_off[0] + O.pixel_tile(cam, 16, pix)
    _, h2, _, _ = G.pair_diagnostics(sc, cam, pix, gt, tl.tile_off, lp)
    mwd = G.min_direction_dot(sc, cam, pix, gt, tl.tile_off, lp)
    hit = h2 > 0
    assert hit.sum() > 10000
    frac = float((mwd[hit] < 1e-4).mean())
    print(f"hit pairs {hit.sum()}, share with min_k |W1_k . d| < 1e-4: {frac:.3f}")
    assert frac >= 0.10


def test_min_direction_dot_matches_direct_evaluation(oracle_lib):
    """Independent restatement on a few pairs: |W1_k . d| with d the unit pixel ray."""
    from oracle import grad as G
    sc = synth.make_scene(50, seed=2, n_sigma=4)
    cam = synth.look_at_camera((0.0, 0.0, 4.0), (0, 0, 0), 32, 24)
    pix = np.array([0, 17, 300, 767], np.int32)
    lists = np.array([0, 3, 9, 49, 7], np.int32)
    off = np.array([0, 2, 3, 5, 5], np.int64)
    got = G.min_direction_dot(sc, cam, pix, np.arange(4, dtype=np.int32), off, lists)
    want = []
    for i, p in enumerate(pix):
        px, py = p % cam.width, p // cam.width
        r = (px + 0.5 - cam.cx) / cam.fx * np.asarray(cam.R_wc[0], np.float64) + \
            (py + 0.5 - cam.cy) / cam.fy * np.asarray(cam.R_wc[1], np.float64) + np.asarray(cam.R_wc[2], np.float64)
        r /= np.linalg.norm(r)
        for j in range(off[i], off[i + 1]):
            want.append(np.abs(np.asarray(sc.W1[lists[j]], np.float64) @ r).min())
    assert np.allclose(got, want, rtol=1e-14, atol=0)
