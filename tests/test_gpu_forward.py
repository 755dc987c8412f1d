"""GPU parity of the forward path through the C ABI against the FP64 oracle.

Tile keys and their order must match the oracle's FP32 key specification bit for
bit; images must match the FP64 oracle within 1e-4 per RGB channel.
"""
import numpy as np
import pytest
import torch

from paper_2510_08491_gb300 import synth
from gpu_util import IMG_TOL, assert_image_close, oracle_images

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2510_08491_gb300 import build
    build.build()
    from paper_2510_08491_gb300.render import Renderer
    return Renderer(0)


def _render(R, scene, cams, **cfg):
    from paper_2510_08491_gb300 import _lib as L
    from paper_2510_08491_gb300.render import pack_scene
    ps = pack_scene(scene)
    img = R.forward(ps, cams, L.make_config(**cfg))
    torch.cuda.synchronize()
    return img.cpu().numpy(), ps


def test_tiny_keys_and_image(R, oracle_lib):
    O = oracle_lib
    wl = synth.workload("tiny64_128px")
    img, _ = _render(R, wl.scene, wl.cameras)
    keys, vals = R.debug_keys()
    ref, flags, tl, _ = oracle_images(O, wl.scene, wl.cameras)
    assert np.array_equal(keys, tl.keys)
    assert np.array_equal(vals, tl.vals)
    assert_image_close(img, ref, flags)
    st = R.stats()
    assert st.n_keys == len(tl.keys) and st.n_composited > 1000


@pytest.mark.parametrize("form", [0, 1])
def test_mlp_multiview_ragged(R, oracle_lib, form):
    """Colour MLP, N_sigma = 16, three views with sizes that leave partial edge tiles."""
    O = oracle_lib
    sc = synth.make_scene(3000, seed=4, center_half=3.0, n_sigma=16, omega0=5.0, color="mlp", n_c=32)
    cams = [synth.look_at_camera((0.0, 1.0, 8.0), (0, 0, 0), 203, 150),
            synth.look_at_camera((8.0, 0.0, 0.5), (0, 0, 0), 96, 77),
            synth.look_at_camera((-5.0, 3.0, -6.0), (0, 0, 0), 161, 33)]
    img, _ = _render(R, sc, cams, form=form)
    keys, vals = R.debug_keys()
    ref, flags, tl, _ = oracle_images(O, sc, cams, form=form)
    assert np.array_equal(keys, tl.keys)
    assert np.array_equal(vals, tl.vals)
    if form == 0:
        assert_image_close(img, ref, flags)
    else:
        # Eq. 8 literally: the phases are measured from the camera (|psi| ~ w0 |W1| |eye - c| / m, hundreds
        # of radians, FP32 ulp ~3e-5 rad) and divided by a_k = w0 W1_k . d / m, which is unbounded as
        # W1_k . d -> 0; the literal form is checked statistically and its outliers are what the stable
        # form removes.
        err = np.abs(img.astype(np.float64) - ref).max(axis=1)
        assert err.mean() < 2e-6 and np.quantile(err, 0.999) < 1e-3, (err.mean(), np.quantile(err, 0.999))


def test_mlp64_ns32_bf16(R, oracle_lib):
    O = oracle_lib
    sc = synth.make_scene(1500, seed=5, center_half=3.0, n_sigma=32, omega0=5.0, color="mlp", n_c=64).to_bf16()
    cams = synth.ring_cameras(2, 10.0, 180, 120)
    img, ps = _render(R, sc, cams)
    assert ps.net.dtype == torch.bfloat16
    ref, flags, tl, _ = oracle_images(O, sc, cams)
    keys, vals = R.debug_keys()
    assert np.array_equal(keys, tl.keys) and np.array_equal(vals, tl.vals)
    assert_image_close(img, ref, flags)


def test_background_and_no_termination(R, oracle_lib):
    O = oracle_lib
    sc = synth.make_scene(400, seed=6, center_half=1.0, n_sigma=8)
    sc.b2[:] = 2.0
    cams = [synth.look_at_camera((0.0, 0.0, 4.0), (0, 0, 0), 100, 90)]
    for t_min in (0.0, 1e-2):
        img, _ = _render(R, sc, cams, t_min=t_min, bg=(0.25, 0.5, 1.0))
        ref, flags, _, _ = oracle_images(O, sc, cams, t_min=t_min, bg=(0.25, 0.5, 1.0))
        assert_image_close(img, ref, flags)


def test_empty_scene_and_all_culled(R, oracle_lib):
    sc = synth.make_scene(50, seed=7, center_half=1.0)
    cams = [synth.look_at_camera((0.0, 0.0, 4.0), (0, 0, 0), 40, 24)]
    img, _ = _render(R, sc.subset(np.arange(0)), cams, bg=(0.1, 0.2, 0.3))
    assert np.allclose(img, [0.1, 0.2, 0.3])
    far = sc.copy()
    far.centers[:, 2] = 10.0  # behind the camera at z = 4 looking down -z
    img, _ = _render(R, far, cams, bg=(0.1, 0.2, 0.3))
    assert np.allclose(img, [0.1, 0.2, 0.3])
    assert R.stats().n_keys == 0


def test_full_size_fwd100k_keys_and_sampled_pixels(R, oracle_lib):
    """The 100k-primitive, four-view 1920 x 1080 workload: full key arrays bit-exact,
    2,000 sampled pixels per view against the oracle."""
    O = oracle_lib
    wl = synth.workload("fwd100k_1080p_4view")
    img, _ = _render(R, wl.scene, wl.cameras)
    keys, vals = R.debug_keys()
    cs = O.CScene(wl.scene)
    tl = O.tile_keys(wl.scene, wl.cameras, 16, cs)
    assert np.array_equal(keys, tl.keys)
    assert np.array_equal(vals, tl.vals)
    rng = np.random.default_rng(0)
    off = 0
    for v, cam in enumerate(wl.cameras):
        pix = rng.choice(cam.n_pixels, size=2000, replace=False).astype(np.int32)
        out = O.render_view_tiled(wl.scene, wl.cameras, v, tl, 16, pix, cs=cs)
        assert_image_close(img[off + pix], out.rgb, out.flags)
        off += cam.n_pixels
