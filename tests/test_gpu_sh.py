"""GPU parity of the spherical-harmonic colour mode (four bands, evaluated per
(view, primitive) along the camera-to-centre direction) against the FP64 oracle:
tile keys, images over several views (the colour changes with the eye), BF16
weights, and gradients of every parameter group including the coefficients and
the centres (through the direction)."""
import numpy as np
import pytest

from paper_2510_08491_gb300 import synth
from gpu_util import assert_image_close, oracle_images

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2510_08491_gb300 import build
    build.build()
    from paper_2510_08491_gb300.render import Renderer
    return Renderer(0)


def _scene(n=3000, seed=17, bf16=False):
    # the paper's primitive: N_sigma = 8 (41 density parameters), w0 = 30, 48 SH coefficients
    sc = synth.make_scene(n, seed=seed, center_half=2.0, n_sigma=8, omega0=30.0, color="sh")
    return sc.to_bf16() if bf16 else sc


@pytest.mark.parametrize("bf16", [False, True])
def test_sh_images_match_oracle(R, oracle_lib, bf16):
    from paper_2510_08491_gb300 import _lib as L
    from paper_2510_08491_gb300.render import pack_scene
    O = oracle_lib
    sc = _scene(bf16=bf16)
    cams = synth.ring_cameras(3, 7.0, 96, 80)
    img = R.forward(pack_scene(sc), cams, L.make_config()).cpu().numpy()
    keys, vals = R.debug_keys()
    ref, flags, tl, _ = oracle_images(O, sc, cams)
    assert np.array_equal(keys, tl.keys) and np.array_equal(vals, tl.vals)
    assert_image_close(img, ref, flags)


def test_sh_gradients_match_oracle(R, oracle_lib):
    from test_gpu_backward import _check, _dl, _gpu_grads, _oracle_grads
    O = oracle_lib
    sc = _scene(n=1500, seed=23)
    cams = [synth.look_at_camera((0.0, 0.5, 6.0), (0, 0, 0), 72, 56),
            synth.look_at_camera((5.0, 1.0, 2.0), (0, 0, 0), 64, 48)]
    dLv = _dl(O, sc, cams, 6)
    g = _gpu_grads(R, sc, cams, np.concatenate(dLv))
    gref = _oracle_grads(O, sc, cams, dLv)
    _check(g, gref, ["centers", "log_scales", "quats", "W1", "b1", "w2", "b2", "sh"])


@pytest.mark.parametrize("color", ["sh", "const"])
def test_alpha_hat_store_and_replay(R, oracle_lib, monkeypatch, color):
    """Without a colour network the forward stores alpha_hat of every composited pair
    (4 bytes) and the backward reads it instead of evaluating the integral again.
    The stored, the recomputed (SNP_FLAG_REPLAY_COLOR) and a partly stored backward
    (the store capped by the SNP_TEST_COLSTORE_PAIRS hook, so that some chunks are
    recomputed) all match the oracle and each other."""
    from test_gpu_backward import _check, _dl, _gpu_grads_cfg, _oracle_grads
    from paper_2510_08491_gb300.render import pack_scene
    O = oracle_lib
    sc = synth.make_scene(1500, seed=29, center_half=2.0, n_sigma=8, omega0=30.0, color=color)
    cams = [synth.look_at_camera((0.0, 0.5, 6.0), (0, 0, 0), 80, 64),
            synth.look_at_camera((5.0, 1.0, 3.0), (0, 0, 0), 48, 72)]
    dLv = _dl(O, sc, cams, 7)
    fields = ["centers", "log_scales", "quats", "W1", "b1", "w2", "b2", "sh" if color == "sh" else "rgb"]
    gref = _oracle_grads(O, sc, cams, dLv)
    g_store = _gpu_grads_cfg(R, sc, cams, np.concatenate(dLv))
    _check(g_store, gref, fields)
    g_replay = _gpu_grads_cfg(R, sc, cams, np.concatenate(dLv), replay_color=True)
    R.forward(pack_scene(sc), cams)
    total = R.stats().n_composited
    monkeypatch.setenv("SNP_TEST_COLSTORE_PAIRS", str(total // 3))
    g_part = _gpu_grads_cfg(R, sc, cams, np.concatenate(dLv))
    _check(g_part, gref, fields)
    for k in fields:
        scale = np.abs(g_store[k]).max() + 1e-30
        assert np.abs(g_store[k] - g_replay[k]).max() <= 1e-5 * scale, k
        assert np.abs(g_part[k] - g_replay[k]).max() <= 1e-5 * scale, k
