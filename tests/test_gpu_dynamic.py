"""GPU parity of time-conditioned scenes (App. Applications, volumetric dynamic
scenes) against the FP64 oracle: views at different timestamps, the density's
phase shifted by xi W_t and, with SH colour, the degree-0 time series; images
(FP32 and BF16 weights, both integral forms), tile keys, and gradients of every
parameter group including W_t and the series coefficients."""
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


def _scene(color, n=2500, seed=31, bf16=False, omega0=30.0):
    sc = synth.make_scene(n, seed=seed, center_half=2.0, n_sigma=8, omega0=omega0, color=color, dynamic=True)
    return sc.to_bf16() if bf16 else sc


def _cams(times, w=88, h=72):
    cams = synth.ring_cameras(len(times), 7.0, w, h)
    for c, t in zip(cams, times):
        c.time = np.float32(t)
    return cams


@pytest.mark.parametrize("color,bf16,form", [("sh", False, 0), ("sh", True, 0), ("const", False, 0),
                                             ("sh", False, 1)])
def test_dynamic_images_match_oracle(R, oracle_lib, color, bf16, form):
    from paper_2510_08491_gb300 import _lib as L
    from paper_2510_08491_gb300.render import pack_scene
    O = oracle_lib
    # the literal Eq. 8 divides by w0 W1_k . d / m and loses FP32 accuracy where that
    # is small (the precision-stress workload measures it, and no test holds it to
    # the stable form's bar); here it only has to show that the time shift reaches
    # it too: w0 = 5 and a 5e-4 bar
    sc = _scene(color, bf16=bf16, omega0=30.0 if form == 0 else 5.0)
    cams = _cams([0.0, 0.5, 1.0])
    img = R.forward(pack_scene(sc), cams, L.make_config(form=form)).cpu().numpy()
    keys, vals = R.debug_keys()
    ref, flags, tl, _ = oracle_images(O, sc, cams, form=form)
    assert np.array_equal(keys, tl.keys) and np.array_equal(vals, tl.vals)
    if form == 0:
        assert_image_close(img, ref, flags)
    else:
        assert_image_close(img, ref, flags, tol=5e-4, tol_flagged=5e-4)


def test_time_changes_the_image_static_ignores_it(R):
    from paper_2510_08491_gb300 import _lib as L
    from paper_2510_08491_gb300.render import pack_scene
    sc = _scene("sh", n=1500)
    ps = pack_scene(sc)
    a = R.forward(ps, _cams([0.2]), L.make_config()).cpu().numpy()
    b = R.forward(ps, _cams([0.7]), L.make_config()).cpu().numpy()
    assert np.abs(a - b).max() > 1e-2
    st = synth.make_scene(1500, seed=31, center_half=2.0, n_sigma=8, omega0=30.0, color="sh")
    ps = pack_scene(st)
    c = R.forward(ps, _cams([0.2]), L.make_config()).cpu().numpy()
    d = R.forward(ps, _cams([0.7]), L.make_config()).cpu().numpy()
    assert np.array_equal(c, d)


@pytest.mark.parametrize("color", ["sh", "const"])
def test_dynamic_gradients_match_oracle(R, oracle_lib, color):
    from test_gpu_backward import _check, _dl, _gpu_grads, _oracle_grads
    O = oracle_lib
    sc = _scene(color, n=1500, seed=37)
    cams = [synth.look_at_camera((0.0, 0.5, 6.0), (0, 0, 0), 72, 56),
            synth.look_at_camera((5.0, 1.0, 2.0), (0, 0, 0), 64, 48)]
    cams[0].time, cams[1].time = np.float32(0.3), np.float32(0.85)
    # no silhouette mask: grazing pairs (|h^2| < 1e-2) are evaluated in float-float
    dLv = _dl(O, sc, cams, 8)
    g = _gpu_grads(R, sc, cams, np.concatenate(dLv))
    gref = _oracle_grads(O, sc, cams, dLv)
    fields = ["centers", "log_scales", "quats", "W1", "b1", "w2", "b2", "wt"]
    fields += ["sh", "sh_t"] if color == "sh" else ["rgb"]
    _check(g, gref, fields)


def test_dynamic_with_colour_mlp_is_unsupported(R):
    from paper_2510_08491_gb300 import _lib as L
    from paper_2510_08491_gb300.render import pack_scene
    sc = synth.make_scene(10, seed=1, color="mlp", dynamic=True)
    with pytest.raises(L.SnpError) as e:
        pack_scene(sc)
    assert e.value.status == L.SNP_ERR_UNSUPPORTED
