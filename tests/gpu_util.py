"""Helpers shared by the GPU parity tests (CUDA path on one side, oracle on the other)."""
import numpy as np

from paper_2510_08491_gb300 import synth

IMG_TOL = 1e-4  # absolute per RGB channel, FP32 image vs FP64 oracle
IMG_TOL_FLAGGED = 2e-4  # pixels whose termination step FP32 may decide differently


def oracle_images(O, scene, cams, ts=16, t_min=1e-4, bg=(0.0, 0.0, 0.0), form=0):
    imgs, tl, outs = O.render_image(scene, cams, ts, t_min, bg, form)
    flat = np.concatenate([im.reshape(-1, 3) for im in imgs])
    flags = np.concatenate([o.flags for o in outs])
    return flat, flags, tl, outs


def image_errors(gpu, ref, flags):
    err = np.abs(gpu.astype(np.float64) - ref).max(axis=1)
    plain = flags == 0
    return err, plain


def assert_image_close(gpu, ref, flags, tol=IMG_TOL, tol_flagged=IMG_TOL_FLAGGED):
    err, plain = image_errors(gpu, ref, flags)
    worst_plain = err[plain].max() if plain.any() else 0.0
    worst_flag = err[~plain].max() if (~plain).any() else 0.0
    assert worst_plain <= tol, f"max |gpu - oracle| = {worst_plain:.3e} > {tol} (mean {err.mean():.2e})"
    assert worst_flag <= tol_flagged, f"flagged pixels: {worst_flag:.3e} > {tol_flagged}"
    return float(worst_plain), float(err.mean())


def grad_rel_errors(g, g_ref):
    """Per group: max_i |g - g*| / (|g*| + rms(g*)) and ||g - g*|| / ||g*||."""
    out = {}
    for k, r in g_ref.items():
        if k not in g:
            continue
        a = np.asarray(g[k], np.float64)
        rms = np.sqrt((r ** 2).mean())
        if rms == 0:
            out[k] = (float(np.abs(a).max()), 0.0)
            continue
        elem = np.abs(a - r) / (np.abs(r) + rms)
        out[k] = (float(elem.max()), float(np.linalg.norm(a - r) / np.linalg.norm(r)))
    return out
