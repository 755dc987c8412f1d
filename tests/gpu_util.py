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


def tile_subset(O, scene, tl, cam_tiles):
    """Oracle inputs for whole sampled tiles: cam_tiles is a list of (view, global tile,
    pixel indices of the view in that tile).  Returns (sub_scene, prims, per-view lists)
    where sub_scene holds only the primitives on those tiles' lists (index remapped),
    so the FP64 oracle runs on a few thousand primitives of a large scene."""
    n = scene.n
    prim_sets = []
    for v, gt, pix in cam_tiles:
        a, b = int(tl.tile_off[gt]), int(tl.tile_off[gt + 1])
        prim_sets.append((tl.vals[a:b].astype(np.int64) % n))
    prims = np.unique(np.concatenate(prim_sets)) if prim_sets else np.zeros(0, np.int64)
    remap = np.full(n, -1, np.int64)
    remap[prims] = np.arange(len(prims))
    sub = scene.subset(prims)
    per_view = {}
    for (v, gt, pix), ps in zip(cam_tiles, prim_sets):
        d = per_view.setdefault(v, {"pix": [], "lists": [], "owner": []})
        d["owner"].append(np.full(len(pix), len(d["lists"]), np.int32))
        d["pix"].append(np.asarray(pix, np.int32))
        d["lists"].append(remap[ps].astype(np.int32))
    out = {}
    for v, d in per_view.items():
        off = np.concatenate([[0], np.cumsum([len(l) for l in d["lists"]])]).astype(np.int64)
        out[v] = (np.concatenate(d["pix"]), np.concatenate(d["owner"]), off, np.concatenate(d["lists"]))
    return sub, prims, out


def sample_tiles(cams, tl, ts, per_view, seed):
    """per_view random whole tiles (with at least one list entry) of every view."""
    rng = np.random.default_rng(seed)
    picks = []
    for v, cam in enumerate(cams):
        tx_n = (cam.width + ts - 1) // ts
        ty_n = (cam.height + ts - 1) // ts
        lens = np.diff(tl.tile_off[tl.view_tile_off[v]:tl.view_tile_off[v] + tx_n * ty_n + 1])
        cand = np.nonzero(lens > 0)[0]
        for lt in rng.choice(cand, size=min(per_view, len(cand)), replace=False):
            ty, tx = divmod(int(lt), tx_n)
            ys, xs = np.mgrid[ty * ts:min(ty * ts + ts, cam.height), tx * ts:min(tx * ts + ts, cam.width)]
            picks.append((v, int(tl.view_tile_off[v] + lt), (ys * cam.width + xs).ravel().astype(np.int32)))
    return picks
