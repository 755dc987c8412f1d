"""FP64 reverse-mode gradient oracle (plain PyTorch CPU autograd, float64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The forward below is the same definition as snp_oracle.c, written a second time
with torch float64 ops so that autograd yields d(sum dL/dC . C)/d(params):
  * Sec. 3.1 Eq. 5/6 density, ellipsoid bound {c + R_q diag(s) v : |v| <= 1},
    s = exp(log_s), q normalised, m = ||s||_inf;
  * Sec. 3.2 entry/exit and the closed-form integral (stable form of Eq. 8);
  * Eq. 9 alpha = 1 - exp(-max(0, alpha_hat));
  * Eq. 4 front-to-back compositing in the given candidate order, with the
    early-termination rule: after compositing entry i stop if T_{i+1} < t_min;
  * colour: constant, the ReLU/sigmoid colour MLP on [ray direction, feature], or
    four bands of real spherical harmonics along the camera-to-centre direction,
    c = max(0, 1/2 + sum_i Y_i(v) sh_i);
  * time-conditioned scenes (App. Applications): phase + xi_t W_t per hidden unit,
    and the degree-0 SH coefficient sh_0 + sum_j a_j xi^j + b_j cos(j xi) + c_j sin(j xi).
Candidate lists (which primitives a pixel walks, in which order) are inputs:
they come from the C oracle's FP32 key specification and are not differentiated.
Pinned by central finite differences of the independent C oracle forward.
"""
from __future__ import annotations

import math
from typing import Dict, Optional

import numpy as np
import torch

F64 = torch.float64


def scene_tensors(scene, requires_grad: bool = True) -> Dict[str, torch.Tensor]:
    out = {}
    for f in scene.fields():
        t = torch.tensor(np.asarray(getattr(scene, f), np.float64), dtype=F64)
        t.requires_grad_(requires_grad)
        out[f] = t
    return out


def pixel_rays(cam, pix: np.ndarray) -> torch.Tensor:
    """Unit rays through pixel centres (OpenCV pinhole), float64."""
    px = (pix % cam.width).astype(np.float64)
    py = (pix // cam.width).astype(np.float64)
    x = (px + 0.5 - float(cam.cx)) / float(cam.fx)
    y = (py + 0.5 - float(cam.cy)) / float(cam.fy)
    R = np.asarray(cam.R_wc, np.float64)
    r = x[:, None] * R[0][None] + y[:, None] * R[1][None] + R[2][None]
    r /= np.linalg.norm(r, axis=1, keepdims=True)
    return torch.tensor(r, dtype=F64)


def sh_basis(v: torch.Tensor) -> torch.Tensor:
    """Real spherical harmonics of degrees 0..3 (index l^2 + l + m, tesseral form)
    at unit vectors v [..., 3]; returns [..., 16]."""
    x, y, z = v[..., 0], v[..., 1], v[..., 2]
    pi = math.pi
    k1 = math.sqrt(3.0 / (4.0 * pi))
    a2, b2, c2 = 0.5 * math.sqrt(15.0 / pi), 0.25 * math.sqrt(5.0 / pi), 0.25 * math.sqrt(15.0 / pi)
    a3, b3 = 0.25 * math.sqrt(35.0 / (2.0 * pi)), 0.5 * math.sqrt(105.0 / pi)
    c3, d3, e3 = 0.25 * math.sqrt(21.0 / (2.0 * pi)), 0.25 * math.sqrt(7.0 / pi), 0.25 * math.sqrt(105.0 / pi)
    return torch.stack([
        torch.full_like(x, 0.5 * math.sqrt(1.0 / pi)),
        k1 * y, k1 * z, k1 * x,
        a2 * x * y, a2 * y * z, b2 * (3 * z * z - 1), a2 * x * z, c2 * (x * x - y * y),
        a3 * y * (3 * x * x - y * y), b3 * x * y * z, c3 * y * (5 * z * z - 1), d3 * z * (5 * z * z - 3),
        c3 * x * (5 * z * z - 1), e3 * z * (x * x - y * y), a3 * x * (x * x - 3 * y * y)], dim=-1)


def _time_series(xi: float) -> torch.Tensor:
    """Basis of the degree-0 colour series at time xi: xi^1..4, cos(j xi), sin(j xi) for j = 1..4."""
    j = np.arange(1, 5, dtype=np.float64)
    return torch.tensor(np.concatenate([xi ** j, np.cos(j * xi), np.sin(j * xi)]), dtype=F64)


def _sh_preact(params, pi: torch.Tensor, eye: torch.Tensor, xi: float = 0.0) -> torch.Tensor:
    """1/2 + sum_i Y_i(v) sh_i per channel, v the unit camera-to-centre direction
    (plus Y_0 times the degree-0 time series for a dynamic scene)."""
    v = params["centers"][pi] - eye[None]
    v = v / torch.linalg.norm(v, dim=-1, keepdim=True)
    Y = sh_basis(v)
    out = 0.5 + torch.einsum("qb,qbc->qc", Y, params["sh"][pi])
    if "sh_t" in params:
        out = out + Y[:, :1] * torch.einsum("j,qjc->qc", _time_series(xi), params["sh_t"][pi])
    return out


def _rotation(q: torch.Tensor) -> torch.Tensor:
    q = q / torch.linalg.norm(q, dim=-1, keepdim=True)
    w, x, y, z = q.unbind(-1)
    R = torch.stack([
        1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
        2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
        2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], dim=-1)
    return R.reshape(q.shape[:-1] + (3, 3))


def render(params: Dict[str, torch.Tensor], scene, cam, pix: np.ndarray, pix_list: np.ndarray,
           list_off: np.ndarray, list_prim: np.ndarray, t_min: float = 1e-4, bg=(0.0, 0.0, 0.0)):
    """Differentiable FP64 render of the given pixels.  Returns rgb [P, 3] (float64 tensor)."""
    P = len(pix)
    # pair layout: pixel-major, list order inside a pixel
    lens = (list_off[pix_list + 1] - list_off[pix_list]).astype(np.int64)
    Lmax = int(lens.max()) if P else 0
    if Lmax == 0:
        bgv = torch.tensor(bg, dtype=F64)
        return bgv.expand(P, 3).clone()
    starts = list_off[pix_list]
    pair_pix = np.repeat(np.arange(P), lens)
    pair_pos = np.arange(lens.sum()) - np.repeat(np.cumsum(lens) - lens, lens)
    pair_prim = list_prim[np.repeat(starts, lens) + pair_pos].astype(np.int64)

    d_all = pixel_rays(cam, pix)
    d = d_all[pair_pix]
    pi = torch.tensor(pair_prim)
    eye = torch.tensor(np.asarray(cam.eye, np.float64), dtype=F64)

    s = torch.exp(params["log_scales"][pi])
    R = _rotation(params["quats"][pi])
    c = params["centers"][pi]
    Minv = R.transpose(-1, -2) / s[:, :, None]  # row a = R[:, a] / s_a
    oc = eye[None] - c
    op = torch.einsum("qab,qb->qa", Minv, oc)
    dp = torch.einsum("qab,qb->qa", Minv, d)
    A = (dp * dp).sum(-1)
    B = (op * dp).sum(-1)
    tm = -B / A
    p = op + tm[:, None] * dp
    h2 = 1.0 - (p * p).sum(-1)
    hit = (h2 > 0).detach()
    h2s = torch.where(hit, h2, torch.ones_like(h2))
    half = torch.sqrt(h2s / A)
    m = s.max(dim=-1).values
    u = (oc + tm[:, None] * d) / m[:, None]
    w0 = float(scene.omega0)
    xi = float(getattr(cam, "time", 0.0))
    W1 = params["W1"][pi]
    phi = w0 * (torch.einsum("qkj,qj->qk", W1, u) + params["b1"][pi])
    if "wt" in params:
        phi = phi + xi * params["wt"][pi]
    th = w0 * torch.einsum("qkj,qj->qk", W1, d) * (half / m)[:, None]
    small = th.abs() < 1e-4
    ths = torch.where(small, torch.ones_like(th), th)
    sinc = torch.where(small, 1.0 - th * th / 6.0, torch.sin(ths) / ths)
    ah = 2.0 * half * (params["b2"][pi] + (params["w2"][pi] * torch.cos(phi) * sinc).sum(-1))
    ah = torch.where(hit, ah, torch.zeros_like(ah))
    ap = torch.relu(ah)

    # colour per pair (evaluated only where it is blended: alpha_hat > 0)
    if scene.color == "mlp":
        sel = torch.nonzero((ap > 0).detach()).squeeze(1)
        ps_ = pi[sel]
        z0 = torch.cat([d[sel], params["feat"][ps_]], dim=-1)
        z1 = torch.relu(torch.einsum("qjk,qk->qj", params["Wc1"][ps_], z0) + params["bc1"][ps_])
        z2 = torch.relu(torch.einsum("qjk,qk->qj", params["Wc2"][ps_], z1) + params["bc2"][ps_])
        c_sel = torch.sigmoid(torch.einsum("qjk,qk->qj", params["Wc3"][ps_], z2) + params["bc3"][ps_])
        col = torch.zeros(len(pi), 3, dtype=F64).index_put((sel,), c_sel)
    elif scene.color == "sh":
        col = torch.relu(_sh_preact(params, pi, eye, xi))
    else:
        col = params["rgb"][pi]

    # padded [P, Lmax] compositing
    flat = torch.tensor(pair_pix * Lmax + pair_pos)
    ap_pad = torch.zeros(P * Lmax, dtype=F64).index_put((flat,), ap).reshape(P, Lmax)
    col_pad = torch.zeros(P * Lmax, 3, dtype=F64).index_put((flat,), col).reshape(P, Lmax, 3)
    tau_incl = torch.cumsum(ap_pad, dim=1)
    tau_excl = tau_incl - ap_pad
    with torch.no_grad():
        if t_min > 0:
            walked = torch.exp(-tau_excl) >= t_min
        else:
            walked = torch.ones_like(ap_pad, dtype=torch.bool)
    apm = torch.where(walked, ap_pad, torch.zeros_like(ap_pad))
    tau_excl_m = torch.cumsum(apm, dim=1) - apm
    T = torch.exp(-tau_excl_m)
    alpha = -torch.expm1(-apm)
    rgb = (T[:, :, None] * alpha[:, :, None] * col_pad).sum(1)
    T_final = torch.exp(-apm.sum(1))
    bgv = torch.tensor(bg, dtype=F64)
    return rgb + T_final[:, None] * bgv[None]


def pair_diagnostics(scene, cam, pix, pix_list, list_off, list_prim):
    """Per candidate pair: (primitive, h^2 of the closest approach, alpha_hat or 0,
    smallest |pre-activation| of the colour MLP's ReLU layers or inf).

    Used by the finite-difference pins to avoid primitives that sit on a kink of
    the forward (a grazing ray, alpha_hat near 0, a ReLU at 0, or a tie in argmax s)."""
    lens = (list_off[pix_list + 1] - list_off[pix_list]).astype(np.int64)
    starts = list_off[pix_list]
    pair_pix = np.repeat(np.arange(len(pix)), lens)
    pair_pos = np.arange(lens.sum()) - np.repeat(np.cumsum(lens) - lens, lens)
    pair_prim = list_prim[np.repeat(starts, lens) + pair_pos].astype(np.int64)
    params = scene_tensors(scene, False)
    pi = torch.tensor(pair_prim)
    d = pixel_rays(cam, pix)[pair_pix]
    eye = torch.tensor(np.asarray(cam.eye, np.float64), dtype=F64)
    s = torch.exp(params["log_scales"][pi])
    Minv = _rotation(params["quats"][pi]).transpose(-1, -2) / s[:, :, None]
    oc = eye[None] - params["centers"][pi]
    op = torch.einsum("qab,qb->qa", Minv, oc)
    dp = torch.einsum("qab,qb->qa", Minv, d)
    A = (dp * dp).sum(-1)
    tm = -(op * dp).sum(-1) / A
    p = op + tm[:, None] * dp
    h2 = 1.0 - (p * p).sum(-1)
    half = torch.sqrt(torch.clamp(h2, min=0.0) / A)
    m = s.max(dim=-1).values
    u = (oc + tm[:, None] * d) / m[:, None]
    W1 = params["W1"][pi]
    w0 = float(scene.omega0)
    xi = float(getattr(cam, "time", 0.0))
    phi = w0 * (torch.einsum("qkj,qj->qk", W1, u) + params["b1"][pi])
    if "wt" in params:
        phi = phi + xi * params["wt"][pi]
    th = w0 * torch.einsum("qkj,qj->qk", W1, d) * (half / m)[:, None]
    small = th.abs() < 1e-4
    ths = torch.where(small, torch.ones_like(th), th)
    sinc = torch.where(small, 1.0 - th * th / 6.0, torch.sin(ths) / ths)
    ah = 2.0 * half * (params["b2"][pi] + (params["w2"][pi] * torch.cos(phi) * sinc).sum(-1))
    ah = torch.where(h2 > 0, ah, torch.zeros_like(ah))
    amin = torch.full_like(ah, float("inf"))
    if scene.color == "mlp":
        z0 = torch.cat([d, params["feat"][pi]], dim=-1)
        a1 = torch.einsum("qjk,qk->qj", params["Wc1"][pi], z0) + params["bc1"][pi]
        a2 = torch.einsum("qjk,qk->qj", params["Wc2"][pi], torch.relu(a1)) + params["bc2"][pi]
        amin = torch.minimum(a1.abs().min(-1).values, a2.abs().min(-1).values)
    elif scene.color == "sh":
        amin = _sh_preact(params, pi, eye, xi).abs().min(-1).values
    return pair_prim, h2.numpy(), ah.numpy(), amin.numpy()


def min_direction_dot(scene, cam, pix, pix_list, list_off, list_prim):
    """Per candidate pair (same order as pair_diagnostics): min_k |W1_k . d| over the
    density network's hidden units, d the unit pixel ray.  This is the directional
    frequency that Eq. 8 divides by (a_k = w0 W1_k . d / m); the precision-stress
    workload is built so that a share of the hit pairs has it below 1e-4."""
    lens = (list_off[pix_list + 1] - list_off[pix_list]).astype(np.int64)
    starts = list_off[pix_list]
    pair_pix = np.repeat(np.arange(len(pix)), lens)
    pair_pos = np.arange(lens.sum()) - np.repeat(np.cumsum(lens) - lens, lens)
    pair_prim = list_prim[np.repeat(starts, lens) + pair_pos].astype(np.int64)
    d = pixel_rays(cam, pix).numpy()[pair_pix]
    W1 = np.asarray(scene.W1, np.float64)[pair_prim]
    return np.abs(np.einsum("qkj,qj->qk", W1, d)).min(axis=1)


def grads(scene, cam, pix, pix_list, list_off, list_prim, dL_dC: np.ndarray, t_min: float = 1e-4,
          bg=(0.0, 0.0, 0.0)):
    """Vector-Jacobian product: d(sum dL_dC * C)/d(every parameter array), float64 numpy."""
    params = scene_tensors(scene, True)
    rgb = render(params, scene, cam, pix, pix_list, list_off, list_prim, t_min, bg)
    L = (rgb * torch.tensor(np.asarray(dL_dC, np.float64), dtype=F64)).sum()
    if L.requires_grad:
        L.backward()
    out = {}
    for k, t in params.items():
        out[k] = np.zeros(t.shape) if t.grad is None else t.grad.numpy().copy()
    return rgb.detach().numpy(), out
