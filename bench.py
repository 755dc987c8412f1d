#!/usr/bin/env python
"""Throughput benchmark of the splattable-neural-primitive tile rasterizer.

One step = one pass of the whole hot path over one batch of synthetic input:
projection/bounding -> key emission -> radix sort -> tile ranges -> forward
rasterizer -> backward rasterizer -> per-primitive gradient post-passes, on the
100k-primitive, four-view 1920 x 1080 workload (N_sigma = 16, colour MLP
N_c = 32, FP32).  Prints one JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--graph] [--autotune]

Other workloads (paper_2510_08491_gb300.synth.workload): diff300k_720p adds the
squared-error loss against a render of the perturbed scene to the step;
batch500k_16view (16 views of uneven size, BF16 weights, N_sigma = 32, N_c = 64)
is timed as replays of one captured CUDA graph with the tile size and chunk
picked by the autotuner.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpixel/s fwd and fwd+bwd at 1080p, 100k–500k primitives vs plain FP32 fwd; % roofline"
WORKLOAD = "fwd100k_1080p_4view"
# workloads timed as graph replays with an autotuned tile size and chunk
BATCHED = ("batch500k_16view",)
FP32_LANES_PER_SM = 128  # FP32 lanes per SM (4 sub-partitions x 32)
MUFU_LANES_PER_SM = 16   # special-function lanes per SM (4 sub-partitions x 4)


def chunks_used(ps, cfg):
    """(forward chunk, backward chunk) a render with cfg stages for this packed scene."""
    from paper_2510_08491_gb300 import _lib as L
    d = ps.desc
    f, b = L.default_chunks(int(d.n_sigma), int(d.color_mode), int(d.n_c), int(cfg.tile_size) or 16, bool(d.dynamic))
    fc = int(cfg.chunk) if cfg.chunk > 0 else f
    bc = min(b, int(cfg.bwd_chunk)) if cfg.bwd_chunk > 0 else b
    return fc, bc


# ----------------------------------------------------------------------------- work model

def work_per_unit(n_sigma: int, n_c: int, colour_store: bool):
    """Arithmetic the raster kernels execute per unit, counted from their code, as
    (FP32 lane-ops, tensor-core multiply-adds, MUFU ops).  Units are the run's own
    counters: candidates (pixel, list entry) tested, hits (ray enters the
    ellipsoid), composited pairs (alpha_hat > 0 before termination).

    FP32 lane-ops: an FMA, FMUL or FADD takes one slot of the FP32 pipe (128 per SM
    per clock; FLOP = 2 x lane-op, the convention of that peak).  Shuffles,
    selects, conversions, shared-memory atomics and address arithmetic are not
    counted.  Tensor multiply-adds: the colour network's hidden layer, one per
    weight and ray (N_c^2), however many split-precision products it takes.
      forward  candidate  28: ray offset, G dr, e + f, |e + f|^2, e x f, |e x f|^2, h^2 A
               hit        29 + 15 N_sigma: reciprocal, h^2, f . dp, s, t, chord (12); offset
                          direction, u_mid, scales (17); per hidden unit W1 . g, phase,
                          theta, sinc series, accumulate (15); MUFU 2 + 3 N_sigma
               composited 10 (weight, optical depth, blend; MUFU 2); colour network
                          6 N_c + 3 (layers 1 and 3, sigmoid), N_c^2 tensor, MUFU 6
      backward composited 177 + 40 N_sigma: compositing derivative (15), geometry and its
                          reverse (38 + 17 + 92), per hidden unit the integral and its
                          derivatives (40); MUFU 3 + 5 N_sigma; colour network 14 N_c
                          (layer-1 replay, layer-3 and layer-1 reverse), 3 N_c^2 tensor
                          (hidden-layer replay, its input gradient, its weight gradient)
               no store   + the forward's hit and candidate work per composited pair (the
                          alpha_hat replay) and, with a colour network, its forward (the
                          store holds colour and alpha_hat, or alpha_hat alone)
    The backward tests no candidates: its pair lists come from the forward's
    composited masks."""
    ns, nc = n_sigma, n_c
    mlp = nc > 0
    fwd = {"cand": (28, 0, 0),
           "hit": (29 + 15 * ns, 0, 2 + 3 * ns),
           "comp": (10 + (6 * nc + 3 if mlp else 0), nc * nc, 2 + (6 if mlp else 0))}
    comp = [177 + 40 * ns + 14 * nc, 3 * nc * nc, 3 + 5 * ns]
    if not colour_store:
        comp[0] += 28 + 29 + 15 * ns
        comp[2] += 2 + 3 * ns
        if mlp:
            comp[0] += 6 * nc + 3
            comp[1] += nc * nc
            comp[2] += 6
    bwd = {"cand": (0, 0, 0), "hit": (0, 0, 0), "comp": tuple(comp)}
    return fwd, bwd


def kernel_work(counts, per_unit):
    """(FP32 FLOP, tensor FLOP, MUFU ops) of one launch."""
    tot = [0.0, 0.0, 0.0]
    for u, c in counts.items():
        for i in range(3):
            tot[i] += float(c) * per_unit[u][i]
    return 2.0 * tot[0], 2.0 * tot[1], tot[2]


def pipe_roofline(work, t_ms, traffic, peaks):
    """Achieved rate and fraction of peak per pipe for one kernel launch of t_ms."""
    fp32, tensor, mufu = work
    t = t_ms * 1e-3
    out = {"fp32": {"achieved": fp32 / t / 1e12, "peak": peaks["fp32_tflops"], "unit": "TFLOP/s"},
           "tensor": {"achieved": tensor / t / 1e12, "peak": peaks["tensor_tflops"], "unit": "TFLOP/s"},
           "mufu": {"achieved": mufu / t / 1e12, "peak": peaks["mufu_tops"], "unit": "Tops/s"}}
    if traffic:
        out["hbm"] = {"achieved": traffic / t / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s"}
    for v in out.values():
        v["frac"] = round(v["achieved"] / v["peak"], 4)
        v["achieved"] = round(v["achieved"], 3)
    return out


def raster_sources_digest() -> str:
    """Digest of the raster kernels' sources (the traffic counters stay valid only for them)."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2510_08491_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(csrc)):
        if f.startswith(("snp_raster", "snp_common", "snp_df", "snp_mma")):
            h.update(f.encode())
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def raster_traffic(workload: str) -> dict:
    """DRAM bytes per launch of each raster kernel from the committed ncu summary
    (profiles/traffic.json), when it was taken on this workload from the current
    kernel sources; otherwise nothing (the counters no longer describe the kernel)."""
    try:
        tr = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    except Exception:
        return {}
    if tr.get("workload") != workload or tr.get("sources") != raster_sources_digest():
        return {}
    return {k: tr[k]["bytes_per_launch"] for k in ("k_raster_fwd", "k_raster_bwd") if k in tr}


def device_peaks(dev: int):
    """Peaks of the roofline: FP32 and MUFU from the device's SM count and the
    measured maximum SM clock, bf16 tensor and HBM copy bandwidth as measured
    (MEASURED_PEAKS.json; the sustained bf16 figure, since the raster kernels run
    inside a long step).  Falls back to the recipe's figures without that file."""
    import torch
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    measured = "sm_max_mhz" in peaks
    return {"sms": sms, "sm_mhz": mhz,
            "fp32_tflops": round(sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12, 2),
            "mufu_tops": round(sms * MUFU_LANES_PER_SM * mhz * 1e6 / 1e12, 3),
            "tensor_tflops": float(peaks.get("bf16_tflops_sustained", 1700.0)),
            "hbm_gbs": float(peaks.get("hbm_gbs", 6800.0)),
            "note": (f"FP32: {sms} SMs x {FP32_LANES_PER_SM} lanes x 2 FLOP x {mhz:.0f} MHz; MUFU: {sms} SMs x "
                     f"{MUFU_LANES_PER_SM} lanes x {mhz:.0f} MHz; " +
                     ("sm_max_mhz, sustained bf16 TFLOP/s and HBM GB/s of measured peaks" if measured
                      else "2070 MHz, 1700 TFLOP/s bf16 sustained, 6800 GB/s (fallback: no measured peaks file)"))}


# ----------------------------------------------------------------------------- multi-rank
def max_over_ranks(x: float) -> float:
    """The maximum of x over all ranks of the default process group (x itself when
    torch.distributed is not initialised).  NCCL reduces a CUDA tensor, gloo a CPU one."""
    import torch
    import torch.distributed as D
    if not (D.is_available() and D.is_initialized()) or D.get_world_size() == 1:
        return float(x)
    dev = "cuda" if D.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    D.all_reduce(t, op=D.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: int, ms_max: float, world: int) -> float:
    """Whole-job throughput of N independent replicas (weak scaling): the units all
    ranks processed, over the slowest rank's time, in millions per second."""
    return world * units_per_rank / (ms_max * 1e-3) / 1e6


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int = 0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                rows.append((float(p[1]), float(p[2]), p[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        sm = sorted(r[0] for r in rows)
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


# ----------------------------------------------------------------------------- oracle (CPU) leg
def oracle_sample(wl, tiles_per_view: int, seed: int = 0, with_grad: bool = True, keep: bool = False):
    """Time the FP64 oracle on a bounded sample of the workload: the key stage of every
    view (pro-rated to the sample), then forward (+ gradient) of `tiles_per_view`
    seeded 16 x 16 tiles per view.  Returns (pixels, seconds, cores[, kept]).

    keep: also return the sample (per view: pixels, oracle colours, termination
    near-tie flags and the dL/dC used) and the oracle's gradient summed over the
    views, for the accuracy report.  dL/dC is then zero on pixels at a termination
    near-tie or with a composited pair at a colour-network ReLU kink, where FP32
    and FP64 may take different branches; that check runs outside the timing."""
    import numpy as np

    from oracle import grad as G
    from oracle import oracle as O
    O.build()
    sc, cams = wl.scene, wl.cameras
    t0 = time.perf_counter()
    cs = O.CScene(sc)
    tl = O.tile_keys(sc, cams, 16, cs)
    t_keys = time.perf_counter() - t0
    rng = np.random.default_rng(seed)
    npx = 0
    t_pix = 0.0
    total_px = sum(c.n_pixels for c in cams)
    kept = {"views": [], "grads": None, "prims": []}
    for v, cam in enumerate(cams):
        tx_n, ty_n = O.tiles_xy(cam, 16)
        tiles = rng.choice(tx_n * ty_n, size=tiles_per_view, replace=False)
        pix = []
        for t in tiles:
            ty, tx = divmod(int(t), tx_n)
            ys, xs = np.mgrid[ty * 16:min(ty * 16 + 16, cam.height), tx * 16:min(tx * 16 + 16, cam.width)]
            pix.append((ys * cam.width + xs).ravel())
        pix = np.concatenate(pix).astype(np.int32)
        t1 = time.perf_counter()
        out = O.render_view_tiled(sc, cams, v, tl, 16, pix, cs=cs)
        t_pix += time.perf_counter() - t1
        if with_grad:
            gt = tl.view_tile_off[v] + O.pixel_tile(cam, 16, pix)
            lp = (tl.vals.astype(np.int64) % sc.n).astype(np.int32)
            dL = rng.normal(size=(len(pix), 3))
            if keep:
                dL[out.flags != 0] = 0.0
                if sc.color == "mlp":
                    _, _, ah, amin = G.pair_diagnostics(sc, cam, pix, gt, tl.tile_off, lp)
                    lens = tl.tile_off[gt + 1] - tl.tile_off[gt]
                    owner = np.repeat(np.arange(len(pix)), lens)
                    dL[np.unique(owner[(ah > 0) & (amin < 1e-4)])] = 0.0
                ut = np.unique(gt)
                kept["prims"].append(np.concatenate([lp[tl.tile_off[t]:tl.tile_off[t + 1]] for t in ut]))
            t1 = time.perf_counter()
            _, g = G.grads(sc, cam, pix, gt, tl.tile_off, lp, dL)
            t_pix += time.perf_counter() - t1
            if keep:
                kept["grads"] = g if kept["grads"] is None else {k: kept["grads"][k] + g[k] for k in g}
                kept["views"].append((pix, out.rgb, out.flags, dL))
        npx += len(pix)
    secs = t_keys * (npx / total_px) + t_pix
    if keep:
        kept["prims"] = np.unique(np.concatenate(kept["prims"])) if kept["prims"] else np.zeros(0, np.int64)
        return npx, secs, os.cpu_count() or 1, kept
    return npx, secs, os.cpu_count() or 1


def accuracy_vs_oracle(r, ps, sc, cams, cfg, kept):
    """Image and gradient error of the CUDA path against the FP64 oracle on the
    oracle leg's sampled tiles: max and mean |C - C*| per channel (pixels at a
    termination near-tie reported apart), and per parameter group the elementwise
    max |g - g*| / (|g*| + rms g*) and ||g - g*|| / ||g*|| over the primitives the
    sampled tiles list (dL/dC set on the sampled pixels only)."""
    import numpy as np
    import torch

    from paper_2510_08491_gb300.render import unpack_geom_grad, unpack_net_grad
    P = sum(c.n_pixels for c in cams)
    img = r.forward(ps, cams, cfg).cpu().numpy().astype(np.float64)
    off = np.concatenate([[0], np.cumsum([c.n_pixels for c in cams])])
    errs, flags = [], []
    dL = np.zeros((P, 3), np.float32)
    for v, (pix, rgb, fl, d) in enumerate(kept["views"]):
        errs.append(np.abs(img[off[v] + pix] - rgb).max(axis=1))
        flags.append(fl)
        dL[off[v] + pix] = d
    err, fl = np.concatenate(errs), np.concatenate(flags)
    plain = fl == 0
    g_geom = torch.zeros_like(ps.geom)
    g_net = torch.zeros(ps.net.shape, dtype=torch.float32, device=ps.net.device)
    r.backward(ps, torch.tensor(dL, device=ps.geom.device), g_geom, g_net)
    torch.cuda.synchronize()
    g = unpack_geom_grad(g_geom)
    g.update(unpack_net_grad(ps, g_net, sc))
    act = kept["prims"]
    groups = {}
    for k, ref in kept["grads"].items():
        if k not in g:
            continue
        a, b = np.asarray(g[k], np.float64)[act], np.asarray(ref, np.float64)[act]
        rms = float(np.sqrt((b ** 2).mean()))
        nb = float(np.linalg.norm(b))
        if rms == 0.0 or nb == 0.0:
            continue
        groups[k] = (float((np.abs(a - b) / (np.abs(b) + rms)).max()), float(np.linalg.norm(a - b) / nb))
    worst_e = max(groups, key=lambda k: groups[k][0])
    worst_n = max(groups, key=lambda k: groups[k][1])
    return {"image_max_abs": float(err[plain].max()), "image_mean_abs": float(err.mean()),
            "image_flagged_max_abs": float(err[~plain].max()) if (~plain).any() else 0.0,
            "pixels": int(len(err)), "flagged_pixels": int((~plain).sum()),
            "grad_elem_max": round(groups[worst_e][0], 7), "grad_elem_group": worst_e,
            "grad_norm_max": round(groups[worst_n][1], 7), "grad_norm_group": worst_n,
            "primitives": int(len(act)),
            "bars": "image 1e-4 abs (flagged 2e-4); gradients 1e-3 elementwise and in norm",
            "oracle": "FP64 CPU oracle on the cpu_baseline leg's sampled tiles"}


# ----------------------------------------------------------------------------- GPU leg
# Training hyperparameters of the paper (App. hyperparameters): Adam learning
# rates per group -- geometry (centres, log-scales, quaternions, constant rgb; the
# paper gives no rate for a constant colour, so it takes the SH rate) and per
# network field (snp_net_layout order: the density and colour MLPs at the MLP
# rate, SH coefficients and their time series at the SH rate, W_t at the MLP
# rate) -- and the synthetic-scene population-control thresholds.
PAPER_LR_GEOM = [1.6e-4, 5e-3, 1e-3, 2.5e-3]
PAPER_LR_NET = [1e-3] * 11 + [2.5e-3, 1e-3, 2.5e-3]
PAPER_POPCTL_SYNTHETIC = (1e-5, 1e-6, 1e-2, 0.5)  # densify, prune, grow scale, prune scale


class TrainState:
    """The rest of a training step after the backward pass: the anisotropy
    regulariser, the population-control statistic and one Adam step (learning
    rates of the paper's App. hyperparameters), plus isolated timings of each."""

    def __init__(self, r, ps, sc):
        import torch
        from paper_2510_08491_gb300 import _lib as L
        self.r, self.ps, self.n = r, ps, ps.n
        self.m_geom, self.v_geom = torch.zeros_like(ps.geom), torch.zeros_like(ps.geom)
        self.m_net = torch.zeros(ps.net.shape, dtype=torch.float32, device="cuda")
        self.v_net = torch.zeros_like(self.m_net)
        self.master = ps.net.float().clone() if ps.net.dtype != torch.float32 else None
        self.ssum = torch.zeros(self.n, dtype=torch.float32, device="cuda")
        self.scnt = torch.zeros(self.n, dtype=torch.int32, device="cuda")
        c = L.AdamConfig()
        c.lr_geom[:] = PAPER_LR_GEOM
        c.lr_net[:] = PAPER_LR_NET
        c.beta1, c.beta2, c.eps, c.step = 0.9, 0.999, 1e-15, 0
        self.cfg = c
        ns, nc = sc.n_sigma, sc.n_c if sc.color == "mlp" else 0
        sizes = [3 * ns, ns, ns, 1, 8, nc * 11, nc, nc * nc, nc, 3 * nc, 3, 48, ns, 36]
        self.net_cols = sum(4 * ((sizes[k] + 3) // 4) for k, o in enumerate(ps.offsets) if o >= 0)
        self.reg_weight = 1e-3

    def step(self, g_geom, g_net):
        self.r.geom_reg(self.ps, self.reg_weight, g_geom)
        self.r.popctl_accumulate(self.ps, g_net, self.ssum, self.scnt)
        self.cfg.step += 1
        self.r.adam_step(self.ps, g_geom, g_net, self.m_geom, self.v_geom, self.m_net, self.v_net, self.cfg,
                         net_master=self.master)

    def _time(self, fn, k):
        import torch
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(k):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / k

    def measure(self, g_geom, g_net, hbm_gbs, hbm_note="HBM copy bandwidth of measured peaks"):
        import torch
        from paper_2510_08491_gb300 import _lib as L

        def adam():
            self.cfg.step += 1
            self.r.adam_step(self.ps, g_geom, g_net, self.m_geom, self.v_geom, self.m_net, self.v_net, self.cfg,
                             net_master=self.master)
        t_adam = self._time(adam, 20)
        # algorithmic bytes: per updated element p, g, m, v read and p, m, v written (28 B;
        # BF16 weights: FP32 master plus the 2-byte rounded copy, 30 B)
        b_el = 30 if self.master is not None else 28
        bytes_adam = self.n * (13 * 28 + self.net_cols * b_el)
        t_reg = self._time(lambda: self.r.geom_reg(self.ps, self.reg_weight, g_geom), 20)
        t_stat = self._time(lambda: self.r.popctl_accumulate(self.ps, g_net, self.ssum, self.scnt), 20)
        pc = L.PopctlConfig(*PAPER_POPCTL_SYNTHETIC, 4.0, 0)
        noise = torch.randn((self.n, 2, 3), device="cuda", generator=torch.Generator("cuda").manual_seed(3))

        def densify():
            a, o, n_out = self.r.popctl_plan(self.ps, self.ssum, self.scnt, pc)
            self.r.popctl_apply(self.ps, a, o, n_out, noise)
        t_pop = self._time(densify, 5)
        gbs = bytes_adam / (t_adam * 1e-3) / 1e9
        return {"adam_ms": round(t_adam, 4), "adam_bytes": int(bytes_adam), "adam_gbs": round(gbs, 1),
                "adam_hbm_frac": round(gbs / hbm_gbs, 4), "regulariser_ms": round(t_reg, 4),
                "statistic_ms": round(t_stat, 4), "plan_apply_ms": round(t_pop, 4),
                "peak_note": hbm_note}


def run_ours(args, rank, world):
    import numpy as np
    import torch

    from paper_2510_08491_gb300 import _lib as L
    from paper_2510_08491_gb300 import build as B
    from paper_2510_08491_gb300 import synth
    from paper_2510_08491_gb300.render import Renderer, pack_scene

    B.build()
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    wl = synth.workload(args.workload)
    sc, cams = wl.scene, wl.cameras
    r = Renderer(dev)
    ps = pack_scene(sc)
    P = sum(c.n_pixels for c in cams)
    batched = args.workload in BATCHED
    use_graph = (args.graph or batched) and not args.train
    cfg = L.make_config(tile_size=args.tile, t_min=wl.t_min, timing=not use_graph, replay_color=args.replay_color)
    if args.autotune or batched:
        cfg = r.autotune(ps, cams, cfg, backward=True)
        cfg.flags = (L.FLAG_STAGE_TIMING if not use_graph else 0) | (L.FLAG_REPLAY_COLOR if args.replay_color else 0)
    img = torch.empty((P, 3), device="cuda", dtype=torch.float32)
    target = None
    if wl.target_scene is not None:
        # the differentiation workload: squared error against a render of the perturbed scene
        target = r.forward(pack_scene(wl.target_scene), cams, L.make_config(t_min=wl.t_min)).clone()
        dL = torch.empty((P, 3), device="cuda", dtype=torch.float32)
        loss = torch.zeros(1, device="cuda", dtype=torch.float32)
    else:
        dL = torch.randn((P, 3), device="cuda", generator=torch.Generator("cuda").manual_seed(1)) * 1e-3
        loss = None
    g_geom = torch.zeros_like(ps.geom)
    g_net = torch.zeros(ps.net.shape, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    train_state = TrainState(r, ps, sc) if args.train else None

    def step():
        g_geom.zero_()
        g_net.zero_()
        r.forward(ps, cams, cfg, out=img)
        if target is not None:
            r.mse_loss(img, target, dL, loss)
        r.backward(ps, dL, g_geom, g_net)
        if train_state is not None:
            train_state.step(g_geom, g_net)

    def fwd_only():
        r.forward(ps, cams, cfg, out=img)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    stats = r.stats()
    counts = {"cand": stats.n_candidates, "hit": stats.n_hits, "comp": stats.n_composited}
    graph = None
    if use_graph:
        from paper_2510_08491_gb300.render import GraphStep
        graph = GraphStep(r, ps, cams, cfg, max_keys=int(stats.n_keys * 1.05) + 4096,
                          dL=None if target is not None else dL, target=target)
        img, g_geom, g_net = graph.image, graph.g_geom, graph.g_net
        if target is not None:
            dL, loss = graph.dL, graph.loss
        for _ in range(args.warmup):
            graph.replay()
        torch.cuda.synchronize()
        timed_step = graph.replay
    else:
        timed_step = step
    dist = world > 1
    if dist:
        import torch.distributed as D
    r.ctx.stage_times(reset=True)
    l0 = L.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk:
        if dist:
            D.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            timed_step()
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            D.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    if graph is not None:
        # graph replays launch no kernel through the library's counter; count one eager step
        l0 = L.kernel_launches()
        step()
        torch.cuda.synchronize()
        launches = L.kernel_launches() - l0
        # per-kernel device times from eager steps with stage timing (same kernels, same config)
        cfg.flags = L.FLAG_STAGE_TIMING | (L.FLAG_REPLAY_COLOR if args.replay_color else 0)
        r.ctx.stage_times(reset=True)
        for _ in range(max(min(args.steps, 5), 2)):
            step()
        torch.cuda.synchronize()
        st = r.ctx.stage_times(reset=True)
    else:
        launches = (L.kernel_launches() - l0) // max(args.steps, 1)
        st = r.ctx.stage_times(reset=True)
    ms = max_over_ranks(ms)
    value = replica_throughput(P, ms, world)

    # forward only (same workload), for the "vs plain FP32 forward" comparison
    for _ in range(2):
        fwd_only()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    nf = max(args.steps, 3)
    for _ in range(nf):
        fwd_only()
    f1.record(stream)
    torch.cuda.synchronize()
    ms_fwd = f0.elapsed_time(f1) / nf
    r.ctx.stage_times(reset=True)

    # end to end through the public API with host buffers, measured two ways:
    #   e2e             the scene's parameters and gradients stay resident on the device
    #                   (uploaded once, as in a training loop whose optimizer runs on the
    #                   GPU); every step copies its image-space input (dL/dimage, or the
    #                   target image of the loss) in from pinned host memory and its
    #                   rendered image (and loss) out;
    #   e2e_with_params every step also copies all parameters in and all gradients out.
    # Both inside the timed region.  The copies run on two copy streams (one per
    # direction), and inputs and outputs are double-buffered (two scene / output buffer
    # sets; with a captured graph, two graphs on one reservation), so that a step's
    # inputs arrive during the previous step's compute and its outputs leave during the
    # next step's, as a training pipeline's prefetch would.  With the training services
    # on (they update the scene in place) the step runs on one buffer set and only the
    # two copy directions overlap.
    h_geom = ps.geom.cpu().pin_memory()
    h_net = ps.net.cpu().pin_memory()
    d_in0 = target if target is not None else dL
    h_in = d_in0.cpu().pin_memory()
    s_h2d, s_d2h = torch.cuda.Stream(), torch.cuda.Stream()
    use_pipe = graph is None and train_state is None
    graphs = None
    if graph is not None and train_state is None:
        # a second graph over its own scene and output buffers, on the same reservation
        from paper_2510_08491_gb300.render import GraphStep, PackedScene
        ps2 = PackedScene(ps.desc, ps.geom.clone(), ps.net.clone(), ps.offsets, ps.stride)
        g2 = GraphStep(r, ps2, cams, cfg, max_keys=0, dL=None if target is not None else dL.clone(),
                       target=target.clone() if target is not None else None, reserve=False)
        graphs = [graph, g2]
        bufs = [{"ps": G.ps, "in": G.target if target is not None else G.dL, "img": G.image, "gg": G.g_geom,
                 "gn": G.g_net, "dL": G.dL, "loss": G.loss} for G in graphs]
    elif use_pipe:
        from paper_2510_08491_gb300.render import PackedScene
        bufs = []
        for b in range(2):
            psb = PackedScene(ps.desc, torch.empty_like(ps.geom), torch.empty_like(ps.net), ps.offsets, ps.stride)
            bufs.append({"ps": psb, "in": torch.empty_like(d_in0), "img": torch.empty((P, 3), device="cuda"),
                         "gg": torch.empty_like(g_geom), "gn": torch.empty_like(g_net),
                         "dL": torch.empty((P, 3), device="cuda") if target is not None else None,
                         "loss": torch.zeros(1, device="cuda") if target is not None else None})
    else:
        bufs = [{"ps": ps, "in": d_in0, "img": img, "gg": g_geom, "gn": g_net,
                 "dL": dL if target is not None else None, "loss": loss}]
    hosts = [{"img": torch.empty((P, 3), dtype=torch.float32).pin_memory(),
              "gg": torch.empty_like(g_geom, device="cpu").pin_memory(),
              "gn": torch.empty_like(g_net, device="cpu").pin_memory(),
              "loss": torch.empty(1, dtype=torch.float32).pin_memory()} for _ in bufs]
    ev = {k: [torch.cuda.Event() for _ in bufs] for k in ("h2d", "done", "d2h")}

    def h2d(b, after=None, params=True):
        with torch.cuda.stream(s_h2d):
            if after is not None:
                s_h2d.wait_event(after)
            B = bufs[b]
            if params:
                B["ps"].geom.copy_(h_geom, non_blocking=True)
                B["ps"].net.copy_(h_net, non_blocking=True)
            B["in"].copy_(h_in, non_blocking=True)
            ev["h2d"][b].record(s_h2d)

    def compute(b):
        B = bufs[b]
        if graphs is not None:
            graphs[b].replay()
            return
        if not use_pipe:
            timed_step()
            return
        B["gg"].zero_()
        B["gn"].zero_()
        r.forward(B["ps"], cams, cfg, out=B["img"])
        if target is not None:
            r.mse_loss(B["img"], B["in"], B["dL"], B["loss"])
            r.backward(B["ps"], B["dL"], B["gg"], B["gn"])
        else:
            r.backward(B["ps"], B["in"], B["gg"], B["gn"])

    def d2h(b, grads=True):
        B, H = bufs[b], hosts[b]
        with torch.cuda.stream(s_d2h):
            s_d2h.wait_event(ev["done"][b])
            H["img"].copy_(B["img"], non_blocking=True)
            if grads:
                H["gg"].copy_(B["gg"], non_blocking=True)
                H["gn"].copy_(B["gn"], non_blocking=True)
            if B["loss"] is not None:
                H["loss"].copy_(B["loss"], non_blocking=True)
            ev["d2h"][b].record(s_d2h)

    def e2e_run(n, full):
        nb = len(bufs)
        start = torch.cuda.Event()
        start.record(stream)
        h2d(0, after=start, params=full)
        for i in range(n):
            b = i % nb
            stream.wait_event(ev["h2d"][b])
            if i >= nb or (nb == 1 and i >= 1):
                stream.wait_event(ev["d2h"][b])  # its outputs have left
            compute(b)
            ev["done"][b].record(stream)
            d2h(b, grads=full)
            if i + 1 < n:
                # the next step's inputs: its buffer's previous compute must be done
                h2d((i + 1) % nb, after=ev["done"][(i + 1) % nb] if i + 1 >= nb else None, params=full)
        for b in range(nb):
            stream.wait_event(ev["d2h"][b])

    ne = max(min(args.steps, 10), 3)

    def e2e_time(full):
        e2e_run(2, full)
        torch.cuda.synchronize()
        x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        x0.record(stream)
        e2e_run(ne, full)
        x1.record(stream)
        torch.cuda.synchronize()
        return x0.elapsed_time(x1) / ne

    # the parameters are uploaded once before the resident measurement (outside its timing)
    for b in range(len(bufs)):
        h2d(b, params=True)
    torch.cuda.synchronize()
    ms_e2e = e2e_time(False)
    ms_e2e_full = e2e_time(True)
    h_loss = hosts[(ne - 1) % len(bufs)]["loss"]
    param_bytes = h_geom.numel() * h_geom.element_size() + h_net.numel() * h_net.element_size()
    grad_bytes = g_geom.numel() * 4 + g_net.numel() * 4
    h2d_bytes = h_in.numel() * 4
    d2h_bytes = P * 3 * 4 + (4 if loss is not None else 0)

    # roofline of the raster kernels (per pipe; the dominant kernel's binding pipe is the headline)
    peaks = device_peaks(dev)
    nc_eff = sc.n_c if sc.color == "mlp" else 0
    colour_store = not args.replay_color
    fwd_u, bwd_u = work_per_unit(sc.n_sigma, nc_eff, colour_store)
    t_fwd = st["raster_fwd"][0] / max(st["raster_fwd"][1], 1)
    t_bwd = st["raster_bwd"][0] / max(st["raster_bwd"][1], 1)
    traffic = raster_traffic(args.workload)
    kernels = {"k_raster_fwd": pipe_roofline(kernel_work(counts, fwd_u), t_fwd, traffic.get("k_raster_fwd"), peaks),
               "k_raster_bwd": pipe_roofline(kernel_work(counts, bwd_u), t_bwd, traffic.get("k_raster_bwd"), peaks)}
    kern = "k_raster_bwd" if t_bwd >= t_fwd else "k_raster_fwd"
    pipes = kernels[kern]
    bind = max(pipes, key=lambda k: pipes[k]["frac"])
    clocks = clk.summary()

    res = {
        "metric": METRIC, "value": round(value, 3), "unit": "Mpixel/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "primitives": sc.n, "views": len(cams),
                   "resolution": f"{cams[0].width}x{cams[0].height}", "n_sigma": sc.n_sigma,
                   "n_c": sc.n_c if sc.color == "mlp" else 0, "weights": sc.weight_dtype,
                   "tile": int(cfg.tile_size), "chunk": chunks_used(ps, cfg)[0],
                   "bwd_chunk": chunks_used(ps, cfg)[1],
                   "ctas_per_sm": {"fwd": int(stats.fwd_ctas_per_sm), "bwd": int(stats.bwd_ctas_per_sm)},
                   "step": "forward+loss+backward" if target is not None else "forward+backward",
                   "graph": graph is not None, "autotuned": bool(args.autotune or batched),
                   "colour_store": not args.replay_color,
                   "parallelism": "replicas" if world > 1 else "single-gpu",
                   "l2": "inputs larger than L2 (network weights %.2f GB)" % (h_net.numel() * h_net.element_size()
                                                                              / 1e9)},
        "fwd_mpix_s": round(world * P / (ms_fwd * 1e-3) / 1e6, 3),
        "fwd_ms": round(ms_fwd, 4),
        "roofline": {"bound": {"fp32": "alu", "mufu": "alu", "tensor": "tensor", "hbm": "hbm"}[bind],
                     "pipe": bind, "kernel": kern, "achieved": pipes[bind]["achieved"], "peak": pipes[bind]["peak"],
                     "unit": pipes[bind]["unit"], "frac": pipes[bind]["frac"],
                     "traffic": traffic.get(kern), "kernels": kernels, "peak_note": peaks["note"],
                     "work_note": "executed arithmetic per candidate / hit / composited pair counted from the "
                                  "kernels (bench.work_per_unit) x the run's counters; fraction = max over pipes"},
        "e2e": {"value": round(world * P / (ms_e2e * 1e-3) / 1e6, 3), "unit": "Mpixel/s",
                "h2d_bytes_per_step": int(h2d_bytes), "d2h_bytes_per_step": int(d2h_bytes),
                "ms_per_step": round(ms_e2e, 4),
                "copies": "per step: the image-space input in, the rendered image (and loss) out; scene "
                          "parameters and gradients resident on the device",
                "overlap": "pipelined (double-buffered, copy streams)" if (use_pipe or graphs is not None)
                           else "copy directions overlapped"},
        "e2e_with_params": {"value": round(world * P / (ms_e2e_full * 1e-3) / 1e6, 3), "unit": "Mpixel/s",
                            "h2d_bytes_per_step": int(h2d_bytes + param_bytes),
                            "d2h_bytes_per_step": int(d2h_bytes + grad_bytes), "ms_per_step": round(ms_e2e_full, 4),
                            "copies": "per step also every parameter in and every gradient out"},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "stage_ms": {k: round(v[0] / max(v[1], 1), 4) for k, v in st.items()},
        "work": {"keys": stats.n_keys, "candidates": counts["cand"], "hits": counts["hit"],
                 "composited": counts["comp"], "pixels": P},
    }
    if loss is not None:
        res["loss"] = float(h_loss.item())
    if train_state is not None:
        res["config"]["step"] += "+regulariser+statistic+adam"
        res["train"] = train_state.measure(g_geom, g_net, peaks["hbm_gbs"],
                                           "HBM copy bandwidth: " + peaks["note"].split("; ")[-1])
    if rank == 0 and not args.no_cpu_baseline and (args.workload == WORKLOAD or args.cpu_baseline):
        npx, secs, cores, kept = oracle_sample(wl, args.cpu_tiles, keep=True)
        res["cpu_baseline"] = {"value": round(npx / secs / 1e6, 6), "unit": "Mpixel/s", "cores": cores,
                               "kind": "oracle",
                               "sample": f"forward+gradient of {args.cpu_tiles} seeded 16x16 tiles per view "
                                         f"({npx} px) plus the key stage pro-rated to the sample; {secs:.1f} s"}
        res["accuracy"] = accuracy_vs_oracle(r, ps, sc, cams, cfg, kept)
    if args.workload == WORKLOAD and not args.no_forms and not args.train:
        # the metric's comparison: the BF16-weight, batched, differentiable form beside
        # the plain FP32 forward (and FP32 forward + backward) of this run
        res["forms"] = {"fp32_forward": {"workload": args.workload, "mpix_s": res["fwd_mpix_s"],
                                         "ms": res["fwd_ms"]},
                        "fp32_fwd_bwd": {"workload": args.workload, "mpix_s": res["value"], "ms": res["ms_per_step"]},
                        "bf16_batched_graph": batched_form(dev, max(min(args.steps, 5), 3), args.warmup)}
    return res


def batched_form(dev: int, steps: int, warmup: int):
    """The BF16-weight, batched, differentiable form on its own workload
    (batch500k_16view: 500k primitives, N_sigma = 32, N_c = 64, BF16 weights, 16
    views of uneven size): forward + backward of all views, one persistent launch
    each, captured in one CUDA graph with the autotuned tile size and chunk, timed
    as graph replays on the device (inputs resident); and its forward alone."""
    import torch

    from paper_2510_08491_gb300 import _lib as L
    from paper_2510_08491_gb300 import synth
    from paper_2510_08491_gb300.render import GraphStep, Renderer, pack_scene
    wl = synth.workload("batch500k_16view")
    cams = wl.cameras
    P = sum(c.n_pixels for c in cams)
    r = Renderer(dev)
    ps = pack_scene(wl.scene)
    cfg = r.autotune(ps, cams, L.make_config(t_min=wl.t_min), backward=True)
    r.forward(ps, cams, cfg)
    torch.cuda.synchronize()
    stats = r.stats()
    K = stats.n_keys
    dL = torch.randn((P, 3), device="cuda", generator=torch.Generator("cuda").manual_seed(1)) * 1e-3
    step = GraphStep(r, ps, cams, cfg, max_keys=int(K * 1.05) + 4096, dL=dL)
    stream = torch.cuda.current_stream()

    def timed(fn, k):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / k

    ms = timed(step.replay, steps)
    img = torch.empty((P, 3), device="cuda")
    ms_fwd = timed(lambda: r.forward(ps, cams, cfg, out=img), steps)
    out = {"workload": "batch500k_16view", "weights": "bf16", "views": len(cams), "pixels": P,
           "tile": int(cfg.tile_size), "chunk": chunks_used(ps, cfg)[0], "bwd_chunk": chunks_used(ps, cfg)[1],
           "ctas_per_sm": {"fwd": int(stats.fwd_ctas_per_sm), "bwd": int(stats.bwd_ctas_per_sm)},
           "graph": True, "autotuned": True,
           "fwd_bwd_mpix_s": round(P / (ms * 1e-3) / 1e6, 3), "fwd_bwd_ms": round(ms, 3),
           "fwd_mpix_s": round(P / (ms_fwd * 1e-3) / 1e6, 3), "fwd_ms": round(ms_fwd, 3), "keys": int(K),
           "work": {"candidates": int(stats.n_candidates), "hits": int(stats.n_hits),
                    "composited": int(stats.n_composited)},
           "accuracy": "held to the same bars by tests/test_gpu_batched.py::"
                       "test_graph_step_matches_oracle_bf16_mlp64_16views (the graph-captured step, "
                       "16 uneven views at a quarter of these sizes) and tests/test_gpu_fullsize.py "
                       "(this workload at full size: keys bit-exact, sampled tiles)"}
    del step, r, ps, img, dL
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return out


def run_reference(args, rank, world):
    from paper_2510_08491_gb300 import synth
    if rank != 0:
        return None
    wl = synth.workload(args.workload)
    times, pxs = [], []
    for i in range(args.warmup + args.steps):
        npx, secs, cores = oracle_sample(wl, args.ref_tiles, seed=i)
        if i >= args.warmup:
            times.append(secs)
            pxs.append(npx)
    value = sum(pxs) / sum(times) / 1e6
    ms = 1e3 * sum(times) / len(times)
    return {"metric": METRIC, "value": round(value, 6), "unit": "Mpixel/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "step": "forward+backward (bounded sample)"},
            "cpu_baseline": {"value": round(value, 6), "unit": "Mpixel/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.ref_tiles} seeded 16x16 tiles per view per step"},
            "e2e": {"value": round(value, 6), "unit": "Mpixel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--cpu-tiles", type=int, default=16)
    ap.add_argument("--ref-tiles", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the BF16 batched graph form (batch500k_16view) beside the default workload")
    ap.add_argument("--cpu-baseline", action="store_true",
                    help="also time the oracle sample on a workload other than the default one")
    ap.add_argument("--graph", action="store_true", help="time replays of a captured CUDA graph of the step")
    ap.add_argument("--autotune", action="store_true", help="pick tile size and chunk with snp_autotune first")
    ap.add_argument("--tile", type=int, default=16, choices=(8, 16, 32), help="tile size (without --autotune)")
    ap.add_argument("--replay-color", action="store_true",
                    help="keep no colour store: the backward evaluates the colour network again")
    ap.add_argument("--train", action="store_true",
                    help="add the regulariser, the population-control statistic and an Adam step to every step "
                         "(eager, no graph) and time each of them alone")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as D
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        D.init_process_group("nccl")
    res = run_ours(args, rank, world) if args.impl == "ours" else run_reference(args, rank, world)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
    if world > 1 and args.impl == "ours":
        import torch.distributed as D
        D.destroy_process_group()


if __name__ == "__main__":
    main()
