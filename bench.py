"""Benchmark of the superquadric renderer's training step on GB300.

One step = one pass of the whole hot path over one synthetic six-camera frame
(4096 superquadrics, 6 x 225 x 400 rays, 100 samples per ray, 200x200x16 grid):
index build (ranges, count, scan, scatter, sort) -> forward render -> loss
gradient (CE + MSE of Supp. A.5) -> backward render.  Metric: ray-samples per
second through forward + backward (R * L / step time); ms_per_step is the
"ms per 6-camera frame".

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]
For N > 1 run under torchrun; every rank renders its own frame (seed 1 + rank),
no collective on the data path, and the timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2511_17361_gb300 import synth  # noqa: E402

WORKLOAD = 1
BWD_ORDER = 0  # SQ_BWD_DEFAULT; --bwd-order
# SFU instructions per (sample, primitive) pair: the forward's occupancy takes 4 lg2
# and 5 ex2, the backward's partial derivatives add 4 rcp
MUFU_MIX = {"fwd": {"ex2": 5, "lg2": 4, "rcp": 0}, "bwd": {"ex2": 5, "lg2": 4, "rcp": 4}}
MUFU_PER_PAIR = {k: sum(v.values()) for k, v in MUFU_MIX.items()}
# Nominal FP32 operations per pair for the FP32-pipe bound: the forward's transform,
# f and class sums (about 45), the backward about twice that.
FP32_PER_PAIR = {"fwd": 45, "bwd": 90}


def _fp32_pipe(dev, pairs, per_pair, ms):
    """The FP32-pipe bound of a pair kernel: pairs x per_pair FP32 operations in ms
    against 128 FP32 lanes per clock per SM at the top clock (2070 MHz)."""
    import torch
    peak = torch.cuda.get_device_properties(dev).multi_processor_count * 128 * 2070e6 / 1e9
    achieved = pairs * per_pair / (ms / 1e3) / 1e9
    return {"ops_per_pair": per_pair, "pairs": pairs, "peak": peak, "unit": "GFP32op/s", "achieved": achieved,
            "frac": achieved / peak}


def mix_peak(sfu, mix):
    """The SFU rate for a kernel's instruction mix: every instruction of the mix
    issued at its own measured rate, G instructions / s."""
    return sum(mix.values()) / sum(n / sfu[op] for op, n in mix.items() if n)
# DRAM traffic per launch from the committed ncu summaries, valid only while the
# kernel source is unchanged (sha256 of the file holding it).
NCU_TRAFFIC = {
    "k_backward": {"src": "sqr_bwd.cu", "src_sha": "1613935cf015e3f4", "bytes_per_launch": 309359616},
    "k_forward": {"src": "sqr_fwd.cu", "src_sha": "2c7c5b9d99e1072e", "bytes_per_launch": 1759382784},
    "k_bwd_sweep": {"src": "sqr_bwd.cu", "src_sha": "1613935cf015e3f4", "bytes_per_launch": 1920811520},
    "k_pm_tiles": {"src": "sqr_bwd_pm.cu", "src_sha": "7fc2f5f99959880c", "bytes_per_launch": 3747588864},
    "k_query_tiles": {"src": "sqr_query.cu", "src_sha": "9af6b77fa1963cdb", "bytes_per_launch": 1784576},
    "k_query_bwd": {"src": "sqr_query.cu", "src_sha": "9af6b77fa1963cdb", "bytes_per_launch": 56938752},
}


def _sha(path):
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def _traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, None once the source changed."""
    tr = NCU_TRAFFIC.get(kernel)
    if tr and tr["src_sha"] == _sha(os.path.join(ROOT, "paper_2511_17361_gb300", "csrc", tr["src"])):
        return tr["bytes_per_launch"]
    return None


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(x: float, world: int, device="cpu") -> float:
    """The slowest rank's value (timings are reported as the max over ranks)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, total_ms: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return world * units_per_rank / (total_ms / 1e3)


# ----------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if len(r) > 5 + i and r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------- reference arm (FP64 oracle)
def _oracle_sample(cfg, n_rays, seed=0):
    R = synth.n_rays(cfg["rig"])
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(R, size=min(n_rays, R), replace=False))


def oracle_step_time(cfg, index_np, ray_ids, targets, threads=0):
    """One oracle fwd + loss-gradient + bwd pass over ray_ids (seconds, threads used;
    threads = 0: all host cores)."""
    import oracle
    t0 = time.perf_counter()
    D, S, _, _ = oracle.render_fwd(cfg["prims"], cfg["grid"], index_np, cfg["rig"], cfg["t"], ray_ids=ray_ids,
                                   threads=threads)
    td, tl = targets
    R = len(ray_ids)
    e = np.exp(S - S.max(1, keepdims=True))
    gs = 2.0 / R * (e / e.sum(1, keepdims=True) - np.eye(S.shape[1])[tl[ray_ids]])
    gd = 0.05 / R * 2 * (D - td[ray_ids])
    oracle.render_bwd(cfg["prims"], cfg["grid"], index_np, cfg["rig"], cfg["t"], gd, gs, ray_ids=ray_ids,
                      threads=threads)
    return time.perf_counter() - t0, (threads if threads > 0 else oracle.max_threads())


def cpu_baseline(cfg, index_np, targets, budget_s=12.0, threads=0):
    """The FP64 oracle on a bounded random ray sample of the same frame."""
    probe = _oracle_sample(cfg, 600 if threads != 1 else 60, seed=1)
    t_probe, used = oracle_step_time(cfg, index_np, probe, targets, threads)
    total = synth.n_rays(cfg["rig"])
    n = int(min(total, max(len(probe), len(probe) * budget_s / max(t_probe, 1e-3))))
    ids = _oracle_sample(cfg, n, seed=2)
    t, used = oracle_step_time(cfg, index_np, ids, targets, threads)
    if t < 0.6 * budget_s and n < total:  # the small probe overstates the cost per ray: size again from this run
        n = int(min(total, n * budget_s / max(t, 1e-3)))
        ids = _oracle_sample(cfg, n, seed=2)
        t, used = oracle_step_time(cfg, index_np, ids, targets, threads)
    L = len(cfg["t"])
    return {"value": n * L / t, "unit": "ray-samples/s", "cores": used, "kind": "oracle",
            "sample": f"{n} random rays of the {cfg['name']} frame (index built by the oracle), "
                      f"forward + loss gradient + backward, FP64, {t:.1f} s"}


def cpu_extra_legs():
    """The other oracle timings on the host cores: the stress frame's 32x32-ray crop
    of camera 0 (forward + backward of seeded cotangents) and the grid query of
    the 8192-superquadric scene at all 640,000 voxel centres."""
    import oracle
    out = {}
    cfg = synth.make_config(2)
    idx = oracle.build_index(cfg["prims"], cfg["grid"])
    W = cfg["rig"]["W"]
    crop = np.array([(96 + i) * W + (184 + j) for i in range(32) for j in range(32)], np.int64)
    gd, gs = synth.cotangents(len(crop), 2)
    t0 = time.perf_counter()
    oracle.render_fwd(cfg["prims"], cfg["grid"], idx, cfg["rig"], cfg["t"], ray_ids=crop)
    oracle.render_bwd(cfg["prims"], cfg["grid"], idx, cfg["rig"], cfg["t"], gd.astype(np.float64),
                      gs.astype(np.float64), ray_ids=crop)
    t = time.perf_counter() - t0
    L = len(cfg["t"])
    out["stress_crop"] = {"value": len(crop) * L / t, "unit": "ray-samples/s", "cores": oracle.max_threads(),
                          "kind": "oracle", "sample": f"the 32x32-ray crop of camera 0 of {cfg['name']} (1024 rays), "
                                                      f"forward + backward, FP64, {t:.2f} s"}
    cfg = synth.make_config(4, seed=4)
    idx = oracle.build_index(cfg["prims"], cfg["grid"])
    t0 = time.perf_counter()
    oracle.query_grid(cfg["prims"], cfg["grid"], idx, tau=0.05)
    t = time.perf_counter() - t0
    nvox = int(np.prod(cfg["grid"]["n"]))
    out["query"] = {"value": nvox / t, "unit": "voxels/s", "cores": oracle.max_threads(), "kind": "oracle",
                    "sample": f"all {nvox} voxel centres of {cfg['name']} (density, semantics, label), "
                              f"FP64, {t:.2f} s"}
    return out


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    cfg = synth.make_config(WORKLOAD, seed=1)
    idx = oracle.build_index(cfg["prims"], cfg["grid"])
    targets = synth.loss_targets(synth.n_rays(cfg["rig"]), 1)
    # each step: a bounded sample sized so that warmup + steps finish in minutes
    probe = _oracle_sample(cfg, 300, seed=1)
    t_probe, threads = oracle_step_time(cfg, idx, probe, targets)
    per_step_budget = max(1.0, 120.0 / max(1, args.steps + args.warmup))
    n = int(max(100, min(synth.n_rays(cfg["rig"]), 300 * per_step_budget / max(t_probe, 1e-3))))
    times = []
    for s in range(args.warmup + args.steps):
        ids = _oracle_sample(cfg, n, seed=100 + s)
        t, threads = oracle_step_time(cfg, idx, ids, targets)
        if s >= args.warmup:
            times.append(t)
    L = len(cfg["t"])
    tot = sum(times)
    value = n * L * len(times) / tot
    line = {"metric": "ray-samples/s (forward + backward), six-camera frame", "value": value,
            "unit": "ray-samples/s", "impl": "reference", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg["name"], "rays_per_step": n, "samples_per_ray": L, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "ray-samples/s", "cores": threads, "kind": "oracle",
                             "sample": f"{n} random rays of the frame per step, FP64 forward + backward"},
            "e2e": {"value": value, "unit": "ray-samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------- GPU arm
def run_mine(args):
    import torch
    rank, world, local = _env_rank()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2511_17361_gb300 import _build
    _build.build()
    from paper_2511_17361_gb300 import sqr

    dev = torch.device("cuda", local)
    cfg = synth.make_config(WORKLOAD, seed=1 + rank)
    if args.cameras != 6:  # a smaller frame for profiler captures (the first k cameras of the ring)
        cfg["rig"] = synth.rig_ring(n_cam=args.cameras)
        cfg["name"] = cfg["name"].replace("ring6", f"ring{args.cameras}")
    grid = {"n": cfg["grid"]["n"], "lo": [float(v) for v in cfg["grid"]["lo"]],
            "vs": [float(v) for v in cfg["grid"]["vs"]]}
    prims = sqr.to_device(cfg["prims"], dev)
    rays = sqr.Rays.from_rig(cfg["rig"], cfg["t"], device=dev)
    R, L, C = rays.R, len(cfg["t"]), cfg["prims"]["logits"].shape[1]
    td_np, tl_np = synth.loss_targets(R, 1 + rank)
    td = torch.from_numpy(td_np).to(dev)
    tl = torch.from_numpy(tl_np).to(dev)

    imode = {"obb": sqr.SQ_INDEX_OBB, "cube": sqr.SQ_INDEX_CUBE, "opacity": sqr.SQ_INDEX_OBB_OPACITY}[args.index]
    flags = BWD_ORDER == 1  # the range-boundary flags serve only the ray-major backward
    ix = sqr.build_index(prims, grid, mode=imode, flags=flags)  # sizes V_sq (host sync once, before timing)
    P = ix.P()
    Q, in_grid = sqr.count_pairs(ix, grid, rays)
    depth = torch.empty(R, device=dev)
    sem = torch.empty((R, C), device=dev)
    tf = torch.empty(R, device=dev)
    loss_out = (torch.empty(1, device=dev), torch.empty(R, device=dev), torch.empty((R, C), device=dev))
    grads = {k: torch.empty_like(prims[k]) for k in sqr.PRIM_KEYS}
    saved = sqr.new_saved(rays, C, dev)

    def step(ev=None):
        if ev: ev[0].record()
        sqr.build_index(prims, grid, mode=imode, index=ix, sync=False)
        if ev: ev[1].record()
        sqr.render_fwd(prims, ix, grid, rays, out=(depth, sem, tf), saved=saved)
        if ev: ev[2].record()
        _, gd, gs = sqr.loss_ce_mse(depth, sem, td, tl, out=loss_out)
        if ev: ev[3].record()
        sqr.render_bwd(prims, ix, grid, rays, gd, gs, saved=saved, out=grads, order=BWD_ORDER)
        if ev: ev[4].record()

    step()
    # the saved state sized to the pages this frame's forward needs (+2%), the
    # buffer for every sample of every ray released before the memory peak is taken
    pages_needed, _ = sqr.saved_header(saved)
    saved_all_bytes = int(saved.numel())
    saved = sqr.new_saved(rays, C, dev, pages=pages_needed + pages_needed // 50 + 16)
    torch.cuda.empty_cache()
    torch.cuda.reset_peak_memory_stats(dev)
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    ix.check()

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > 129 MB L2
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    sampler = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    sqr.profile_enable(True)  # CUDA events around every library kernel, on its stream
    for s in range(args.steps):
        flush.fill_(float(s))
        step(evs[s])
    torch.cuda.synchronize()
    sqr.profile_enable(False)
    clocks = sampler.stop()
    kernel_ms = {k: sqr.profile_query(k) for k in ("k_forward", "k_backward", "k_pm_tiles", "k_bwd_sweep")}
    launches_timed, _, dropped = sqr.profile_query(None)
    phase = np.array([[evs[s][i].elapsed_time(evs[s][i + 1]) for i in range(4)] for s in range(args.steps)])
    step_ms = phase.sum(1)
    total_ms = max_over_ranks(float(step_ms.sum()), world, dev)
    if world > 1:
        torch.distributed.barrier()
    value = job_throughput(R * L * args.steps, world, total_ms)

    # ---- end to end through the public API: pinned host inputs in, gradients + loss out
    host_in = {k: torch.from_numpy(np.ascontiguousarray(cfg["prims"][k])).pin_memory() for k in sqr.PRIM_KEYS}
    host_in["td"], host_in["tl"] = torch.from_numpy(td_np).pin_memory(), torch.from_numpy(tl_np).pin_memory()
    host_in["K"] = torch.from_numpy(np.ascontiguousarray(cfg["rig"]["K"])).pin_memory()
    host_in["c2w"] = torch.from_numpy(np.ascontiguousarray(cfg["rig"]["cam2world"])).pin_memory()
    host_in["t"] = torch.from_numpy(np.ascontiguousarray(cfg["t"])).pin_memory()
    host_out = {k: torch.empty_like(host_in[k]).pin_memory() for k in sqr.PRIM_KEYS}
    host_loss = torch.empty(1).pin_memory()
    h2d = sum(v.numel() * v.element_size() for v in host_in.values())
    d2h = sum(v.numel() * v.element_size() for v in host_out.values()) + 4

    def e2e_step():
        for k in sqr.PRIM_KEYS:
            prims[k].copy_(host_in[k], non_blocking=True)
        td.copy_(host_in["td"], non_blocking=True)
        tl.copy_(host_in["tl"], non_blocking=True)
        rays.K.copy_(host_in["K"], non_blocking=True)
        rays.cam2world.copy_(host_in["c2w"], non_blocking=True)
        rays.t.copy_(host_in["t"], non_blocking=True)
        step()
        for k in sqr.PRIM_KEYS:
            host_out[k].copy_(grads[k], non_blocking=True)
        host_loss.copy_(loss_out[0], non_blocking=True)
        torch.cuda.current_stream().synchronize()

    e2e_step()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_ms = 0.0
    for s in range(args.steps):
        flush.fill_(float(s))
        e0.record()
        e2e_step()
        e1.record()
        torch.cuda.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    e2e_value = job_throughput(R * L * args.steps, world, e2e_ms)

    # ---- pairs evaluated: the backward's own per-primitive count of the pairs of
    # composited samples (one extra call, outside the timed region); the forward
    # evaluates the same pairs plus those of at most a chunk of samples past a ray's stop
    visits = torch.zeros(int(prims["means"].shape[0]), dtype=torch.int64, device=dev)
    sqr.render_bwd(prims, ix, grid, rays, loss_out[1], loss_out[2], saved=saved, out=grads,
                   order=sqr.SQ_BWD_PRIMITIVE_MAJOR, pair_visits=visits)
    q_eval = int(visits.sum().item())
    peak_mem = int(torch.cuda.max_memory_allocated(dev))
    saved_bytes = int(saved.numel())
    pages_after, save_status = sqr.saved_header(saved)
    assert save_status == sqr.SQ_OK and pages_after == pages_needed, "saved-state pages changed between steps"

    # ---- roofline of the pair kernels (SFU-bound: MUFU ops per pair) against the
    # measured SFU rate; frac_survey is the coarser count of every in-grid sample's
    # pairs Q, 9 MUFU each, against the nominal 16 MUFU/clk/SM at the top clock
    mean_phase = phase.mean(0)
    names = ["index", "fwd", "loss", "bwd"]
    props = torch.cuda.get_device_properties(dev)
    sm_count = props.multi_processor_count
    peak_mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    nominal = sm_count * 16 * peak_mhz * 1e6 / 1e9  # G MUFU ops / s
    # the FP32-pipe bound beside it: FP32_PER_PAIR over 128 FP32 lanes per clock per
    # SM at the top clock
    fp32_peak = sm_count * 128 * peak_mhz * 1e6 / 1e9  # G FP32 ops / s
    sfu = {op: sqr.measure_sfu(op) / 1e9 for op in ("ex2", "lg2", "rcp")}
    pair_kernels = {}
    for kname in ("k_forward", "k_backward", "k_pm_tiles"):
        n_launch, k_total_ms, _ = kernel_ms[kname]
        if n_launch == 0:
            continue
        k_mean_ms = k_total_ms / n_launch
        kind = "fwd" if kname == "k_forward" else "bwd"
        mufu, peak = MUFU_PER_PAIR[kind], mix_peak(sfu, MUFU_MIX[kind])
        achieved = q_eval * mufu / (k_mean_ms / 1e3) / 1e9
        pair_kernels[kname] = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak,
                               "unit": "GMUFUop/s", "frac": achieved / peak, "frac_evaluated": achieved / peak,
                               "frac_survey": Q * 9 / (k_mean_ms / 1e3) / 1e9 / nominal,
                               "mufu_per_pair": mufu, "pairs_evaluated": q_eval, "pairs_Q": Q,
                               "traffic": _traffic(kname), "kernel_ms_per_launch": k_mean_ms,
                               "fp32_pipe": {"ops_per_pair": FP32_PER_PAIR[kind], "pairs": q_eval, "peak": fp32_peak,
                                             "unit": "GFP32op/s",
                                             "achieved": q_eval * FP32_PER_PAIR[kind] / (k_mean_ms / 1e3) / 1e9,
                                             "frac": q_eval * FP32_PER_PAIR[kind] / (k_mean_ms / 1e3) / 1e9 /
                                             fp32_peak}}
    # the dominant kernel: the longer of the pair-evaluating kernels
    kdom = max(pair_kernels, key=lambda k: pair_kernels[k]["kernel_ms_per_launch"]) if pair_kernels else None
    roof = dict(pair_kernels[kdom]) if kdom else None
    if roof:
        roof["peak_source"] = (f"measured SFU rates (sq_measure_sfu: ex2/lg2/rcp {sfu['ex2']:.0f}/{sfu['lg2']:.0f}/"
                               f"{sfu['rcp']:.0f} G/s), combined for the kernel's mix of "
                               f"{roof['mufu_per_pair']} per pair; frac_survey: nominal {sm_count} SMs x 16/clk x "
                               f"{peak_mhz:.0f} MHz = {nominal:.0f} G/s")
    hbm_peak = _hbm_peak()
    # the HBM-bound kernel of the step: the backward's back-to-front sweep reads the
    # saved T_j, alpha_j, s_j of every composited sample (and t_j, gD, gS) and
    # writes (dL/dalpha_j, w_j); the composited counts come from the saved state
    CP = (C + 3) // 4 * 4
    composited = int(sqr.saved_counts(saved, rays, C).sum().item())
    sweep_bytes = composited * ((2 + CP) * 4 + 4 + 8) + R * (1 + C) * 4 + R * 4
    n_sw, sw_ms, _ = kernel_ms["k_bwd_sweep"]
    hbm = None
    if n_sw > 0:
        gbps = sweep_bytes / (sw_ms / n_sw / 1e3) / 1e9
        hbm = {"kernel": "k_bwd_sweep", "bound": "hbm", "algorithmic_bytes": sweep_bytes, "achieved_GBps": gbps,
               "frac": gbps / hbm_peak, "peak_gbs": hbm_peak, "traffic": _traffic("k_bwd_sweep"),
               "composited_samples": composited}

    line = {"metric": "ray-samples/s (forward + backward), six-camera frame", "value": value,
            "unit": "ray-samples/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": cfg["name"], "rays": R, "samples_per_ray": L, "superquadrics": int(
                prims["means"].shape[0]), "grid": list(grid["n"]), "index_entries_P": P, "pairs_Q": Q,
                "pairs_evaluated": q_eval, "in_grid_samples": in_grid, "composited_samples": composited,
                "index": {"obb": "OBB, tau_cut 0.01", "cube": "cube N_v = 5",
                          "opacity": "opacity-aware OBB, tau_cut 0.01"}[args.index],
                "l2": "flushed (256 MB write) between timed steps",
                "backward_order": {0: "primitive-major (the default)", 1: "ray-major",
                                   2: "primitive-major"}[BWD_ORDER],
                "parallelism": f"replicas x{world} (one frame per GPU)"},
            "phases_ms": {n: float(v) for n, v in zip(names, mean_phase)},
            "gpu_launches": launches_timed + dropped,
            "kernel_ms_per_launch": {k: (v[1] / v[0] if v[0] else None) for k, v in kernel_ms.items()},
            "e2e": {"value": e2e_value, "unit": "ray-samples/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "roofline": roof, "pair_kernels": pair_kernels, "sfu_measured_Gops": sfu, "hbm": hbm,
            "memory": {"peak_mem_bytes": peak_mem, "saved_state_bytes": saved_bytes,
                       "saved_state_pages": pages_needed, "saved_state_bytes_every_sample": saved_all_bytes,
                       "what": "torch.cuda.max_memory_allocated over the timed and end-to-end steps: inputs, "
                               "index, saved forward state (sized to the pages of composited samples the "
                               "forward needed, +2%), outputs, gradients and the library's workspaces "
                               "(all caller-owned torch tensors)"},
            "clocks": clocks}
    extras = world == 1 and not args.no_extras and args.cameras == 6 and args.index == "obb" and BWD_ORDER == 0
    if extras:
        # the other workloads, each a few seconds, after the frame's buffers are freed
        del saved, grads, loss_out, depth, sem, tf, flush, host_in, host_out
        torch.cuda.empty_cache()
        xs = max(3, min(args.steps, 5))
        line["stress_ab"] = stress_result(sqr, dev, xs, 2)
        torch.cuda.empty_cache()
        line["batched"] = batch_result(sqr, dev, "batch", xs, 2)
        torch.cuda.empty_cache()
        line["temporal"] = batch_result(sqr, dev, "temporal", xs, 2)
        torch.cuda.empty_cache()
        line["query"] = query_result(sqr, dev, max(5, args.steps), 3, sfu=sfu)
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        idx_np = oracle.build_index(cfg["prims"], cfg["grid"])
        line["cpu_baseline"] = cpu_baseline(cfg, idx_np, (td_np, tl_np), budget_s=args.cpu_budget)
        if extras:
            line["cpu_baseline"]["one_core"] = cpu_baseline(cfg, idx_np, (td_np, tl_np),
                                                            budget_s=max(3.0, args.cpu_budget / 3), threads=1)
            line["cpu_baseline"].update(cpu_extra_legs())
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ----------------------------------------------------------------------- other workloads
def _hbm_peak():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0)
    except Exception:
        return 6800.0


def _flush_buffer(dev):
    import torch
    return torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > 129 MB L2


def query_result(sqr, dev, steps, warmup, sfu=None):
    """Supp. A.4 grid query of the 8192-superquadric scene at all 640,000 voxel
    centres of the 200x200x16 grid (tau = 0.05): density, semantics and labels;
    then the voxel losses and the query backward."""
    import torch
    cfg = synth.make_config(4, seed=4)
    prims = sqr.to_device(cfg["prims"], dev)
    grid = {"n": cfg["grid"]["n"], "lo": [float(v) for v in cfg["grid"]["lo"]],
            "vs": [float(v) for v in cfg["grid"]["vs"]]}
    ix = sqr.build_index(prims, grid)
    P = ix.P()
    nvox = ix.v_n.numel()
    C = cfg["prims"]["logits"].shape[1]
    out = (torch.empty(nvox, device=dev), torch.empty((nvox, C), device=dev),
           torch.empty(nvox, dtype=torch.uint8, device=dev))
    # synthetic voxel labels (0..C-1 occupied class, C free) for the voxel losses
    rng = np.random.default_rng(4)
    vlab = torch.from_numpy(rng.integers(0, C + 1, nvox).astype(np.int32)).to(dev)
    lout = (torch.empty(3, device=dev), torch.empty(2, dtype=torch.int32, device=dev),
            torch.empty(nvox, device=dev), torch.empty((nvox, C), device=dev))
    grads = {k: torch.empty_like(prims[k]) for k in sqr.PRIM_KEYS}

    def backward():  # voxel CE + BCE losses, then the query backward of their gradients
        _, _, gd, gsem = sqr.loss_voxel(out[0], out[1], vlab, out=lout)
        sqr.query_grid_bwd(prims, ix, grid, gd, gsem, out=grads)

    for _ in range(max(3, warmup)):
        sqr.query_grid(prims, ix, grid, 0.05, out=out)
        backward()
    flush = _flush_buffer(dev)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    torch.cuda.synchronize()
    sqr.profile_enable(True)
    for s in range(steps):
        flush.fill_(float(s))
        ev[s][0].record()
        sqr.query_grid(prims, ix, grid, 0.05, out=out)
        ev[s][1].record()
        backward()
        ev[s][2].record()
    torch.cuda.synchronize()
    sqr.profile_enable(False)
    ms = sum(e[0].elapsed_time(e[1]) for e in ev) / steps
    ms_bwd = sum(e[1].elapsed_time(e[2]) for e in ev) / steps
    qk = "k_query_tiles"  # the tile-major kernel (grids up to 65535 per axis), else k_query
    n_q, q_ms, _ = sqr.profile_query(qk)
    if n_q == 0:
        qk = "k_query"
        n_q, q_ms, _ = sqr.profile_query(qk)
    n_qb, qb_ms, _ = sqr.profile_query("k_query_bwd")
    launches, _, dropped = sqr.profile_query(None)
    k_ms, kb_ms = q_ms / max(n_q, 1), qb_ms / max(n_qb, 1)
    if sfu is None:
        sfu = {op: sqr.measure_sfu(op) / 1e9 for op in ("ex2", "lg2", "rcp")}
    peak_f, peak_b = mix_peak(sfu, MUFU_MIX["fwd"]), mix_peak(sfu, MUFU_MIX["bwd"])
    # every voxel centre evaluates its whole list: P pairs, 9 MUFU each (13 in the backward)
    achieved, achieved_b = P * 9 / (k_ms / 1e3) / 1e9, P * 13 / (kb_ms / 1e3) / 1e9
    out_bytes = nvox * (1 + C) * 4 + nvox
    hbm_bytes = out_bytes + 4 * P + 8 * nvox
    return {"metric": "voxel queries/s (density + semantics + label), 200x200x16 grid",
            "value": nvox / (ms / 1e3), "unit": "voxels/s", "ms_per_step": ms, "steps": steps,
            "config": {"workload": cfg["name"], "superquadrics": int(prims["means"].shape[0]), "voxels": nvox,
                       "index_entries_P": P, "tau": 0.05, "l2": "flushed (256 MB write) between timed steps"},
            "gpu_launches": launches + dropped, "kernel_ms_per_launch": {qk: k_ms, "k_query_bwd": kb_ms},
            "backward": {"what": "voxel CE + BCE losses (sq_loss_voxel) and the query backward of their gradients",
                         "ms_per_step": ms_bwd, "value": nvox / (ms_bwd / 1e3), "unit": "voxels/s",
                         "roofline": {"bound": "alu", "kernel": "k_query_bwd", "achieved": achieved_b,
                                      "peak": peak_b, "unit": "GMUFUop/s", "frac": achieved_b / peak_b,
                                      "traffic": _traffic("k_query_bwd"),
                                      "fp32_pipe": _fp32_pipe(dev, P, FP32_PER_PAIR["bwd"], kb_ms)}},
            "roofline": {"bound": "alu", "kernel": qk, "achieved": achieved, "peak": peak_f,
                         "unit": "GMUFUop/s", "frac": achieved / peak_f, "traffic": _traffic(qk),
                         "fp32_pipe": _fp32_pipe(dev, P, FP32_PER_PAIR["fwd"], k_ms)},
            "sfu_measured_Gops": sfu,
            "hbm": {"kernel": qk, "bound": "hbm", "algorithmic_bytes": hbm_bytes,
                    "achieved_GBps": hbm_bytes / (k_ms / 1e3) / 1e9,
                    "frac": hbm_bytes / (k_ms / 1e3) / 1e9 / _hbm_peak(), "peak_gbs": _hbm_peak()}}


def run_query(args):
    import torch
    from paper_2511_17361_gb300 import _build
    _build.build()
    from paper_2511_17361_gb300 import sqr
    dev = torch.device("cuda", 0)
    sampler = ClockSampler(0)
    sampler.start()
    r = query_result(sqr, dev, args.steps, args.warmup)
    clocks = sampler.stop()
    line = {"metric": r.pop("metric"), "value": r.pop("value"), "unit": r.pop("unit"), "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r.pop("ms_per_step"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic"}
    r.pop("steps")
    line.update(r)
    line["clocks"] = clocks
    print(json.dumps(line))
    return 0


def batch_result(sqr, dev, kind, steps, warmup):
    """Twelve uneven scenes (kind "batch") or the 13 frames of a temporal horizon
    (kind "temporal"): per-scene launches vs one batched persistent launch per
    pass (autotuned), eager and captured in a CUDA graph."""
    import torch
    temporal = kind == "temporal"
    cfgs = synth.make_temporal_config() if temporal else synth.make_batch_config(3)
    scenes, targets = [], []
    for i, c in enumerate(cfgs):
        prims = sqr.to_device(c["prims"], dev)
        rays = sqr.Rays.from_rig(c["rig"], c["t"], device=dev)
        grid = {"n": c["grid"]["n"], "lo": [float(v) for v in c["grid"]["lo"]], "vs": [float(v) for v in c["grid"]["vs"]]}
        ix = sqr.build_index(prims, grid, flags=True)  # the autotuner also times the ray-major order
        sc = sqr.Scene(prims, ix, grid, rays, training=True)
        td, tl = synth.loss_targets(rays.R, 300 + i)
        C = c["prims"]["logits"].shape[1]
        targets.append((torch.from_numpy(td).to(dev), torch.from_numpy(tl).to(dev),
                        (torch.empty(1, device=dev), torch.empty(rays.R, device=dev),
                         torch.empty((rays.R, C), device=dev))))
        scenes.append(sc)
    samples = sum(sc.rays.R * sc.rays.t.numel() for sc in scenes)

    def loss_all():
        for sc, (td, tl, out) in zip(scenes, targets):
            sqr.loss_ce_mse(sc.depth, sc.sem, td, tl, out=out)
            sc.grad_depth.copy_(out[1])
            sc.grad_sem.copy_(out[2])

    def per_scene_step():
        for sc, (td, tl, out) in zip(scenes, targets):
            sqr.build_index(sc.prims, sc.grid, index=sc.index, sync=False)
            sqr.render_fwd(sc.prims, sc.index, sc.grid, sc.rays, out=(sc.depth, sc.sem, sc.t_final), saved=sc.saved)
            sqr.loss_ce_mse(sc.depth, sc.sem, td, tl, out=out)
            sqr.render_bwd(sc.prims, sc.index, sc.grid, sc.rays, out[1], out[2], saved=sc.saved, out=sc.grads)

    tuning = sqr.autotune(scenes, reps=2)
    saved_bytes = sum(sc.fit_saved() for sc in scenes)  # to the pages the tuned forward needed, +5%
    torch.cuda.empty_cache()

    def batched_step():
        for sc in scenes:
            sqr.build_index(sc.prims, sc.grid, index=sc.index, sync=False)
        sqr.render_batched(sqr.SQ_OP_FWD, scenes, tuning)
        loss_all()
        sqr.render_batched(sqr.SQ_OP_BWD, scenes, tuning)

    flush = _flush_buffer(dev)

    def timed(fn):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        for s in range(steps):
            flush.fill_(float(s))
            ev[s][0].record()
            fn()
            ev[s][1].record()
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / steps

    for _ in range(warmup):
        per_scene_step()
        batched_step()
    ms_per_scene = timed(per_scene_step)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        batched_step()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batched_step()
    ms_graph = timed(graph.replay)
    ms_batched = timed(batched_step)
    what = "13-frame temporal horizon (T = 6)" if temporal else "12-scene uneven batch"
    return {"metric": f"ray-samples/s (forward + backward), {what}", "value": samples / (ms_graph / 1e3),
            "unit": "ray-samples/s", "ms_per_step": ms_graph, "steps": steps,
            "config": {"workload": "temporal13_ring6_N1600" if temporal else "batch12_uneven", "scenes": len(scenes),
                       "ray_samples": samples,
                       "rays": [sc.rays.R for sc in scenes], "superquadrics": [int(sc.prims["means"].shape[0])
                                                                             for sc in scenes],
                       "samples_per_ray": [int(sc.rays.t.numel()) for sc in scenes], "tuning": tuning,
                       "l2": "flushed (256 MB write) between timed steps"},
            "per_scene_launches": {"ms_per_step": ms_per_scene, "value": samples / (ms_per_scene / 1e3)},
            "batched_eager": {"ms_per_step": ms_batched, "value": samples / (ms_batched / 1e3)},
            "batched_graph": {"ms_per_step": ms_graph, "value": samples / (ms_graph / 1e3)},
            "graph_over_per_scene": ms_per_scene / ms_graph, "saved_state_bytes": saved_bytes}


def run_batch(args):
    import torch
    from paper_2511_17361_gb300 import _build
    _build.build()
    from paper_2511_17361_gb300 import sqr
    dev = torch.device("cuda", 0)
    r = batch_result(sqr, dev, args.workload, args.steps, args.warmup)
    line = {"metric": r.pop("metric"), "value": r.pop("value"), "unit": r.pop("unit"), "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r.pop("ms_per_step"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic"}
    r.pop("steps")
    line.update(r)
    print(json.dumps(line), flush=True)
    return 0


def stress_result(sqr, dev, steps, warmup):
    """The backward stress frame (16,384 clustered superquadrics, six 225x400
    cameras, L = 100): index + forward, then the backward in each order (the
    ray-major run walk and the primitive-major tiles of Processes 2-3)."""
    import torch
    cfg = synth.make_config(2)
    grid = {"n": cfg["grid"]["n"], "lo": [float(v) for v in cfg["grid"]["lo"]],
            "vs": [float(v) for v in cfg["grid"]["vs"]]}
    prims = sqr.to_device(cfg["prims"], dev)
    rays = sqr.Rays.from_rig(cfg["rig"], cfg["t"], device=dev)
    R, L, C = rays.R, len(cfg["t"]), cfg["prims"]["logits"].shape[1]
    ix = sqr.build_index(prims, grid, flags=True)  # the ray-major order reads the range-boundary flags
    Q, _ = sqr.count_pairs(ix, grid, rays)
    saved = sqr.new_saved(rays, C, dev)
    depth, sem, _ = sqr.render_fwd(prims, ix, grid, rays, saved=saved)
    td, tl = synth.loss_targets(R, 2)
    _, gd, gs = sqr.loss_ce_mse(depth, sem, torch.from_numpy(td).to(dev), torch.from_numpy(tl).to(dev))
    grads = {k: torch.empty_like(prims[k]) for k in sqr.PRIM_KEYS}
    visits = torch.zeros(prims["means"].shape[0], dtype=torch.int64, device=dev)
    sqr.render_bwd(prims, ix, grid, rays, gd, gs, saved=saved, out=grads, order=sqr.SQ_BWD_PRIMITIVE_MAJOR,
                   pair_visits=visits)
    flush = _flush_buffer(dev)
    res = {"config": {"workload": cfg["name"], "rays": R, "samples_per_ray": L,
                      "superquadrics": int(prims["means"].shape[0]), "index_entries_P": ix.P(), "pairs_Q": Q,
                      "pairs_evaluated": int(visits.sum().item()), "max_list": int(ix.v_n.max().item())}}

    def timed(fn, kern):
        for _ in range(warmup):
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        sqr.profile_enable(True)
        for s in range(steps):
            flush.fill_(float(s))
            ev[s][0].record()
            fn()
            ev[s][1].record()
        torch.cuda.synchronize()
        sqr.profile_enable(False)
        n, kms, _ = sqr.profile_query(kern) if kern else (0, 0.0, 0)
        return sum(a.elapsed_time(b) for a, b in ev) / steps, (kms / n if n else None)

    ms_fwd, kf = timed(lambda: (sqr.build_index(prims, grid, index=ix, sync=False, flags=True),
                                sqr.render_fwd(prims, ix, grid, rays, saved=saved)), "k_forward")
    res["index_fwd_ms"], res["k_forward_ms"] = ms_fwd, kf
    for name, order, kern in (("ray_major", sqr.SQ_BWD_RAY_MAJOR, "k_backward"),
                              ("primitive_major", sqr.SQ_BWD_PRIMITIVE_MAJOR, "k_pm_tiles")):
        ms, km = timed(lambda: sqr.render_bwd(prims, ix, grid, rays, gd, gs, saved=saved, out=grads, order=order),
                       kern)
        res[name] = {"bwd_ms": ms, f"{kern}_ms": km, "ray_samples_per_s": R * L / ((ms + ms_fwd) / 1e3)}
    res["primitive_over_ray_major"] = res["ray_major"]["bwd_ms"] / res["primitive_major"]["bwd_ms"]
    return res


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["mine", "reference"], default="mine")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the frame workload (skip the stress A/B, batch, horizon and query keys)")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--index", choices=["obb", "cube", "opacity"], default="obb",
                    help="voxel neighbourhood of the frame workload's index (default: OBB, tau_cut 0.01)")
    ap.add_argument("--bwd-order", choices=["default", "ray", "primitive"], default="default",
                    help="backward order (Sec. 3.3.3): ray-major run walk or primitive-major tiles")
    ap.add_argument("--cameras", type=int, choices=range(1, 7), default=6,
                    help="cameras of the frame workload's ring (default 6; fewer give a smaller case for ncu)")
    ap.add_argument("--workload", choices=["frame", "batch", "temporal", "query"], default="frame",
                    help="frame: one six-camera frame (default); batch: 12 uneven scenes, batched vs per scene; "
                         "temporal: the 13 frames of a T = 6 horizon, batched vs per frame; "
                         "query: grid query of an 8192-superquadric scene at all 640,000 voxel centres")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        args.warmup = 3
    global BWD_ORDER
    BWD_ORDER = {"default": 0, "ray": 1, "primitive": 2}[args.bwd_order]
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("batch", "temporal"):
        return run_batch(args)
    if args.workload == "query":
        return run_query(args)
    return run_mine(args)


if __name__ == "__main__":
    sys.exit(main())
