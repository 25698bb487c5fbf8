"""Benchmark: model visibilities per second for one major cycle's prediction.

Workload (default, the largest that fits one GPU): 256 antennas in a 10 km
disc, 490 hour angles over -1h .. +1h, 15 993 600 visibilities at 1.4 GHz,
with 50 000 clean components in 20 Gaussian blobs inside a 2 deg field,
wavelet level J = 12 (synthetic, seeded; see synth/). --workload medium
takes the medium array (64 antennas, 1 008 000 visibilities, 5 000
components) instead; the medium step is also reported beside the headline.

One step = the whole hot path over that batch:
  wt_build_tree (components -> sphere pixels -> coefficient tree, Sec. 3.5)
  -> wt_predict_vis (Eq. 17 per visibility, the chosen form)
  -> subtract_model (V_resid = V - V_M, Sec. 2.2).
The chosen form is WT_MIXED_FAST with the regrouped Eq. 17 (float64-accurate
phase, sin/cos from the special-function unit, compensated float32
accumulation), whose error against the FP64 oracle is measured in the same
run and must stay <= 1e-6 of the peak amplitude sum |C|; the plain float64
form is timed on the same batch beside it.

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events
on the launching stream; the L2 cache is flushed (a 512 MB write) before
every timed step, outside the events. Inputs are resident in HBM. Under
torchrun the batch is world x 490 hour angles and each rank takes its
contiguous block of 490 (weak scaling), and the max time over ranks is
reported. The e2e figure repeats the step through the public API from
pinned host buffers, host<->device copies inside the timed region. The
rooflines divide by the pipe rates wt_measure_pipe_rates measures on the
same GPU.

--impl reference times the CPU oracle (as it stands, OpenMP over the
visibilities on every host core) on a bounded strided sample of the same
workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

MEDIUM_J = 12
METRIC = "model visibilities/s"
UNIT = "vis/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--J", type=int, default=MEDIUM_J)
    p.add_argument("--workload", default=None, choices=["large", "medium"],
                   help="the batch of the headline step: large (256 antennas, 15 993 600 visibilities, 50 000 "
                        "components; the default) or medium (64 antennas, 1 008 000 visibilities, 5 000 "
                        "components; the default of --forms-once)")
    p.add_argument("--form", default="fast", choices=["fast", "mixed"],
                   help="chosen form of the step: WT_MIXED_FAST (default) or WT_MIXED")
    p.add_argument("--sum", default="regrouped", choices=["regrouped", "explicit"],
                   help="evaluation order of Eq. 17 in the step: regrouped (V = sum_n w_n eta_n, default) or "
                        "explicit (eta and the three sigma per node)")
    p.add_argument("--no-extras", action="store_true", help="skip the per-form side measurements")
    p.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    p.add_argument("--forms-once", action="store_true",
                   help="run each predictor once on the medium workload after one warm-up (a bounded "
                        "command for profilers); prints nothing but a short summary")
    p.add_argument("--only", default="",
                   help="with --forms-once: comma-separated names of the calls to run (default: all)")
    p.add_argument("--sweep", action="store_true",
                   help="print the run-time scaling study (J and distinct-component sweeps, paper-context "
                        "workload) as one JSON line instead of the benchmark line")
    return p.parse_args()


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, reasons)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- ranks

def max_over_ranks(values, dist, device):
    """Element-wise maximum of per-rank timings (the slowest rank sets the
    whole job's time)."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


# ---------------------------------------------------------------- native

def tree_launches(J):
    """libwtvis kernels per wt_build_tree: map 1, radix sort (3 per pass of 8
    key bits over 2J + 2 bits), gather 1, levels 1, records 1."""
    passes = (2 * J + 2 + 7) // 8
    return 4 + 3 * passes


def predictor_launches(wt, which):
    """libwtvis kernels per wt_predict_vis in a mixed form: the regrouped
    Eq. 17 runs as a grid pass and an exact pass over the tiles it leaves."""
    return 2 if which == wt.WT_SUM_EQ17_REGROUPED else 1


def time_steps(wt, torch, w, J, mode, which, steps, warmup, dev, flush, clocks=None, dist=None, world=1):
    """W untimed steps, then K timed steps of build + predict + subtract on
    the resident inputs of workload w; per step the whole step and the
    predictor are timed by CUDA events on the launching stream, L2 flushed
    before each step (outside the events)."""
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    l, m, fl, uvw = d(w.l), d(w.m), d(w.flux), d(w.uvw)
    n_vis = w.n_vis
    rng = np.random.default_rng(7)
    obs = d((rng.standard_normal(n_vis) + 1j * rng.standard_normal(n_vis)).astype(np.complex64))
    model = torch.empty(n_vis, dtype=torch.complex64, device=dev)
    resid = torch.empty_like(model)
    stream = torch.cuda.current_stream(dev)
    for _ in range(warmup):
        t = wt.wt_build_tree(l, m, fl, w.ra0, w.dec0, J)
        wt.wt_predict_vis(t, uvw, mode=mode, which=which, out=model)
        wt.subtract_model(obs, model, mode=mode, out=resid)
        t.close()
    torch.cuda.synchronize()
    wt.wt_device_status()
    times, pred_times = [], []
    if dist is not None and world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.start()
    for _ in range(steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tree = wt.wt_build_tree(l, m, fl, w.ra0, w.dec0, J)
        p0.record(stream)
        wt.wt_predict_vis(tree, uvw, mode=mode, which=which, out=model)
        p1.record(stream)
        wt.subtract_model(obs, model, mode=mode, out=resid)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        pred_times.append(p0.elapsed_time(p1) / 1e3)
        tree.close()
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks is not None else None
    if dist is not None and world > 1:
        dist.barrier()
    wt.wt_device_status()
    tree = wt.wt_build_tree(l, m, fl, w.ra0, w.dec0, J)
    info = tree.info()
    return dict(t_step=statistics.mean(times), t_pred=statistics.mean(pred_times), clocks=clk, info=info,
                tree=tree, tensors=(l, m, fl, uvw, obs, model, resid),
                launches_per_step=tree_launches(J) + predictor_launches(wt, which) + 1)


def e2e_steps(wt, torch, w, J, mode, which, steps, warmup, dev, flush, tensors):
    """The step through the public API from pinned host buffers: uploads of
    the components, baselines and observed visibilities, the build, the
    prediction and subtraction, and the download of the residuals, all
    inside the timed region (the visibilities in E2E_CHUNKS pieces on two
    streams, so that one piece's copies overlap another's prediction; the
    uploads start with the step and overlap the tree build)."""
    l, m, fl, uvw, obs, model, resid = tensors
    n_vis = w.n_vis
    stream = torch.cuda.current_stream(dev)
    hl, hm, hf = (torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (w.l, w.m, w.flux))
    huvw = torch.from_numpy(np.ascontiguousarray(w.uvw)).pin_memory()
    hobs = obs.cpu().pin_memory()
    hres = torch.empty_like(hobs).pin_memory()
    dl, dm, df = torch.empty_like(l), torch.empty_like(m), torch.empty_like(fl)
    duvw, dobs = torch.empty_like(uvw), torch.empty_like(obs)
    side = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]
    bounds = np.linspace(0, n_vis, E2E_CHUNKS + 1).astype(int)
    e2e_times = []
    for it in range(warmup + steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dl.copy_(hl, non_blocking=True)
        dm.copy_(hm, non_blocking=True)
        df.copy_(hf, non_blocking=True)
        tree = wt.wt_build_tree(dl, dm, df, w.ra0, w.dec0, J)
        built = torch.cuda.Event()
        built.record(stream)
        for c in range(E2E_CHUNKS):
            a, b = int(bounds[c]), int(bounds[c + 1])
            s2 = side[c % 2]
            s2.wait_event(e0)
            with torch.cuda.stream(s2):
                duvw[a:b].copy_(huvw[a:b], non_blocking=True)
                dobs[a:b].copy_(hobs[a:b], non_blocking=True)
                s2.wait_event(built)
                wt.wt_predict_vis(tree, duvw[a:b], mode=mode, which=which, out=model[a:b], stream=s2)
                wt.subtract_model(dobs[a:b], model[a:b], mode=mode, out=resid[a:b], stream=s2)
                hres[a:b].copy_(resid[a:b], non_blocking=True)
        for s2 in side:
            stream.wait_stream(s2)
        e1.record(stream)
        e1.synchronize()
        tree.close()
        if it >= warmup:
            e2e_times.append(e0.elapsed_time(e1) / 1e3)
    h2d = sum(x.numel() * x.element_size() for x in (hl, hm, hf, huvw, hobs))
    d2h = hres.numel() * hres.element_size()
    return statistics.mean(e2e_times), h2d, d2h


def pipe_peaks(wt, torch, sm_max_mhz):
    """Pipe peaks of this GPU from wt_measure_pipe_rates (per clock per SM)
    times the SM count and the maximum SM clock; nominal figures when the
    measurement fails."""
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = sm_max_mhz or 2070.0
    try:
        r = wt.wt_measure_pipe_rates()
        src = "wt_measure_pipe_rates on this GPU (per clock per SM) x %d SMs x %.0f MHz" % (n_sm, mhz)
    except Exception as e:   # noqa: BLE001 - reported in the line
        r = {"ffma": 128.0, "ffma2_elems": 128.0, "dfma": 2.0, "mufu_sin": 16.0, "mufu_tanh": 16.0,
             "mufu_tanh_bf16x2_elems": 32.0, "mufu_ex2": 16.0}
        src = "nominal (%d SMs x 128 FP32 / 2 FP64 / 16 SFU lanes x %.0f MHz); probe failed: %s" % (n_sm, mhz, e)
    hz = mhz * 1e6
    return {"fp32_tflops": 2.0 * r["ffma"] * n_sm * hz / 1e12,          # an FMA is 2 flops
            "fp32_top_s": r["ffma"] * n_sm * hz / 1e12,                # FMA-pipe element ops
            "fp64_tflops": 2.0 * r["dfma"] * n_sm * hz / 1e12,
            "fp64_inst_per_s": r["dfma"] * n_sm * hz,
            "sfu_top_s": r["mufu_sin"] * n_sm * hz / 1e12,
            "sfu_tanh_top_s": r["mufu_tanh"] * n_sm * hz / 1e12,
            "sfu_tanh_bf16x2_top_s": r["mufu_tanh_bf16x2_elems"] * n_sm * hz / 1e12,
            "sfu_ex2_top_s": r["mufu_ex2"] * n_sm * hz / 1e12,
            "per_clk_per_sm": r, "n_sm": n_sm, "sm_mhz": mhz, "peak_source": src}


def wavelet_roofline(info, n_vis, J, t_pred, peaks, form, summ, traffic):
    """Roofline of the wavelet predictor for one launch over n_vis
    visibilities taking t_pred seconds. The fraction is of the method's
    algorithmic work per visibility: a phase of 7 flops per leaf (three
    products and two sums of B.s, the rounding to the nearest integer and its
    subtraction) and 40 flops per tree node (the eta recursion, the
    Hadamard butterflies of the three sigma and the gamma sigma products),
    against the measured float32 peak; the leaves' sin and cos (2 per leaf)
    against the special-function unit's measured rate. pipe_busy is the
    form's own float32 FMA-pipe element ops (the double-float phase
    emulation included) against the FMA pipe's measured element rate."""
    n_leaves, n_nodes = info["n_leaves"], info["n_nodes"]
    flops = n_vis * (ALG_FLOPS_PHASE_PER_LEAF * n_leaves + ALG_FLOPS_PER_NODE * n_nodes)
    achieved = flops / t_pred / 1e12
    sfu = n_vis * 2 * n_leaves / t_pred / 1e12
    op_leaf, op_node, op_low = OPS[(form, summ)]
    n_low = int(info["per_level"][J - 2]) if J >= 3 else 0
    ops = n_vis * (op_leaf * n_leaves + op_node * (n_nodes - n_leaves - n_low) + op_low * n_low)
    busy = ops / t_pred / 1e12
    return {
        "bound": "alu",
        "achieved": achieved,
        "peak": peaks["fp32_tflops"],
        "unit": "TFLOP/s (float32; algorithmic: 7 flops per (vis, leaf) phase + 40 per (vis, tree node))",
        "frac": achieved / peaks["fp32_tflops"],
        "peak_source": peaks["peak_source"],
        "algorithmic_flops_per_launch": flops,
        "sfu": {"achieved": sfu, "peak": peaks["sfu_top_s"], "unit": "T op/s (sin and cos of each leaf)",
                "frac": sfu / peaks["sfu_top_s"], "peak_source": peaks["peak_source"]},
        "pipe_busy": {"achieved": busy, "peak": peaks["fp32_top_s"],
                      "unit": "T op/s (the form's own float32 FMA-pipe element ops, phase emulation included)",
                      "frac": busy / peaks["fp32_top_s"], "ops_per_leaf": op_leaf,
                      "ops_per_internal_node": op_node, "ops_per_level_J_minus_1_node": op_low},
        "traffic": traffic,
        "traffic_note": ("dram__bytes_read.sum + dram__bytes_write.sum of one launch of this form on this "
                         "workload (profiles/)" if traffic is not None else "not captured for this form and size"),
        "algorithmic_bytes": 32 * n_vis,
        "kernel": "k_wavelet_mixed (Eq. 17 %s), one CTA per tile of visibilities" % summ,
        "launch_ms": t_pred * 1e3,
    }


def native(args):
    import torch
    import torch.distributed as dist

    import paper_1909_03956_gb300 as wt

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wt.load()

    J = args.J
    w = synth.large(J=J, shard=(rank, world)) if args.workload == "large" else shard_workload(synth.medium(J=J),
                                                                                             rank, world)
    n_vis = w.n_vis
    S = float(np.abs(w.flux).sum())
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    mode = wt.WT_MIXED_FAST if args.form == "fast" else wt.WT_MIXED
    which = wt.WT_SUM_EQ17_REGROUPED if args.sum == "regrouped" else wt.WT_SUM_EQ17
    stream = torch.cuda.current_stream(dev)

    clocks = ClockSampler(local)
    hd = time_steps(wt, torch, w, J, mode, which, args.steps, args.warmup, dev, flush, clocks, dist, world)
    t_step, t_pred, clk, info, tree_keep = hd["t_step"], hd["t_pred"], hd["clocks"], hd["info"], hd["tree"]
    if world > 1:
        t_step, t_pred = max_over_ranks([t_step, t_pred], dist, dev)
    l, m, fl, uvw, obs, model, resid = hd["tensors"]
    peaks = pipe_peaks(wt, torch, clk.get("sm_max_mhz") if clk else None)

    # accuracy of the chosen form against the FP64 oracle on a strided sample
    err = None
    if rank == 0:
        import oracle as O
        idx = np.arange(0, n_vis, max(1, n_vis // 4000))
        ot = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, J)
        ref = ot.vis_eq17(w.uvw[idx], threads=os.cpu_count() or 1)
        err = float(np.max(np.abs(model.cpu().numpy()[idx] - ref)) / S)

    # the plain float64 form (explicit Eq. 17) on the same batch: one call
    out64 = torch.empty(n_vis, dtype=torch.complex128, device=dev)
    wt.wt_predict_vis(tree_keep, uvw, mode=wt.WT_FP64, which=wt.WT_SUM_EQ17, out=out64)
    t_fp64 = _time_call(lambda: wt.wt_predict_vis(tree_keep, uvw, mode=wt.WT_FP64, which=wt.WT_SUM_EQ17,
                                                  out=out64), stream, flush, reps=1)
    del out64

    t_e2e, h2d, d2h = e2e_steps(wt, torch, w, J, mode, which, args.steps, args.warmup, dev, flush, hd["tensors"])
    if world > 1:
        (t_e2e,) = max_over_ranks([t_e2e], dist, dev)

    extras = {}
    if rank == 0 and not args.no_extras:
        med = synth.medium(J=MEDIUM_J)
        md = time_steps(wt, torch, med, MEDIUM_J, mode, which, min(args.steps, 20), 3, dev, flush)
        extras["medium"] = {
            "workload": med.name, "n_vis": med.n_vis, "n_comp": med.n_comp, "J": MEDIUM_J,
            "n_leaves": md["info"]["n_leaves"], "n_nodes": md["info"]["n_nodes"],
            "value": med.n_vis / md["t_step"], "unit": UNIT, "ms_per_step": md["t_step"] * 1e3,
            "predict_ms": md["t_pred"] * 1e3,
            "roofline": wavelet_roofline(md["info"], med.n_vis, MEDIUM_J, md["t_pred"], peaks, args.form, args.sum,
                                         TRAFFIC_BYTES.get((med.name, args.form, args.sum)))}
        mtree, mt = md["tree"], md["tensors"]
        extras.update(side_measurements(wt, torch, med, mt[0], mt[1], mt[2], mt[3], mtree, stream, flush, peaks))
        mtree.close()
        del md, mt
        extras["major_cycle"] = major_cycle_measurement(wt, torch, dev, stream, flush)
        extras["batched"] = batched_measurement(wt, torch, dev, stream, flush, peaks)
        extras["mixed_config"] = mixed_measurement(wt, torch, dev, stream, flush)
        extras["learned"] = learned_measurement(wt, torch, dev, stream, flush)
    tree_keep.close()

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    roof = wavelet_roofline(info, n_vis, J, t_pred, peaks, args.form, args.sum,
                            TRAFFIC_BYTES.get((w.name, args.form, args.sum)))
    value = world * n_vis / t_step
    fp64_value = world * n_vis / t_fp64
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_step * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("f32+f64 (double-float phase, f32 SFU sincos, Kahan f32 sum, packed f32 pairs)"
                  if args.form == "fast"
                  else "f32+f64 (double-float phase, f32 polynomial sincos, Kahan f32 sum, packed f32 pairs)"),
        "data": "synthetic (seeded; stand-in for the paper's simulated VLA data)",
        "config": {
            "workload": w.name,
            "n_vis": n_vis,
            "n_comp": w.n_comp,
            "J": J,
            "n_leaves": info["n_leaves"],
            "n_nodes": info["n_nodes"],
            "form": ("wavelet Eq.17 " + ("regrouped" if args.sum == "regrouped" else "explicit") + ", "
                     + ("WT_MIXED_FAST" if args.form == "fast" else "WT_MIXED")),
            "step": "wt_build_tree + wt_predict_vis + subtract_model",
            "parallelism": ("dp%d (one batch of %d x 490 hour angles; each rank a contiguous block of 490, "
                            "the tree built per rank from the same component list)" % (world, world)
                            if args.workload == "large" else
                            "dp%d (each rank a contiguous range of the batch's visibilities, the tree built "
                            "per rank from the same component list)" % world),
            "l2": "flushed (512 MB write) before every timed step; inputs larger than L2",
        },
        "vis_terms_per_s": value * info["n_leaves"],
        "vis_nodes_per_s": value * info["n_nodes"],
        "max_rel_err_vs_fp64_oracle": err,
        "fp64_plain": {"form": "wavelet Eq.17 explicit, WT_FP64 (float64 throughout)",
                       "vis_per_s": fp64_value, "predict_ms": t_fp64 * 1e3,
                       "chosen_over_fp64_predictor": t_fp64 / t_pred,
                       "chosen_step_over_fp64_predictor": value / fp64_value},
        "predict_ms": t_pred * 1e3,
        "roofline": roof,
        "pipe_peaks": peaks,
        "e2e": {"value": world * n_vis / t_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "note": "tree build, then the visibilities in %d pieces on two streams (copies overlap "
                        "predictions), all copies inside the timed region" % E2E_CHUNKS},
        "gpu_launches": hd["launches_per_step"] * args.steps,
        "gpu_launches_per_step": hd["launches_per_step"],
        "clocks": clk,
    }
    line.update(extras)
    if not args.no_cpu and world == 1:
        line["cpu_baseline"] = cpu_baseline(w, J, budget_s=8.0)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def shard_workload(w, rank, world):
    """Rank r of `world` takes the contiguous r-th range of the batch's
    visibilities; every rank keeps the whole component list (each builds the
    same tree from it). One rank: the workload unchanged."""
    if world <= 1:
        return w
    a, b = shard_range(w.n_vis, rank, world)
    return synth.Workload(w.name + "_shard%dof%d" % (rank, world), w.uvw[a:b], w.l, w.m, w.flux, w.J,
                          w.ra0, w.dec0, w.freq_hz, dict(w.extra))


def shard_range(n, rank, world):
    """[a, b) of rank `rank`: contiguous, in rank order, sizes differing by at
    most one."""
    return n * rank // world, n * (rank + 1) // world


# Algorithmic flops per visibility of the wavelet route: per leaf the phase
# B.(s - P) (3 multiplies, 2 adds, rounding to the nearest integer and its
# subtraction); per tree node (leaves included) the eta recursion (6 complex
# adds), the Hadamard butterflies of the three sigma (about 8 complex adds)
# and the three complex x real gamma sigma products.
ALG_FLOPS_PHASE_PER_LEAF = 7
ALG_FLOPS_PER_NODE = 40


# Float32 FMA-pipe operations (adds, multiplies, FMAs; a packed pair counts
# 2) of the mixed Eq. 17 forms, counted from each form's arithmetic at two
# visibilities per thread (the bench's launch shape); instruction overhead
# (record decode, loads, stores, branches, register moves, roundings to
# integer) is not counted, and the special-function unit's sin and cos are
# counted separately against that unit's own peak. A complex add is 2 ops.
#   phase (every leaf): three double-float products (4 each), two
#     error-free sums (6 each), reduction by the nearest integer (1), tail
#     (4): 29.
#   polynomial sin/cos: quadrant reduction and angle (5), sin and cos
#     polynomials (5 each): 15 (the quadrant selection runs on the ALU).
#   fast sin/cos: the angle (2) and the SFU argument scaling (1): 3, plus
#     sin and cos on the special-function unit (2 SFU ops).
#   explicit internal node: butterflies (8), xi (2), three sigma (6),
#     gamma.sigma (6), Kahan add (8): 30.
#   regrouped: a leaf adds xi to its parent's sum (2) and w xi to its
#     parent's plain sum of leaf terms (2); a node at level J - 1 adds w xi
#     to its leaves' sum (2) and that to its parent's plain sum (2); any
#     other internal node adds w xi (plus, at level J - 2, its children's
#     sum) to V (2, with a Kahan add of 8); every internal node passes xi to
#     its parent's sum (2).
OPS_PHASE = 12 + 12 + 1 + 4
# The regrouped forms' phase on the head grid: per coordinate the head on the
# grid (2), its remainder (1) and the two cross terms (2); the heads' sum (2),
# the reduction (1), the tails' sum (2): 20.
OPS_PHASE_GRID = 3 * 5 + 2 + 1 + 2
OPS_LEAF = OPS_PHASE + 15
OPS_NODE = 30
OPS_LEAF_FAST = OPS_PHASE + 3
OPS_RG_LEAF = 2 + 2
OPS_RG_NODE = 2 + 8 + 2
OPS_RG_LOW = 2 + 2 + 2
# (form, sum) -> (per leaf, per internal node, per internal node at level J - 1)
OPS = {("mixed", "explicit"): (OPS_LEAF, OPS_NODE, OPS_NODE),
       ("fast", "explicit"): (OPS_LEAF_FAST, OPS_NODE, OPS_NODE),
       ("mixed", "regrouped"): (OPS_LEAF - OPS_PHASE + OPS_PHASE_GRID + OPS_RG_LEAF, OPS_RG_NODE, OPS_RG_LOW),
       ("fast", "regrouped"): (OPS_LEAF_FAST - OPS_PHASE + OPS_PHASE_GRID + OPS_RG_LEAF, OPS_RG_NODE, OPS_RG_LOW)}
SFU_OPS_LEAF = {"fast": 2, "mixed": 0}
# DRAM bytes of one k_wavelet_mixed launch at J = 12, from ncu
# (dram__bytes_read.sum + dram__bytes_write.sum), per (workload, form, sum);
# a form whose kernel or launch shape changed since its capture has no entry.
TRAFFIC_BYTES = {("large_256ant_15993600vis_50000comp", "fast", "regrouped"): 388_350_000 + 107_320_000}
# Double-float form (WT_FP64_DF, regrouped Eq. 17), float32 FMA-pipe ops per
# (vis, leaf): phase 32 (three double-float products of 5, two error-free
# sums of 6, reduction 1, tail 4), sin/cos 135 (argument reduction 8, 2 pi f,
# x^2, x^3 and x^3/6 as double-float products of 7, the float32 tails 6,
# three double-float sums of 10-11 and one of 11, the rotation by the table
# entry: four products of 7 and two sums of 11), w eta into V 36, the
# parent's sum 22; per (vis, internal node): quarter 4, w eta into V 36, the
# parent's sum 22.
OPS_DF_LEAF = 32 + 135 + 36 + 22
OPS_DFT_DF = 32 + 135 + 36   # per (vis, component) of the double-float direct sum
OPS_DF_NODE = 4 + 36 + 22
# Direct sum (k_dft_mixed, two visibilities x two components per step), FMA-pipe
# element ops per (visibility, component): phase 20 on the head grid (the
# grid pass; the exact pass's 29 only for tiles beyond the grid's range),
# angle and SFU scaling 3 (fast) or polynomial sin/cos 15, the flux times
# (cos, sin) 2, half a Kahan add of a pair of terms 4. float64 (k_dft_fp64), FP64-pipe instructions per
# term: phase 3, table reduction and polynomials 14, rotation by the table
# entry 2 (+2 multiplies), multiply-add into V 2 -> 21 (roundings to integer
# and the table load not counted).
OPS_DFT_FAST = OPS_PHASE_GRID + 3 + 2 + 4
OPS_DFT = OPS_PHASE_GRID + 15 + 2 + 4
OPS_DFT_FP64 = 21
# Direct sum with the phase on the tensor cores (k_dft_tc), FMA-pipe element
# ops per (visibility, component) in the epilogue: the accumulators'
# recombination modulo 1 7, the angle 2, the SFU's scaling 1, the flux times
# (cos, sin) 2, a Kahan add of a pair per eight terms 1 -> 13. Tensor cores:
# four MMAs of K = 16 per (visibility, component), 128 flops.
OPS_DFT_TC = 13
TC_FLOPS_DFT_TERM = 128
# Algorithmic work per (visibility, component) of the direct sum: the phase
# (3 multiplies, 2 adds), its reduction (rounding and subtraction), the
# complex multiply-add by a real flux (4): 11 flops, plus one sin and one cos.
ALG_FLOPS_DFT_TERM = 11
# Hardware tanh per sample of the learned response's inference: the SiLU of
# both hidden layers of 64 units.
MLP_TANH_PER_SAMPLE = 128
# Passes over the training samples of each response network (Adam, batches
# of 8 192, learning rate 3e-3 with cosine decay). Measured on the large
# workload's levels 10 and 9 (10 M samples each): 2 passes left response
# errors of 0.25 and 0.46 RMS, 8 passes 0.13 and 0.21, 24 passes 0.088 and
# 0.093 (2.2 s of training per network).
MLP_TRAIN_EPOCHS = 24
# Pieces of the batch in the end-to-end leg (copies of one overlap the prediction of another).
E2E_CHUNKS = 4
# Measured copy bandwidth (hbm_gbs) and cuBLAS bf16 GEMM throughput (burst,
# bf16_tflops) of the GB300s this runs on, from MEASURED_PEAKS.json beside
# this file when it is there, else an earlier measurement on a GB300.
def _measured_peaks():
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "MEASURED_PEAKS.json"
    except (OSError, ValueError, KeyError, TypeError):
        return 6690.1, 1861.7, "earlier measurement on a GB300"


HBM_PEAK_GBPS, BF16_PEAK_TFLOPS, PEAKS_SOURCE = _measured_peaks()


def _time_call(fn, stream, flush, reps=3):
    import torch
    ts = []
    for _ in range(reps):
        flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b) / 1e3)
    return statistics.median(ts)


def side_measurements(wt, torch, w, l, m, fl, uvw, tree, stream, flush, peaks):
    n = w.n_vis
    info = tree.info()
    n_leaves, n_int = info["n_leaves"], info["n_nodes"] - info["n_leaves"]
    out64 = torch.empty(n, dtype=torch.complex128, device=uvw.device)
    out32 = torch.empty(n, dtype=torch.complex64, device=uvw.device)
    r = {}
    t = _time_call(lambda: wt.wt_build_tree(l, m, fl, w.ra0, w.dec0, w.J), stream, flush)
    r["build_tree_ms"] = t * 1e3
    for name, mode, which, out in [("wavelet_fp64_eq17", wt.WT_FP64, wt.WT_SUM_EQ17, out64),
                                   ("wavelet_mixed_eq17", wt.WT_MIXED, wt.WT_SUM_EQ17, out32),
                                   ("wavelet_fp64_eq17_regrouped", wt.WT_FP64, wt.WT_SUM_EQ17_REGROUPED, out64),
                                   ("wavelet_fp64_df_eq17_regrouped", wt.WT_FP64_DF, wt.WT_SUM_EQ17_REGROUPED,
                                    out64),
                                   ("wavelet_mixed_eq17_regrouped", wt.WT_MIXED, wt.WT_SUM_EQ17_REGROUPED, out32),
                                   ("wavelet_fp64_eq16", wt.WT_FP64, wt.WT_SUM_EQ16, out64),
                                   ("wavelet_mixed_eq16", wt.WT_MIXED, wt.WT_SUM_EQ16, out32),
                                   ("wavelet_mixed_fast_eq17", wt.WT_MIXED_FAST, wt.WT_SUM_EQ17, out32),
                                   ("wavelet_mixed_fast_eq17_regrouped", wt.WT_MIXED_FAST, wt.WT_SUM_EQ17_REGROUPED,
                                    out32),
                                   ("wavelet_mixed_fast_eq16", wt.WT_MIXED_FAST, wt.WT_SUM_EQ16, out32),
                                   ("wavelet_mixed_tc_eq16", wt.WT_MIXED_TC, wt.WT_SUM_EQ16, out32)]:
        t = _time_call(lambda: wt.wt_predict_vis(tree, uvw, mode=mode, which=which, out=out), stream, flush)
        r[name + "_vis_per_s"] = n / t
    t = _time_call(lambda: wt.dft_predict_vis(l, m, fl, uvw, mode=wt.WT_FP64, out=out64), stream, flush, reps=1)
    r["dft_fp64_vis_per_s"] = n / t
    t = _time_call(lambda: wt.dft_predict_vis(l, m, fl, uvw, mode=wt.WT_FP64_DF, out=out64), stream, flush)
    r["dft_fp64_df_vis_per_s"] = n / t
    t = _time_call(lambda: wt.dft_predict_vis(l, m, fl, uvw, mode=wt.WT_MIXED, out=out32), stream, flush)
    r["dft_mixed_vis_per_s"] = n / t
    t = _time_call(lambda: wt.dft_predict_vis(l, m, fl, uvw, mode=wt.WT_MIXED_FAST, out=out32), stream, flush)
    r["dft_mixed_fast_vis_per_s"] = n / t
    # the phase contraction on the tensor cores; its error against the
    # double-float form still in out64 (float64-class, ~1e-13)
    t = _time_call(lambda: wt.dft_predict_vis(l, m, fl, uvw, mode=wt.WT_MIXED_TC, out=out32), stream, flush)
    r["dft_mixed_tc_vis_per_s"] = n / t
    r["dft_mixed_tc_max_rel_err_vs_df"] = float((out32.to(torch.complex128) - out64).abs().max()) / float(fl.abs().sum())
    r["dft_terms"] = w.n_comp
    t = _time_call(lambda: wt.subtract_model(out32, out32, mode=wt.WT_MIXED, out=out32), stream, flush)
    r["subtract_c64_GBps"] = 24 * n / t / 1e9
    # the subtraction at a size where HBM, not the launch, sets the time:
    # 64 Mi complex64 visibilities, 1.5 GiB moved per call (two reads, one write)
    big = 64 * 1024 * 1024
    a = torch.zeros(big, dtype=torch.complex64, device=uvw.device)
    b = torch.zeros_like(a)
    t = _time_call(lambda: wt.subtract_model(a, b, mode=wt.WT_MIXED, out=a), stream, flush)
    r["subtract_c64_64Mi_GBps"] = 24 * big / t / 1e9
    r["subtract_c64_64Mi_frac_of_hbm"] = 24 * big / t / 1e9 / HBM_PEAK_GBPS
    del a, b
    # the learned response's inference alone, one sample per visibility, on
    # 16 copies of the batch (16 M samples, the learned workload's size: a
    # single medium batch is a 60 us launch, dominated by its ramp)
    mlp = wt.Mlp(w.J, w.ra0, w.dec0, depth=3, x_max=1e30, seed=1)
    uvw16 = uvw.repeat(16, 1)
    r_out = torch.empty(uvw16.shape[0], dtype=torch.complex64, device=uvw.device)
    t_mlp = _time_call(lambda: mlp.eval(uvw16, out=r_out), stream, flush)
    t_mlp1 = _time_call(lambda: mlp.eval(uvw, out=out32), stream, flush)
    mlp.close()
    n_mlp = uvw16.shape[0]
    del uvw16, r_out
    r["mlp_eval_samples_per_s"] = n_mlp / t_mlp
    r["mlp_eval_samples"] = n_mlp
    r["mlp_eval_1M_samples_per_s"] = n / t_mlp1
    # rooflines of the side kernels: the algorithmic work per unit (see the
    # constants) against the measured pipe peaks, and each form's own
    # operation count as pipe_busy
    nc = w.n_comp

    def dft_roof(rate, ops_per_term, fp64=False):
        terms = rate * nc
        if fp64:
            return {"bound": "fp64", "frac": terms * ALG_FLOPS_DFT_TERM / 1e12 / peaks["fp64_tflops"],
                    "unit": "algorithmic float64 flops (11 per term) of the measured FP64 peak",
                    "pipe_busy": {"frac": terms * ops_per_term / peaks["fp64_inst_per_s"],
                                  "ops_per_term": ops_per_term,
                                  "unit": "the form's FP64-pipe instructions per term, of the measured rate"}}
        return {"bound": "alu", "frac": terms * ALG_FLOPS_DFT_TERM / 1e12 / peaks["fp32_tflops"],
                "unit": "algorithmic float32 flops (11 per term) of the measured FP32 peak",
                "sfu_frac": terms * 2 / 1e12 / peaks["sfu_top_s"],
                "pipe_busy": {"frac": terms * ops_per_term / 1e12 / peaks["fp32_top_s"], "ops_per_term": ops_per_term,
                              "unit": "the form's float32 FMA-pipe element ops per term, of the measured rate"}}

    mlp_tflops = n_mlp * 8832 / t_mlp / 1e12
    roof = {
        "dft_mixed_fast": dft_roof(r["dft_mixed_fast_vis_per_s"], OPS_DFT_FAST),
        "dft_mixed_tc": {"bound": "sfu",
                         "frac": r["dft_mixed_tc_vis_per_s"] * nc * 2 / 1e12 / peaks["sfu_top_s"],
                         "unit": "sin and cos of every term of the measured SFU rate (the phase is on the tensor "
                                 "cores)",
                         "alg_fp32_frac": r["dft_mixed_tc_vis_per_s"] * nc * ALG_FLOPS_DFT_TERM / 1e12
                         / peaks["fp32_tflops"],
                         "pipe_busy": {"frac": r["dft_mixed_tc_vis_per_s"] * nc * OPS_DFT_TC / 1e12
                                       / peaks["fp32_top_s"], "ops_per_term": OPS_DFT_TC,
                                       "unit": "the form's float32 FMA-pipe element ops per term, of the measured "
                                               "rate"},
                         "tensor": {"achieved_tflops": r["dft_mixed_tc_vis_per_s"] * nc * TC_FLOPS_DFT_TERM / 1e12,
                                    "flops_per_term": TC_FLOPS_DFT_TERM,
                                    "frac_of_bf16_peak": r["dft_mixed_tc_vis_per_s"] * nc * TC_FLOPS_DFT_TERM / 1e12
                                    / BF16_PEAK_TFLOPS}},
        "dft_mixed": dft_roof(r["dft_mixed_vis_per_s"], OPS_DFT),
        "dft_fp64": dft_roof(r["dft_fp64_vis_per_s"], OPS_DFT_FP64, fp64=True),
        "dft_fp64_df": dft_roof(r["dft_fp64_df_vis_per_s"], OPS_DFT_DF),
        "wavelet_fp64_df": {"bound": "alu",
                            "pipe_busy": {"frac": r["wavelet_fp64_df_eq17_regrouped_vis_per_s"]
                                          * (OPS_DF_LEAF * n_leaves + OPS_DF_NODE * n_int) / 1e12
                                          / peaks["fp32_top_s"],
                                          "ops_per_leaf": OPS_DF_LEAF, "ops_per_internal_node": OPS_DF_NODE}},
        "subtract_c64_64Mi": {"bound": "hbm", "frac": r["subtract_c64_64Mi_frac_of_hbm"],
                              "peak_gbps": HBM_PEAK_GBPS, "peak_source": PEAKS_SOURCE},
        "mlp_eval": {"bound": "sfu",
                     "frac": n_mlp * MLP_TANH_PER_SAMPLE / t_mlp / 1e12 / peaks["sfu_tanh_top_s"],
                     "unit": "hardware tanh of the two SiLU layers (%d per sample) of the measured tanh rate"
                             % MLP_TANH_PER_SAMPLE,
                     "of_sine_rate": n_mlp * MLP_TANH_PER_SAMPLE / t_mlp / 1e12 / peaks["sfu_top_s"],
                     "samples": n_mlp,
                     "tensor": {"achieved_tflops": mlp_tflops, "frac": mlp_tflops / BF16_PEAK_TFLOPS,
                                "peak_tflops": BF16_PEAK_TFLOPS, "peak_source": PEAKS_SOURCE,
                                "flops_per_sample": 8832}},
        "peak_source": peaks["peak_source"],
    }
    return {"forms": r, "side_rooflines": roof}


def batched_measurement(wt, torch, dev, stream, flush, peaks):
    """Config B: 128 antennas, 64 channels over 1.0-1.8 GHz, per-channel
    component lists of log-uniform size 100..20 000 and J in 10..13; one
    graph-captured launch against 64 single-channel launches."""
    import oracle as O
    w = synth.batched()
    chans = w.extra["channels"]
    uvw_m = torch.as_tensor(w.extra["uvw_m"], device=dev)
    n = uvw_m.shape[0]
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    trees = [wt.wt_build_tree(d(c["l"]), d(c["m"]), d(c["flux"]), w.ra0, w.dec0, c["J"]) for c in chans]
    freqs = [c["freq"] for c in chans]
    out = torch.empty((len(chans), n), dtype=torch.complex64, device=dev)
    wt.wt_predict_vis_batched(trees, freqs, uvw_m, mode=wt.WT_MIXED_FAST, out=out)   # plan: tune + capture
    torch.cuda.synchronize()
    t_b = _time_call(lambda: wt.wt_predict_vis_batched(trees, freqs, uvw_m, mode=wt.WT_MIXED_FAST, out=out),
                     stream, flush, reps=3)
    # accuracy on a strided sample of every channel
    idx = np.arange(0, n, n // 64)
    got = out.cpu().numpy()[:, idx]
    err = 0.0
    for c, ch in enumerate(chans):
        t = O.Tree(ch["l"], ch["m"], ch["flux"], w.ra0, w.dec0, ch["J"])
        ref = t.vis_eq17(w.extra["uvw_m"][idx] * (ch["freq"] / synth.C_LIGHT))
        err = max(err, float(np.max(np.abs(got[c] - ref)) / np.abs(ch["flux"]).sum()))
    # the same work as 64 single-channel launches (baselines pre-scaled)
    uvws = [uvw_m * (f / synth.C_LIGHT) for f in freqs]
    outs = [out[c] for c in range(len(chans))]

    def per_channel():
        for c in range(len(chans)):
            wt.wt_predict_vis(trees[c], uvws[c], mode=wt.WT_MIXED_FAST, which=wt.WT_SUM_EQ17_REGROUPED,
                              out=outs[c])
    per_channel()
    t_p = _time_call(per_channel, stream, flush, reps=3)
    sizes = [t.info() for t in trees]
    for t in trees:
        t.close()
    total_vis = n * len(chans)
    # FMA-pipe element ops of the graph launch, per channel's tree (fast regrouped counts)
    op_leaf, op_node, op_low = OPS[("fast", "regrouped")]
    ops, alg = 0, 0
    for x in sizes:
        low = int(x["per_level"][x["J"] - 2]) if x["J"] >= 3 else 0
        ops += n * (op_leaf * x["n_leaves"] + op_node * (x["n_nodes"] - x["n_leaves"] - low) + op_low * low)
        alg += n * (ALG_FLOPS_PHASE_PER_LEAF * x["n_leaves"] + ALG_FLOPS_PER_NODE * x["n_nodes"])
    return {"workload": w.name, "n_ch": len(chans), "n_vis_per_ch": n,
            "n_comp_range": [min(len(c["l"]) for c in chans), max(len(c["l"]) for c in chans)],
            "J_range": [min(c["J"] for c in chans), max(c["J"] for c in chans)],
            "nodes_range": [min(x["n_nodes"] for x in sizes), max(x["n_nodes"] for x in sizes)],
            "graph_launch_vis_per_s": total_vis / t_b, "per_channel_launches_vis_per_s": total_vis / t_p,
            "graph_launch_ms": t_b * 1e3, "per_channel_ms": t_p * 1e3, "max_rel_err_vs_fp64_oracle": err,
            "graph_launch_roofline": {"bound": "alu", "achieved": alg / t_b / 1e12, "peak": peaks["fp32_tflops"],
                                      "unit": "TFLOP/s (algorithmic: 7 per (vis, leaf) + 40 per (vis, node))",
                                      "frac": alg / t_b / 1e12 / peaks["fp32_tflops"],
                                      "pipe_busy": {"frac": ops / t_b / 1e12 / peaks["fp32_top_s"],
                                                    "unit": "float32 FMA-pipe element ops of the form"},
                                      "peak_source": peaks["peak_source"]},
            "form": "WT_MIXED_FAST Eq. 17 regrouped (both legs)"}


def major_cycle_measurement(wt, torch, dev, stream, flush, n=2048, minor_iter=1000, n_major=3, gain=0.1):
    """The major cycle closed on the GPU (Sec. 2.2): the medium array's
    visibilities of the medium sky (5 000 components in 20 blobs), imaged on
    an n x n grid with pixels of 0.45 / max |u| (every baseline inside the
    grid), n_major Cotton-Schwab cycles of minor_iter Hogbom iterations with
    the tree prediction (regrouped Eq. 17, fast form, J from the Table 1
    rule for the pixel size). Timed: the whole clean, and its parts alone
    (dirty image, minor cycle, tree build + prediction + subtraction)."""
    w = synth.medium()
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    uvw = d(w.uvw)
    dl = 0.45 / float(np.max(np.abs(w.uvw[:, :2])))
    J = wt.wt_recommended_J(dl)
    obs = wt.dft_predict_vis(d(w.l), d(w.m), d(w.flux), uvw, mode=wt.WT_MIXED)
    torch.cuda.synchronize()
    wt.wt_clean(uvw, obs, n, dl, w.ra0, w.dec0, J, mode=wt.WT_MIXED_FAST, gain=gain, minor_iter=minor_iter,
                n_major=n_major)                                    # warm-up: FFT plan, shapes tuned per tree size
    res = {}
    t_clean = _time_call(lambda: res.update(out=wt.wt_clean(uvw, obs, n, dl, w.ra0, w.dec0, J, mode=wt.WT_MIXED_FAST,
                                                            gain=gain, minor_iter=minor_iter, n_major=n_major)),
                         stream, flush, reps=1)
    pix, flux, resid, img = res["out"]
    # the parts alone
    beam = wt.wt_dirty_image(uvw, None, n, dl)
    dirty = torch.empty((n, n), dtype=torch.float32, device=dev)
    t_dirty = _time_call(lambda: wt.wt_dirty_image(uvw, obs, n, dl, out=dirty), stream, flush)
    work = dirty.clone()
    t_minor = _time_call(lambda: (work.copy_(dirty), wt.wt_hogbom(work, beam, gain, minor_iter)), stream, flush,
                         reps=1)
    l = d((pix.cpu().numpy() % n - n // 2) * dl)
    m = d((pix.cpu().numpy() // n - n // 2) * dl)
    f = flux.double()
    model = torch.empty_like(obs)

    def predict():
        t = wt.wt_build_tree(l, m, f, w.ra0, w.dec0, J)
        wt.wt_predict_vis(t, uvw, mode=wt.WT_MIXED_FAST, which=wt.WT_SUM_EQ17_REGROUPED, out=model)
        wt.subtract_model(obs, model, mode=wt.WT_MIXED_FAST, out=model)
        t.close()
    t_pred = _time_call(predict, stream, flush)
    rms0 = float(torch.sqrt(torch.mean(torch.abs(obs) ** 2)))
    rms1 = float(torch.sqrt(torch.mean(torch.abs(resid) ** 2)))
    nn = n * n
    out = {"workload": "medium_64ant_1008000vis_5000comp", "image": [n, n], "pixel_rad": dl, "J": J,
           "gain": gain, "minor_iter": minor_iter, "n_major": n_major, "components": int(pix.numel()),
           "clean_ms": t_clean * 1e3, "dirty_image_ms": t_dirty * 1e3, "minor_cycle_ms": t_minor * 1e3,
           "minor_iteration_us": t_minor / minor_iter * 1e6,
           # per Hogbom iteration the kernel reads and writes the image and reads the beam: 12 B per pixel
           "minor_iteration_GBps": 12 * nn / (t_minor / minor_iter) / 1e9,
           "predict_subtract_ms": t_pred * 1e3, "residual_rms_over_data_rms": rms1 / rms0,
           "total_component_flux": float(flux.sum()), "true_flux": float(np.sum(w.flux)),
           "note": "5 000 components in 20 extended blobs: 3 000 Hogbom iterations take a fraction of the flux"}
    out["point_sources"] = major_cycle_points(wt, torch, dev, stream, flush, w, uvw, n, dl, J, gain)
    # a wider spread, where the w term matters, imaged without it and with
    # w-projection (64 planes)
    out["point_sources_400px"] = major_cycle_points(wt, torch, dev, stream, flush, w, uvw, n, dl, J, gain, half=400)
    out["point_sources_400px_wproj"] = major_cycle_points(wt, torch, dev, stream, flush, w, uvw, n, dl, J, gain,
                                                          half=400, w_planes=64)
    return out


def major_cycle_points(wt, torch, dev, stream, flush, w, uvw, n, dl, J, gain, n_src=100, minor_iter=1500,
                       n_major=5, half=100, threshold=0.02, w_planes=0):
    """The same major cycle on a sky Hogbom can take apart: n_src point
    sources at pixel centres within `half` pixels of the phase centre,
    fluxes log-uniform in [0.1, 1] (seeded), observed through the medium
    array (direct sum, mixed form), cleaned down to `threshold`. Reported:
    the flux recovered (all of it, and the part on the true pixels) and the
    residual visibilities' rms against the data's, after 1, 3 and n_major
    major cycles."""
    rng = np.random.default_rng(1916)
    ix = rng.integers(-half, half + 1, n_src)
    iy = rng.integers(-half, half + 1, n_src)
    l = ix * dl
    m = iy * dl
    f = 10.0 ** rng.uniform(-1.0, 0.0, n_src)
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    obs = wt.dft_predict_vis(d(l), d(m), d(f), uvw, mode=wt.WT_MIXED)
    rms0 = float(torch.sqrt(torch.mean(torch.abs(obs) ** 2)))
    true_pix = (iy + n // 2) * n + (ix + n // 2)
    per = []
    for k in sorted({1, 3, n_major}):
        pix, flux, resid, img = wt.wt_clean(uvw, obs, n, dl, w.ra0, w.dec0, J, mode=wt.WT_MIXED_FAST, gain=gain,
                                            threshold=threshold, minor_iter=minor_iter, n_major=k,
                                            w_planes=w_planes)
        torch.cuda.synchronize()
        fl = flux.double().cpu().numpy()
        on = np.isin(pix.cpu().numpy(), true_pix)
        per.append({"n_major": k, "components": int(len(fl)), "flux_recovered_frac": float(fl.sum() / f.sum()),
                    "flux_on_true_pixels_frac": float(fl[on].sum() / f.sum()),
                    "residual_rms_over_data_rms": float(torch.sqrt(torch.mean(torch.abs(resid) ** 2))) / rms0})
    t_clean = _time_call(lambda: wt.wt_clean(uvw, obs, n, dl, w.ra0, w.dec0, J, mode=wt.WT_MIXED_FAST, gain=gain,
                                             threshold=threshold, minor_iter=minor_iter, n_major=n_major,
                                             w_planes=w_planes), stream, flush, reps=1)
    return {"sources": n_src, "half_width_pixels": half, "true_flux": float(f.sum()), "minor_iter": minor_iter,
            "threshold": threshold, "n_major": n_major, "imaging": "w-projection, %d planes" % w_planes
            if w_planes else "nearest cell, no w term", "clean_ms": t_clean * 1e3, "by_major_cycle": per}


def mixed_measurement(wt, torch, dev, stream, flush):
    """Config X: 128 antennas, 2 032 000 visibilities per channel at 1.3 and
    1.5 GHz, 20 000 clustered components, J = 12; the mixed form against the
    FP64 oracle, for the wavelet route and the direct sum."""
    import oracle as O
    w = synth.mixed()
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    l, m, f = d(w.l), d(w.m), d(w.flux)
    S = float(np.abs(w.flux).sum())
    out = {"workload": w.name, "n_vis_per_ch": int(w.extra["uvw_m"].shape[0]), "n_comp": w.n_comp, "J": w.J}
    tree = wt.wt_build_tree(l, m, f, w.ra0, w.dec0, w.J)
    info = tree.info()
    out["n_leaves"], out["n_nodes"] = info["n_leaves"], info["n_nodes"]
    rg = wt.WT_SUM_EQ17_REGROUPED
    forms = [("wavelet_mixed", wt.WT_MIXED, wt.WT_SUM_EQ17), ("wavelet_mixed_regrouped", wt.WT_MIXED, rg),
             ("wavelet_mixed_fast_regrouped", wt.WT_MIXED_FAST, rg)]
    errs = {n: [] for n, _, _ in forms}
    tws = {n: 0.0 for n, _, _ in forms}
    errs_d, td = [], 0.0
    errs_tc, ttc = [], 0.0
    ot = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, w.J)
    for fr in w.extra["freqs"]:
        uvw_np = w.extra["uvw_m"] * (fr / synth.C_LIGHT)
        uvw = d(uvw_np)
        vw = torch.empty(uvw.shape[0], dtype=torch.complex64, device=dev)
        vd = torch.empty_like(vw)
        idx = np.arange(0, uvw_np.shape[0], uvw_np.shape[0] // 400)
        ref = ot.vis_eq17(uvw_np[idx])
        for name, mode, which in forms:
            wt.wt_predict_vis(tree, uvw, mode=mode, which=which, out=vw)
            tws[name] += _time_call(lambda: wt.wt_predict_vis(tree, uvw, mode=mode, which=which, out=vw), stream,
                                    flush)
            errs[name].append(float(np.max(np.abs(vw.cpu().numpy()[idx] - ref)) / S))
        wt.dft_predict_vis(l, m, f, uvw, mode=wt.WT_MIXED, out=vd)
        td += _time_call(lambda: wt.dft_predict_vis(l, m, f, uvw, mode=wt.WT_MIXED, out=vd), stream, flush, reps=1)
        ref_d = O.dft(w.l, w.m, w.flux, uvw_np[idx])
        errs_d.append(float(np.max(np.abs(vd.cpu().numpy()[idx] - ref_d)) / S))
        # the direct sum with its phases on the tensor cores
        wt.dft_predict_vis(l, m, f, uvw, mode=wt.WT_MIXED_TC, out=vd)
        ttc += _time_call(lambda: wt.dft_predict_vis(l, m, f, uvw, mode=wt.WT_MIXED_TC, out=vd), stream, flush)
        errs_tc.append(float(np.max(np.abs(vd.cpu().numpy()[idx] - ref_d)) / S))
    n_tot = 2 * out["n_vis_per_ch"]
    tree.close()
    for name, _, _ in forms:
        out[name + "_vis_per_s"] = n_tot / tws[name]
        out[name + "_max_rel_err"] = max(errs[name])
    out.update({"dft_mixed_vis_per_s": n_tot / td, "dft_mixed_vis_terms_per_s": n_tot * w.n_comp / td,
                "dft_max_rel_err": max(errs_d), "dft_mixed_tc_vis_per_s": n_tot / ttc,
                "dft_mixed_tc_vis_terms_per_s": n_tot * w.n_comp / ttc, "dft_mixed_tc_max_rel_err": max(errs_tc)})
    return out


def learned_measurement(wt, torch, dev, stream, flush, n_train=10_000_000, depth=4, levels=(11, 10)):
    """The learned response where it saves work: the large workload's tree
    (J = 12) truncated at a coarser level j_t, its level-j_t nodes standing
    for their pixels with a full-pixel response, against the same truncation
    centre-snapped (the method without the network) and against the full
    tree at J. Per truncation level the network MLP_jt is trained on n_train
    responses the oracle generates (baselines drawn from the array, +-B).
    Every form is timed on all visibilities and judged on a strided sample
    against the true visibilities (Eq. 12 at the true positions); the
    learned form also against its exact-response counterpart."""
    import oracle as O
    w = synth.learned()
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    J = w.J
    uvw = d(w.uvw)
    l, m, f = d(w.l), d(w.m), d(w.flux)
    tree = wt.wt_build_tree(l, m, f, w.ra0, w.dec0, J)
    info = tree.info()
    out = torch.empty(w.n_vis, dtype=torch.complex64, device=dev)
    S = float(np.abs(w.flux).sum())
    sidx = strided(w.n_vis, 600)
    su = w.uvw[sidx]
    v_true = O.dft(w.l, w.m, w.flux, su, threads=host_cores())
    rms = lambda a, b: float(np.sqrt(np.mean(np.abs(a - b) ** 2)) / S)

    def timed(fn):
        fn()
        t = _time_call(fn, stream, flush)
        return w.n_vis / t, out.cpu().numpy()[sidx]

    res = {"workload": w.name, "J": J, "n_vis": w.n_vis, "n_comp": w.n_comp, "n_leaves": info["n_leaves"],
           "n_nodes": info["n_nodes"], "depth": depth, "train_samples": n_train,
           "error": "RMS |V - V_true| / sum |C| over %d strided baselines; V_true = Eq. 12 at the true positions"
                    % len(sidx)}
    rate, v = timed(lambda: wt.wt_predict_vis(tree, uvw, mode=wt.WT_MIXED_FAST, which=wt.WT_SUM_EQ17_REGROUPED,
                                              out=out))
    res["full_J"] = {"form": "Eq. 17 regrouped, WT_MIXED_FAST, %d leaves" % info["n_leaves"], "vis_per_s": rate,
                     "terms_per_vis": info["n_leaves"], "rms_err_vs_true": rms(v, v_true)}
    rng = np.random.default_rng(21)
    for jt in levels:
        n_jt = int(info["per_level"][jt - 1])
        t0 = time.perf_counter()
        idx = rng.integers(0, w.n_vis, n_train)
        tr_uvw = w.uvw[idx] * np.where(rng.random((n_train, 1)) < 0.5, -1.0, 1.0)
        tgt = O.pixel_response(jt, depth, w.ra0, w.dec0, tr_uvw)
        t_gen = time.perf_counter() - t0
        x_max = float(np.max(np.abs(tr_uvw * O.level_pixel_size(jt)))) * 1.0001
        mlp = wt.Mlp(jt, w.ra0, w.dec0, depth=depth, x_max=x_max, seed=5)
        tu = d(tr_uvw)
        tt = d(np.stack([tgt.real, tgt.imag], axis=1).astype(np.float32))
        del tr_uvw, tgt
        steps = MLP_TRAIN_EPOCHS * (n_train // 8192)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        loss = mlp.train(tu, tt, steps=steps, batch=8192, lr=3e-3)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        del tu, tt
        r_net = mlp.eval(d(su)).cpu().numpy()
        r_ex = O.pixel_response(jt, depth, w.ra0, w.dec0, su)
        rate_l, v_l = timed(lambda: wt.wt_predict_vis_truncated(tree, jt, uvw, response=wt.WT_RESPONSE_LEARNED,
                                                                mlp=mlp, out=out))
        rate_s, v_s = timed(lambda: wt.wt_predict_vis_truncated(tree, jt, uvw, out=out))
        rate_e, v_e = timed(lambda: wt.wt_predict_vis_truncated(tree, jt, uvw, response=wt.WT_RESPONSE_EXACT,
                                                                depth=depth, out=out))
        res["truncated_level_%d" % jt] = {
            "terms_per_vis": n_jt, "x_max": x_max, "oracle_target_gen_s": t_gen, "train_s": t_train,
            "train_steps": steps, "final_minibatch_loss": loss,
            "response_rms_err_vs_exact": float(np.sqrt(np.mean(np.abs(r_net - r_ex) ** 2))),
            "learned": {"vis_per_s": rate_l, "rms_err_vs_true": rms(v_l, v_true),
                        "max_rel_err_vs_exact_response_form": float(np.max(np.abs(v_l - v_e)) / S)},
            "centre_snapped": {"vis_per_s": rate_s, "rms_err_vs_true": rms(v_s, v_true)},
            "exact_response": {"vis_per_s": rate_e, "rms_err_vs_true": rms(v_e, v_true),
                               "note": "float64 response by %d sub-pixels per visibility (the yardstick)"
                                       % (4 ** depth)},
        }
        mlp.close()
    # hard thresholding with full-pixel responses: the tree truncated at j0
    # plus the detail coefficients of levels j0 .. J-1 with |gamma| >= tau;
    # the responses exact (float64 quadrature), learned (one network per
    # level j0 .. J for its level's responses down to the common finest level
    # j0 + d0, trained on n_train oracle responses each) or none
    d0 = depth + 1
    ex = tree.export()
    offs, gam = ex["level_offsets"], ex["gamma"]
    for j0 in (9, 11):
        nets, errs, t_gen, t_train = [], [], 0.0, 0.0
        for L in range(j0, J + 1):
            dL = d0 - (L - j0)
            t0 = time.perf_counter()
            idx = rng.integers(0, w.n_vis, n_train)
            tr_uvw = w.uvw[idx] * np.where(rng.random((n_train, 1)) < 0.5, -1.0, 1.0)
            tgt = O.pixel_response(L, dL, w.ra0, w.dec0, tr_uvw)
            t_gen += time.perf_counter() - t0
            x_max = float(np.max(np.abs(tr_uvw * O.level_pixel_size(L)))) * 1.0001
            mlp = wt.Mlp(L, w.ra0, w.dec0, depth=dL, x_max=x_max, seed=7 + L)
            tu, tt = d(tr_uvw), d(np.stack([tgt.real, tgt.imag], axis=1).astype(np.float32))
            del tr_uvw, tgt
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            mlp.train(tu, tt, steps=MLP_TRAIN_EPOCHS * (n_train // 8192), batch=8192, lr=3e-3)
            torch.cuda.synchronize()
            t_train += time.perf_counter() - t0
            del tu, tt
            r_net = mlp.eval(d(su)).cpu().numpy()
            errs.append(float(np.sqrt(np.mean(np.abs(r_net - O.pixel_response(L, dL, w.ra0, w.dec0, su)) ** 2))))
            nets.append(mlp)
        g_fine = np.abs(gam[offs[j0 - 1]:offs[J - 1]]).ravel()
        for frac in (0.1, 0.5):
            tau = float(np.quantile(g_fine, 1.0 - frac))
            kept_nodes = int(np.sum(np.any(np.abs(gam[offs[j0 - 1]:offs[J - 1]]) >= tau, axis=1)))
            terms = int(info["per_level"][j0 - 1]) + 4 * kept_nodes
            rate_x, v_x = timed(lambda: wt.wt_predict_vis_thresholded(tree, j0, tau, uvw,
                                                                      response=wt.WT_RESPONSE_EXACT, depth=d0,
                                                                      out=out))
            rate_s, v_s = timed(lambda: wt.wt_predict_vis_thresholded(tree, j0, tau, uvw, out=out))
            rate_l, v_l = timed(lambda: wt.wt_predict_vis_thresholded(tree, j0, tau, uvw,
                                                                      response=wt.WT_RESPONSE_LEARNED, mlps=nets,
                                                                      out=out))
            res["thresholded_j0_%d_keep_%d_percent" % (j0, round(100 * frac))] = {
                "tau": tau, "kept_coefficients": int(np.sum(g_fine >= tau)), "terms_per_vis": terms,
                "exact_response": {"vis_per_s": rate_x, "rms_err_vs_true": rms(v_x, v_true),
                                   "note": "float64 responses, %d .. %d sub-pixels per level"
                                           % (4 ** (d0 - (J - j0)), 4 ** d0)},
                "learned": {"vis_per_s": rate_l, "rms_err_vs_true": rms(v_l, v_true),
                            "max_rel_err_vs_exact_response_form": float(np.max(np.abs(v_l - v_x)) / S),
                            "response_rms_err_vs_exact_per_level": errs,
                            "networks": "one per level %d .. %d, %d oracle responses each (%.1f s to generate, "
                                        "%.2f s to train all)" % (j0, J, n_train, t_gen, t_train)},
                "centre_snapped": {"vis_per_s": rate_s, "rms_err_vs_true": rms(v_s, v_true)}}
        for mlp in nets:
            mlp.close()
    tree.close()
    return res


# ---------------------------------------------------------------- oracle (CPU)

def host_cores():
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def strided(n, k):
    """A deterministic strided subset of k of n indices (every n // k-th)."""
    return np.arange(0, n, max(1, n // k))[:k]


def _oracle_step(w, J, idx, threads):
    """Seconds of one oracle step on a subset: the tree build (the pointer
    tree of Sec. 3.5), Eq. 17 on the baselines w.uvw[idx] over `threads`
    OpenMP threads, and the subtraction."""
    import oracle as O
    t0 = time.perf_counter()
    tr = O.Tree(w.l, w.m, w.flux, w.ra0, w.dec0, J)
    t1 = time.perf_counter()
    v = tr.vis_eq17(w.uvw[idx], threads=threads)
    O.subtract(v, v)
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1


def cpu_baseline(w, J, budget_s=8.0, min_sample=65536):
    """The oracle as it stands on the host cores, single-threaded and with
    OpenMP over the visibilities on every core, on one strided subset of at
    least min_sample visibilities (about budget_s of single-thread work):
    tree build + Eq. 17 + subtract, the per-visibility rate extrapolated to
    the whole batch."""
    cores = host_cores()
    _, te = _oracle_step(w, J, strided(w.n_vis, 512), 1)
    per_vis = max(te / 512, 1e-9)
    n_s = int(min(w.n_vis, max(min_sample, budget_s / per_vis)))
    idx = strided(w.n_vis, n_s)
    n_s = len(idx)
    tb1, te1 = _oracle_step(w, J, idx, 1)
    tbn, ten = _oracle_step(w, J, idx, cores)
    rate = lambda tb, te: w.n_vis / (tb + te * w.n_vis / n_s)
    return {"value": rate(tbn, ten), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "oracle tree build + Eq. 17 (OpenMP over visibilities, %d threads) + subtract on %d "
                      "strided visibilities of %d, extrapolated to the full batch; %.1f s" % (cores, n_s, w.n_vis,
                                                                                            tbn + ten),
            "single_thread": {"value": rate(tb1, te1), "unit": UNIT, "cores": 1,
                              "sample": "the same subset on one thread; %.1f s" % (tb1 + te1)}}


def reference(args):
    """The CPU oracle on the headline workload: each step is the oracle's
    tree build, Eq. 17 on a strided sample of the batch's visibilities
    (OpenMP over visibilities on every host core) and the subtraction; the
    sample is sized for about 1.5 s per step, and value is the sample's
    visibilities over the step's time."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    J = args.J
    w = synth.large(J=J) if args.workload == "large" else synth.medium(J=J)
    cores = host_cores()
    _, te = _oracle_step(w, J, strided(w.n_vis, 2048), cores)
    per_vis = max(te / 2048, 1e-9)
    n_s = len(strided(w.n_vis, int(min(w.n_vis, max(2048, 1.5 / per_vis)))))
    idx = strided(w.n_vis, n_s)
    for _ in range(args.warmup):
        _oracle_step(w, J, idx[: max(1, n_s // 8)], cores)
    steps = []
    for _ in range(args.steps):
        tb, te = _oracle_step(w, J, idx, cores)
        steps.append(tb + te)
    t = statistics.mean(steps)
    val = n_s / t
    line = {
        "impl": "reference",
        "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n_vis": w.n_vis, "n_comp": w.n_comp, "J": J,
                   "vis_per_step": n_s, "form": "CPU oracle, Eq. 17, f64",
                   "step": "oracle tree build + Eq. 17 on a strided sample of the batch + subtract"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d strided visibilities of %d per step (OpenMP over visibilities, %d threads); "
                                   "not extrapolated: value = sample / step time" % (n_s, w.n_vis, cores)},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def sweep(args):
    """Run-time scaling as in Sec. 3.6.1: per-visibility time of the Eq. 17
    predictor (the bench's fast regrouped form, the explicit mixed form and
    float64) against J on the medium workload and on a fixed
    set of distinct components, against the number of distinct components at
    fixed J, and the paper-context workload (27 antennas, 1 263 600
    visibilities, J = 20, 15 and 140 distinct components) beside the paper's
    own 146 s and 1000 s per major cycle on its unstated CPU."""
    import torch

    import paper_1909_03956_gb300 as wt
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    wt.load()
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)

    # form name -> (mode, sum): the bench's form, the explicit mixed form, float64
    kinds = {"fast_regrouped": (wt.WT_MIXED_FAST, wt.WT_SUM_EQ17_REGROUPED), "mixed": (wt.WT_MIXED, wt.WT_SUM_EQ17),
             "fp64": (wt.WT_FP64, wt.WT_SUM_EQ17)}

    def measure(w, J, forms=("fast_regrouped", "mixed", "fp64")):
        l, m, f, uvw = d(w.l), d(w.m), d(w.flux), d(w.uvw)
        tree = wt.wt_build_tree(l, m, f, w.ra0, w.dec0, J)
        info = tree.info()
        r = {"J": J, "n_leaves": info["n_leaves"], "n_nodes": info["n_nodes"]}
        for name in forms:
            mode, which = kinds[name]
            c64 = mode != wt.WT_FP64
            out = torch.empty(w.n_vis, dtype=torch.complex64 if c64 else torch.complex128, device=dev)
            wt.wt_predict_vis(tree, uvw, mode=mode, which=which, out=out)
            t = _time_call(lambda: wt.wt_predict_vis(tree, uvw, mode=mode, which=which, out=out), stream, flush,
                           reps=3 if c64 else 1)
            r[name + "_ns_per_vis"] = t / w.n_vis * 1e9
        tree.close()
        return r

    res = {"kind": "scaling sweep (Sec. 3.6.1)", "unit": "ns per visibility, one GB300"}
    med = synth.medium()
    res["medium_J_sweep"] = [measure(med, J) for J in range(8, 15)]
    fixed = {}
    for nd in (10, 20, 40, 80, 140):
        w = synth.medium_fixed(nd)
        fixed[str(nd)] = [measure(w, J, forms=("fast_regrouped", "mixed")) for J in (12, 15, 20, 25)]
    res["fixed_distinct_J_sweep"] = fixed
    res["paper_context"] = []
    for nd, paper_s in ((15, 146.0), (140, 1000.0)):
        w = synth.paper_context(n_distinct=nd)
        r = measure(w, 20)
        r.update({"n_vis": w.n_vis, "n_distinct": nd, "paper_s_per_major_cycle": paper_s,
                  "gpu_fp64_s_per_major_cycle": r["fp64_ns_per_vis"] * w.n_vis / 1e9,
                  "gpu_mixed_s_per_major_cycle": r["mixed_ns_per_vis"] * w.n_vis / 1e9,
                  "gpu_fast_regrouped_s_per_major_cycle": r["fast_regrouped_ns_per_vis"] * w.n_vis / 1e9})
        res["paper_context"].append(r)
    print(json.dumps(res), flush=True)


def forms_once(args):
    import torch

    import paper_1909_03956_gb300 as wt
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    wt.load()
    w = synth.large(J=args.J) if args.workload == "large" else synth.medium(J=args.J)
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    l, m, f, uvw = d(w.l), d(w.m), d(w.flux), d(w.uvw)
    tree = wt.wt_build_tree(l, m, f, w.ra0, w.dec0, w.J)
    o64 = torch.empty(w.n_vis, dtype=torch.complex128, device=dev)
    o32 = torch.empty(w.n_vis, dtype=torch.complex64, device=dev)
    sub = uvw[:131072].contiguous()
    runs = [("wavelet_mixed_fast", lambda: wt.wt_predict_vis(tree, uvw, mode=wt.WT_MIXED_FAST, out=o32)),
            ("wavelet_mixed", lambda: wt.wt_predict_vis(tree, uvw, mode=wt.WT_MIXED, out=o32)),
            ("wavelet_fp64", lambda: wt.wt_predict_vis(tree, uvw, mode=wt.WT_FP64, out=o64)),
            ("dft_mixed", lambda: wt.dft_predict_vis(l, m, f, uvw, mode=wt.WT_MIXED, out=o32)),
            ("dft_mixed_tc", lambda: wt.dft_predict_vis(l, m, f, uvw, mode=wt.WT_MIXED_TC, out=o32)),
            ("dft_fp64_131072", lambda: wt.dft_predict_vis(l, m, f, sub, mode=wt.WT_FP64, out=o64[:131072])),
            ("subtract_c64", lambda: wt.subtract_model(o32, o32, mode=wt.WT_MIXED, out=o32))]
    # the learned response's tensor-core inference on every visibility
    mlp = wt.Mlp(w.J, w.ra0, w.dec0, depth=3, x_max=1e30, seed=1)
    r_out = torch.empty(w.n_vis, dtype=torch.complex64, device=dev)
    runs.append(("mlp_eval", lambda: mlp.eval(uvw, out=r_out)))
    uvw16 = uvw.repeat(16, 1)
    r_out16 = torch.empty(uvw16.shape[0], dtype=torch.complex64, device=dev)
    runs.append(("mlp_eval_16x", lambda: mlp.eval(uvw16, out=r_out16)))
    # batched: 8 channels of the medium workload's components at 1.0 .. 1.8 GHz
    freqs = list(np.linspace(1.0e9, 1.8e9, 8))
    btrees = [wt.wt_build_tree(l, m, f, w.ra0, w.dec0, 10 + (c % 4)) for c in range(8)]
    uvw_m = d(w.uvw * (synth.C_LIGHT / 1.4e9))
    b_out = torch.empty((8, w.n_vis), dtype=torch.complex64, device=dev)
    runs.append(("batched_8ch", lambda: wt.wt_predict_vis_batched(btrees, freqs, uvw_m, mode=wt.WT_MIXED_FAST,
                                                                   out=b_out)))
    # the subtraction where HBM sets the time: 64 Mi complex64
    big_a = torch.zeros(64 * 1024 * 1024, dtype=torch.complex64, device=dev)
    big_b = torch.zeros_like(big_a)
    runs.append(("subtract_64Mi", lambda: wt.subtract_model(big_a, big_b, mode=wt.WT_MIXED, out=big_a)))
    runs.append(("build_tree", lambda: wt.wt_build_tree(l, m, f, w.ra0, w.dec0, w.J).close()))
    # the major cycle's imaging at 2048 x 2048 (the bench's major-cycle workload)
    n_img = 2048
    dl_img = 0.45 / float(np.max(np.abs(w.uvw[:, :2])))
    img_obs = torch.zeros(w.n_vis, dtype=torch.complex64, device=dev)
    img_out = torch.empty((n_img, n_img), dtype=torch.float32, device=dev)
    img_beam = torch.empty((n_img, n_img), dtype=torch.float32, device=dev)
    runs.append(("dirty_image_2048", lambda: wt.wt_dirty_image(uvw, img_obs, n_img, dl_img, out=img_out)))
    runs.append(("hogbom_2048_x20", lambda: (wt.wt_dirty_image(uvw, None, n_img, dl_img, out=img_beam),
                                             img_out.copy_(img_beam),
                                             wt.wt_hogbom(img_out, img_beam, 0.1, 20))))
    rg = wt.WT_SUM_EQ17_REGROUPED
    runs.append(("wavelet_mixed_fast_regrouped",
                 lambda: wt.wt_predict_vis(tree, uvw, mode=wt.WT_MIXED_FAST, which=rg, out=o32)))
    runs.append(("wavelet_mixed_regrouped", lambda: wt.wt_predict_vis(tree, uvw, mode=wt.WT_MIXED, which=rg, out=o32)))
    runs.append(("wavelet_fp64_df_regrouped",
                 lambda: wt.wt_predict_vis(tree, uvw, mode=wt.WT_FP64_DF, which=rg, out=o64)))
    if args.only:
        keep = set(args.only.split(","))
        runs = [(n, fn) for n, fn in runs if n in keep]
    for name, fn in runs:
        fn()
        torch.cuda.synchronize()
        fn()
        torch.cuda.synchronize()
    wt.wt_device_status()
    tree.close()
    for t in btrees:
        t.close()
    mlp.close()
    print("forms-once ok: " + ", ".join(n for n, _ in runs), flush=True)


def main():
    args = parse()
    if args.workload is None:
        args.workload = "medium" if args.forms_once else "large"
    if args.forms_once:
        forms_once(args)
        return
    if args.sweep:
        sweep(args)
        return
    if args.impl == "reference":
        reference(args)
    else:
        native(args)


if __name__ == "__main__":
    main()
