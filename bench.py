#!/usr/bin/env python
"""Throughput of the FerroX time step (TDGL update + Poisson solve to a 1e-10
relative residual) on the 256x256x32 MFIM Q-V sweep workload, one JSON line.

A step is one time step of the whole hot path: the fused TDGL update (Eq. TDGL2)
and the variable-permittivity Poisson solve it is coupled to, converged on the
device.  The timed steps are the first steps of the Q-V sweep (-2 V first),
after Step 0 and W warm-up steps.  Inputs are resident in HBM; L2 (129 MB) is
flushed between timed steps by writing a 256 MB buffer, because the working set
of this workload (~100 MB) would otherwise stay in L2 from one step to the next.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision fp64|mixed]

Multi-GPU: the workload is one device stack whose domain is not split, so
N > 1 runs N independent replicas (one per rank, seed + rank); value is the
cells x steps of all ranks over the max-over-ranks time.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mcell-steps/s incl. Poisson to 1e-10 residual; HBM % of peak; vs plain FP64"
UNIT = "Mcell-steps/s"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # SMs x DFMA/clk/SM x flop/FMA x max clock
FP64_PEAK_GINSTR = 152 * 2 * 2.070                 # FP64 pipe instructions per second (G/s)
HBM_FALLBACK_GBS = 6800.0


# ---------------------------------------------------------------------- helpers -------

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(x: float, ws: int) -> float:
    """Max over ranks (identity for one rank)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": HBM_FALLBACK_GBS}, "fallback"


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2210_15668_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(fn.encode() + f.read())
    return h.hexdigest()[:16]


def measured_traffic(precision, kernel):
    """DRAM bytes per launch from an ncu capture of the current source, else None."""
    tpath = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(tpath):
        return None
    tj = json.load(open(tpath))
    if tj.get("source_hash") != source_hash():
        return None
    return tj.get("per_launch_bytes", {}).get(f"{precision}:{kernel}")


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in rows for q in range(4) if r[5 + q].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------- algorithmic work -------

# FP64 pipe instructions per unit of work (the FP64 forms are bound by this pipe)
FAST_INNER = -8  # fast and learned forms: V-cycles per FP64 residual chosen on the device (<= 8)

FP64_INSTR = {"smooth_fine": 7.0, "smooth_coarse": 7.0, "resid": 10.0, "tdgl": 30.0, "restrict": 8.0,
              "prolong": 4.5}
# the direct FP64 form's fine sweeps run on b / diag with couplings divided by the
# diagonal: two additions and four multiply-adds per cell
FP64_INSTR_DIRECT_FINE = 6.0
# algorithmic bytes per unit of FP64 work (the same counts as the library's): a colour
# sweep moves 24 B per updated cell, residual + restriction and prolongation 17 B per
# fine cell
FP64_BYTES_PER_UNIT = {"smooth_fine": 24.0, "smooth_coarse": 24.0, "restrict": 17.0, "prolong": 17.0}


def kernel_work(kind, cells, fe_cells, dyn_cells, tsz):
    """Algorithmic (bytes, flops) of ONE launch of a kernel class on the fine level.

    Minimum traffic the method needs per launch (each array element read or
    written once), and arithmetic with an FMA counted as two flops."""
    if kind == "smooth_fine":      # one colour: read the other colour's e, own r; write own e
        return 0.5 * cells * 3 * tsz, 0.5 * cells * 11
    if kind == "resid":            # read phi, b (dynamic planes), write r (T)
        return cells * (8 + tsz) + dyn_cells * 8, cells * 19
    if kind == "tdgl":             # read P, phi; write new P; write b on dynamic planes
        return fe_cells * 24 + dyn_cells * 8, fe_cells * 45
    if kind == "restrict":         # read e, r of the fine level, write r of the coarse level
        return cells * 2 * tsz + cells / 8 * tsz, cells * 15
    if kind == "prolong":          # read coarse e, read+write fine e
        return cells * 2 * tsz + cells / 8 * tsz, cells * 16
    if kind == "update":           # read e, read+write phi
        return cells * (tsz + 16), cells * 1
    if kind == "copy":
        return fe_cells * 16, 0.0
    return None, None


def class_rooflines(prof, hbm_peak, fp64_classes=(), df_classes=()):
    """Per kernel class of one eager, event-timed step: time, launches, algorithmic
    bytes (from the library's own per-launch count), effective GB/s and fraction of
    the measured HBM peak; plus the whole step (sum over classes).  fp64_classes are
    labelled bound by the FP64 pipe, df_classes (the mixed form's double-float outer
    residual) by instruction issue on the FP32 and integer pipes."""
    out = {}
    tb = tm = 0.0
    for k, (ms, n, by) in prof.items():
        if not n:
            continue
        gbs = by / (ms / 1e3) / 1e9 if ms > 0 else None
        out[k] = {"ms": round(ms, 4), "launches": n, "bytes": by,
                  "gbs": gbs, "hbm_frac": gbs / hbm_peak if gbs else None}
        if k in df_classes:
            out[k]["bound"] = "issue (double-float on the FP32 and integer pipes)"
        elif k in fp64_classes:
            out[k]["bound"] = "alu (FP64 pipe)"
        tb += by
        tm += ms
    whole = {"bytes": tb, "eager_ms": tm, "gbs": tb / (tm / 1e3) / 1e9 if tm else None}
    whole["hbm_frac"] = whole["gbs"] / hbm_peak if whole["gbs"] else None
    return out, whole


# -------------------------------------------------------------------- workloads -------

def workload_config(name):
    """The bench workload, or a larger/smaller copy of it used for ncu captures."""
    from paper_2210_15668_gb300 import inputs as I
    cfg = I.mfim_sweep()
    cfg["label"] = "mfim_256x256x32 Q-V sweep (first steps at -2 V), seed 1"
    if name == "mfim_256x256x32":
        return cfg
    if name in ("mfism_256x256x64", "mfism_512x512x128"):
        m = I.mfism_mixed() if name == "mfism_256x256x64" else I.mfism_large()
        m["sweep"] = [m["v_top"]]
        m["steps_per_point"] = 10 ** 9
        m["label"] = (f"{name} MFISM (p-Si N_A 1e24, n_i 1e16, 300 K; damped Newton), "
                      f"seed {m['seed']}, 0 V")
        return m
    if name.startswith("mfim_"):
        nx, ny, nz = (int(v) for v in name[5:].split("x"))
        cfg["geom"] = I.make_geometry(nx, ny, I.mfim_stack(nz))
        cfg["label"] = f"{name} MFIM (same stack recipe), seed 1, -2 V"
        return cfg
    raise SystemExit(f"unknown workload {name}")


# ------------------------------------------------------------------------ ours -------

def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    from paper_2210_15668_gb300 import ferrox, inputs as I

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    cfg = workload_config(args.workload)
    geom = cfg["geom"]
    nz = I.nz_of(geom)
    cells = geom["nx"] * geom["ny"] * nz
    fe_mask = I.fe_plane_mask(geom)
    fe_cells = int(fe_mask.sum()) * geom["nx"] * geom["ny"]
    dyn = fe_mask | np.roll(fe_mask, 1) | np.roll(fe_mask, -1)
    dyn_cells = int(dyn.sum()) * geom["nx"] * geom["ny"]
    P0 = I.random_polarization(geom, cfg["seed"] + rank)
    sweep, per_point = cfg["sweep"], cfg["steps_per_point"]

    def make(precision):
        num = ferrox.make_numerics(cfg["dt"], order=1, tol=1e-10, precision=precision, max_cycles=200,
                                   guess=args.guess, nu1=args.nu1, nu2=args.nu2, inner=args.inner)
        d = ferrox.Device(geom, P0, numerics=num)
        d.set_bias(0.0, sweep[0])
        d.solve_poisson()                                  # Step 0 (untimed)
        return d

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def timed_run(d, K, W, clocks=None):
        stream = d.stream
        point = 0
        for s in range(W):
            flush.zero_()
            d.step(1)
        torch.cuda.synchronize()
        st0 = d.stats()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        barrier(ws)
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        for s in range(K):
            p = (W + s) // per_point
            if p != point and p < len(sweep):
                point = p
                d.set_bias(0.0, sweep[p])
            flush.zero_()
            ev[s][0].record(stream)
            d.step(1)
            ev[s][1].record(stream)
        torch.cuda.synchronize()
        barrier(ws)
        ck = clocks.stop() if clocks else None
        t_ms = sum(a.elapsed_time(b) for a, b in ev)
        st1 = d.stats()
        return t_ms, st0, st1, ck

    prec_main = {"mixed": ferrox.MIXED, "fp64": ferrox.FP64, "fp64_defect": ferrox.FP64_DEFECT}[args.precision]
    dev = make(prec_main)
    learned_main = None
    if args.learned:
        learned_main = train_network_on(args, ferrox, I)
        lv2 = dev.levels()[2]
        dev._net = ferrox.NN(lv2[2], lv2[1], lv2[0], params=learned_main["params"])
        dev.attach_nn(dev._net, 2)
    clocks = ClockSampler(local) if rank == 0 else None
    t_ms, st0, st1, ck = timed_run(dev, args.steps, args.warmup, clocks)
    if learned_main is not None:
        learned_main["corrections_rejected"] = st1["nn_rejected"] - st0["nn_rejected"]
    t_max = reduce_max(t_ms, ws)
    K = args.steps
    value = ws * cells * K / (t_max / 1e3) / 1e6
    cycles_per_step = (st1["cycles"] - st0["cycles"]) / K
    vcycles_per_step = (st1["vcycles"] - st0["vcycles"]) / K
    launches = st1["launches"] - st0["launches"]

    # per-kernel breakdown of one step (eager, event-timed) -> roofline of the dominant kernel
    sp0 = dev.stats()
    prof = dev.profile_step(with_bytes=True)
    sp1 = dev.stats()
    tsz = 4 if prec_main == ferrox.MIXED else 8
    # the dominant kernel: the class that moves the most algorithmic bytes per step
    # (the fine-level sweep).  Event-timed one by one, the small coarse-level launches
    # look as long as the fine sweeps, but inside the step's CUDA graph programmatic
    # launch overlaps them (graph step ~0.6 of the eager sum); every class is reported
    # in roofline["classes"].
    modeled = [k for k in prof if prof[k][1] and prof[k][2] > 0]
    dom = max(modeled, key=lambda k: prof[k][2])
    dom_ms, dom_n, dom_bytes = prof[dom]
    step_ms = sum(v[0] for v in prof.values())
    peaks, peak_src = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", HBM_FALLBACK_GBS))
    by = dom_bytes / max(dom_n, 1)
    _, fl = kernel_work(dom, cells, fe_cells, dyn_cells, tsz)
    avg_s = dom_ms / max(dom_n, 1) / 1e3
    gbs = by / avg_s / 1e9 if by else None
    tfl = fl / avg_s / 1e12 if fl else None
    fp64_kernel = prec_main != ferrox.MIXED or dom in ("resid", "tdgl", "update")
    traffic = measured_traffic(args.precision, dom)
    share = dom_ms / step_ms if step_ms else None
    fp64_classes = (("tdgl", "resid", "update") if prec_main == ferrox.MIXED else
                    ("tdgl", "resid", "update", "smooth_fine", "smooth_coarse", "restrict", "prolong", "tail"))
    classes, whole = class_rooflines(prof, hbm_peak, fp64_classes,
                                     ("resid",) if prec_main == ferrox.MIXED else ())
    whole["graph_ms_per_step"] = t_max / K
    whole["vcycles_profiled_step"] = sp1["vcycles"] - sp0["vcycles"]
    whole["vcycles_per_timed_step"] = vcycles_per_step
    if fp64_kernel:
        if dom in FP64_BYTES_PER_UNIT:
            units = by / FP64_BYTES_PER_UNIT[dom]
        else:
            units = {"resid": cells, "tdgl": fe_cells}.get(dom, cells)
        ipu = FP64_INSTR.get(dom, 0.0)
        if dom == "smooth_fine" and prec_main == ferrox.FP64:
            ipu = FP64_INSTR_DIRECT_FINE
        gi = ipu * units / avg_s / 1e9
        roof = {"bound": "alu", "achieved": gi, "peak": FP64_PEAK_GINSTR, "unit": "G FP64-instr/s",
                "share_of_step": share, "frac": gi / FP64_PEAK_GINSTR, "traffic": traffic,
                "kernel": dom, "peak_source": "derived: 152 SMs x 2 FP64 instr/clk x 2.07 GHz",
                "work": f"{ipu} FP64 instructions per unit",
                "flop_view": {"achieved_tflops": tfl, "peak_tflops": FP64_PEAK_TFLOPS},
                "hbm_view": {"achieved_gbs": gbs, "peak_gbs": hbm_peak, "algorithmic_bytes_per_launch": by,
                             "frac": gbs / hbm_peak if gbs else None, "peak_source": peak_src}}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "share_of_step": share,
                "frac": gbs / hbm_peak if gbs else None, "traffic": traffic, "kernel": dom,
                "algorithmic_bytes_per_launch": by, "peak_source": peak_src}
    roof["classes"] = classes
    roof["whole_step"] = whole
    roof["dominant_by"] = "algorithmic bytes per step"
    breakdown = {k: {"ms": round(v[0], 4), "launches": v[1]} for k, v in prof.items() if v[1]}
    dev.close()

    # the other precision on the same workload ("vs plain FP64")
    other = None
    if not args.no_compare:
        prec_o = ferrox.FP64 if prec_main == ferrox.MIXED else ferrox.MIXED
        d2 = make(prec_o)
        t2, s20, s21, _ = timed_run(d2, K, args.warmup)
        t2 = reduce_max(t2, ws)
        v2 = ws * cells * K / (t2 / 1e3) / 1e6
        prof2 = d2.profile_step(with_bytes=True)
        cl2, wh2 = class_rooflines(prof2, hbm_peak, ("tdgl", "resid", "update"),
                                   ("resid",) if prec_o == ferrox.MIXED else ())
        wh2["graph_ms_per_step"] = t2 / K
        other = {"precision": "fp64" if prec_o == ferrox.FP64 else "mixed", "value": v2,
                 "ms_per_step": t2 / K, "vcycles_per_step": (s21["vcycles"] - s20["vcycles"]) / K,
                 "roofline_classes": cl2, "whole_step": wh2}
        d2.close()
    # the GB300-native fast form: FP32 multigrid in FP64 defect correction, an
    # extrapolated initial guess and FAST_INNER V-cycles per FP64 residual (same
    # residual test)
    fast = None
    if not args.no_compare:
        def make_fast():
            num = ferrox.make_numerics(cfg["dt"], order=1, tol=1e-10, precision=ferrox.MIXED,
                                       max_cycles=200, guess=1, inner=FAST_INNER)
            d = ferrox.Device(geom, P0, numerics=num)
            d.set_bias(0.0, sweep[0])
            d.solve_poisson()
            return d
        d4 = make_fast()
        t4, s40, s41, _ = timed_run(d4, K, args.warmup)
        t4 = reduce_max(t4, ws)
        prof4 = d4.profile_step(with_bytes=True)
        cl4, wh4 = class_rooflines(prof4, hbm_peak, ("tdgl", "resid", "update"), ("resid",))
        wh4["graph_ms_per_step"] = t4 / K
        fast = {"precision": "mixed", "guess": "extrapolated", "inner": FAST_INNER,
                "value": ws * cells * K / (t4 / 1e3) / 1e6, "ms_per_step": t4 / K,
                "vcycles_per_step": (s41["vcycles"] - s40["vcycles"]) / K,
                "outer_iterations_per_step": (s41["cycles"] - s40["cycles"]) / K,
                "roofline_classes": cl4, "whole_step": wh4}
        d4.close()
    learned = None if (args.no_compare or args.no_learned) else run_learned(args, ws, cfg, geom, P0, cells,
                                                                            sweep, timed_run)
    batch = None if args.no_batch else run_batch_qv(args, ws)
    batch64 = None if args.no_batch else run_batch_qv(args, ws, precision=0)
    mfism = None if args.no_mfism else run_mfism(args, ws, hbm_peak)
    mixed_v = value if prec_main == ferrox.MIXED else (other or {}).get("value")
    fp64_v = value if prec_main != ferrox.MIXED else (other or {}).get("value")

    # end to end through the public API with host buffers (pinned), copies inside the region
    e2e = None
    if not args.no_e2e:
        d3 = make(prec_main)
        # the state a step takes and returns: P on the ferroelectric film (zero
        # elsewhere in the model) and phi, in pinned host memory
        lo, hi = d3.fe_planes()
        Ph = torch.empty((1, hi - lo + 1, geom["ny"], geom["nx"]), dtype=torch.float64).pin_memory().numpy()
        fh = torch.empty((nz, geom["ny"], geom["nx"]), dtype=torch.float64).pin_memory().numpy()
        d3.get_state_fe(Ph, fh)
        Ke = max(1, min(K, args.e2e_steps))
        torch.cuda.synchronize()
        barrier(ws)
        t0 = time.perf_counter()
        for s in range(Ke):
            d3.set_state_fe(Ph, fh)
            d3.step(1)
            d3.get_state_fe(Ph, fh)
        te = reduce_max(time.perf_counter() - t0, ws)
        e2e = {"value": ws * cells * Ke / te / 1e6, "unit": UNIT, "steps": Ke,
               "h2d_bytes_per_step": int(Ph.nbytes + fh.nbytes),
               "d2h_bytes_per_step": int(Ph.nbytes + fh.nbytes)}
        d3.close()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_seconds)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K,
            "warmup": args.warmup, "ms_per_step": t_max / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec_main != ferrox.MIXED else "f32+f64",
            "data": "synthetic",
            "config": bench_config(ws, args) if args.workload == "mfim_256x256x32" else
            dict(bench_config(ws, args), workload=cfg["label"], cells=cells),
            "vcycles_per_step": vcycles_per_step,
            "outer_iterations_per_step": cycles_per_step, "gpu_launches": launches,
            "learned_main": None if learned_main is None else
            {k: v for k, v in learned_main.items() if k != "params"},
            "roofline": roof, "kernel_breakdown_ms_one_step": breakdown,
            "vs_plain_fp64": (mixed_v / fp64_v) if (mixed_v and fp64_v) else None,
            "other_precision": other, "fast_form": fast,
            "vs_plain_fp64_fast_form": (fast["value"] / fp64_v) if (fast and fp64_v) else None,
            "learned_form": learned, "batch_qv": batch, "batch_qv_fp64": batch64, "mfism": mfism, "e2e": e2e, "cpu_baseline": cpu,
            "clocks": ck}
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# --------------------------------------------------------------- learned warm start -----

def run_learned(args, ws, cfg, geom, P0, cells, sweep, timed_run):
    """Mixed form + extrapolated guess + the learned warm start: snapshots recorded on
    the workload itself (bias points of the sweep), GPU training, then timed steps."""
    import numpy as np
    import torch

    from paper_2210_15668_gb300 import ferrox
    num = ferrox.make_numerics(cfg["dt"], order=1, tol=1e-10, precision=ferrox.MIXED,
                               max_cycles=200, guess=1, inner=FAST_INNER)
    d = ferrox.Device(geom, P0, numerics=num)
    lv = d.levels()[2]
    net = ferrox.NN(lv[2], lv[1], lv[0], capacity=args.nn_snapshots, seed=7)
    d.set_bias(0.0, sweep[0])
    d.solve_poisson()
    d.attach_nn(net, 1)
    t0 = time.perf_counter()
    for k in range(args.nn_snapshots):
        if k % 25 == 0:
            d.set_bias(0.0, sweep[(k // 25) % len(sweep)])
        d.step(1)
    losses = net.train(epochs=args.nn_epochs, lr=3e-4, batch=8)
    torch.cuda.synchronize()
    prep = time.perf_counter() - t0
    d.attach_nn(None, 0)
    d.set_bias(0.0, sweep[0])
    d.attach_nn(net, 2)
    K = args.steps
    t, s0, s1, _ = timed_run(d, K, args.warmup)
    t = reduce_max(t, ws)
    out = {"precision": "mixed", "guess": "extrapolated + learned", "inner": FAST_INNER,
           "value": ws * cells * K / (t / 1e3) / 1e6, "ms_per_step": t / K,
           "vcycles_per_step": (s1["vcycles"] - s0["vcycles"]) / K,
           "outer_iterations_per_step": (s1["cycles"] - s0["cycles"]) / K,
           "corrections_rejected": s1["nn_rejected"] - s0["nn_rejected"],
           "snapshots": args.nn_snapshots, "epochs": args.nn_epochs,
           "train_loss_first_last": [float(losses[0]), float(losses[-1])],
           "collect_and_train_s": prep, "params": 79.5e3}
    d.close()
    net.close()
    return out


def train_network_on(args, ferrox, I, snapshots=None, epochs=None):
    """Collect snapshots on the --nn-train-on workloads (default: the 256x256x32 MFIM
    and 256x256x64 MFISM) and train one network on all of them (the weights carry
    over between grids: the network is fully convolutional)."""
    import torch
    nsnap = args.nn_snapshots if snapshots is None else snapshots
    nep = args.nn_epochs if epochs is None else epochs
    params, losses, t0 = None, [], time.perf_counter()
    for name in args.nn_train_on.split(","):
        cfg = workload_config(name)
        g = cfg["geom"]
        num = ferrox.make_numerics(cfg["dt"], order=1, tol=1e-10, precision=ferrox.MIXED, guess=1)
        d = ferrox.Device(g, I.random_polarization(g, cfg["seed"]), numerics=num)
        lv = d.levels()[2]
        net = ferrox.NN(lv[2], lv[1], lv[0], capacity=nsnap,
                        params=params if params is not None else ferrox.nn_init_params(7))
        sweep = cfg["sweep"]
        d.set_bias(0.0, sweep[0])
        d.solve_poisson()
        d.attach_nn(net, 1)
        for k in range(nsnap):
            if len(sweep) > 1 and k % 25 == 0:
                d.set_bias(0.0, sweep[(k // 25) % len(sweep)])
            d.step(1)
        losses += [float(x) for x in net.train(epochs=nep, lr=3e-4, batch=8)]
        w, b, _, _ = net.params()
        params = ([wi.reshape(27, ci, co) for wi, (ci, co) in zip(w, ferrox.NN_LAYERS)], b)
        d.close()
        net.close()
    torch.cuda.synchronize()
    return {"params": params, "snapshots_per_workload": nsnap, "epochs": nep,
            "trained_on": args.nn_train_on,
            "train_loss_first_last": [losses[0], losses[-1]],
            "collect_and_train_s": time.perf_counter() - t0}


# ------------------------------------------------------------- MFISM workloads -----

MFISM_INNER = 4   # V-cycles per Newton (FP64) residual in the fast MFISM form


def time_steps(d, K, W, flush):
    """W untimed steps, then K steps each bracketed by CUDA events on the context's
    stream, L2 flushed before every step.  Returns (total ms, stats before, after)."""
    import torch
    for _ in range(W):
        flush.zero_()
        d.step(1)
    torch.cuda.synchronize()
    st0 = d.stats()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for s in range(K):
        flush.zero_()
        ev[s][0].record(d.stream)
        d.step(1)
        ev[s][1].record(d.stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev), st0, d.stats()


def run_mfism(args, ws, hbm_peak):
    """The two MFISM stacks (metal / p-Si / SiO2 / HZO / metal, damped Newton with
    Boltzmann carriers, MG to 1e-10): 256x256x64 (seed 2) and 512x512x128 (seed 5),
    at 0 V, each in plain FP64 multigrid (the defect-correction Newton form), the
    fast mixed form (FP32 V-cycles in FP64 Newton defect correction, extrapolated
    guess, MFISM_INNER V-cycles per Newton residual), and on 512x512x128 the same
    with the learned warm start, the network trained on 256x256x32 MFIM and
    256x256x64 MFISM snapshots."""
    import torch
    from paper_2210_15668_gb300 import ferrox, inputs as I
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    K, W = args.steps, args.warmup
    net_params = None
    out = {}
    for name in ("mfism_256x256x64", "mfism_512x512x128"):
        cfg = workload_config(name)
        geom = cfg["geom"]
        cells = geom["nx"] * geom["ny"] * I.nz_of(geom)
        P0 = I.random_polarization(geom, cfg["seed"])
        forms = [("fp64", dict(precision=ferrox.FP64)),
                 ("mixed_fast", dict(precision=ferrox.MIXED, guess=1, inner=MFISM_INNER))]
        if name == "mfism_512x512x128" and not args.no_learned:
            forms.append(("mixed_fast_learned", dict(precision=ferrox.MIXED, guess=1, inner=MFISM_INNER)))
        res = {"cells": cells, "steps": K, "warmup": W, "tol": 1e-10,
               "l2": "flushed between timed steps (256 MB write)", "label": cfg["label"]}
        for form, kw in forms:
            num = ferrox.make_numerics(cfg["dt"], order=1, tol=1e-10, max_cycles=200, **kw)
            d = ferrox.Device(geom, P0, numerics=num)
            d.set_bias(0.0, cfg["v_top"])
            d.solve_poisson()
            net = None
            extra = {}
            if form.endswith("learned"):
                if net_params is None:
                    tr = train_network_on(args, ferrox, I, snapshots=args.mfism_nn_snapshots,
                                          epochs=args.mfism_nn_epochs)
                    net_params = tr["params"]
                    extra = {k: v for k, v in tr.items() if k != "params"}
                lv2 = d.levels()[2]
                net = ferrox.NN(lv2[2], lv2[1], lv2[0], params=net_params)
                d.attach_nn(net, 2)
            t, s0, s1 = time_steps(d, K, W, flush)
            t = reduce_max(t, ws)
            r = {"value": ws * cells * K / (t / 1e3) / 1e6, "unit": UNIT, "ms_per_step": t / K,
                 "vcycles_per_step": (s1["vcycles"] - s0["vcycles"]) / K,
                 "newton_iterations_per_step": (s1["cycles"] - s0["cycles"]) / K}
            r.update(extra)
            if net is not None:
                r["corrections_rejected"] = s1["nn_rejected"] - s0["nn_rejected"]
            else:
                prof = d.profile_step(with_bytes=True)
                fp64c = ("tdgl", "resid", "update") + (() if kw["precision"] == ferrox.MIXED else
                                                      ("smooth_fine", "smooth_coarse", "restrict",
                                                       "prolong", "tail"))
                cl, wh = class_rooflines(prof, hbm_peak, fp64c,
                                         ("resid",) if kw["precision"] == ferrox.MIXED else ())
                wh["graph_ms_per_step"] = t / K
                r["roofline_classes"] = cl
                r["whole_step"] = wh
            res[form] = r
            d.close()
            if net is not None:
                net.close()
        if "fp64" in res and "mixed_fast" in res:
            res["vs_plain_fp64"] = res["mixed_fast"]["value"] / res["fp64"]["value"]
        out[name] = res
    return out


# ------------------------------------------------------- batched Q-V sweep workload -----

def run_batch_qv(args, ws, precision=None):
    """64 MFIM instances (lateral sizes from {32,48,64,96,128}, Nz = 16, V ~ U[-2, 2],
    seed 3) advanced by the engine the autotuner picks: one persistent launch per
    call, or a CUDA graph of per-phase launches.  FP64 residual; FP32 smoothing in
    the mixed form, FP64 in the FP64 form."""
    import numpy as np
    import torch

    from paper_2210_15668_gb300 import ferrox, inputs as I
    if precision is None:
        precision = ferrox.MIXED
    inst = I.batch_sweep()
    geoms = [x["geom"] for x in inst]
    P0s = [I.random_polarization(g, x["seed"]) for g, x in zip(geoms, inst)]
    cells = sum(p.size for p in P0s)
    B = ferrox.Batch(geoms, P0s, ferrox.make_numerics(4e-13, tol=1e-10, precision=precision))
    B.set_bias(np.zeros(len(inst)), [x["v_top"] for x in inst])
    B.solve_poisson()
    B.step(max(3, args.warmup // 4))            # includes the launch-shape tuning
    torch.cuda.synchronize()
    s0 = B.stats()
    K = args.batch_steps
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("batch_timed")   # lets ncu select this launch
    a.record()
    B.step(K)                                    # K steps in one call
    b.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    t = reduce_max(a.elapsed_time(b), ws)
    s1 = B.stats()
    tuning = B.tuning()
    engine = ("one persistent cooperative launch per call" if tuning["engine"] == 0
              else "a CUDA graph per step: one launch per phase, the solve loop in a WHILE node")
    # one more step with the same kernels launched one by one, CUDA-event timed per
    # phase class (profilers cannot see the kernel nodes of the step's graph)
    phases = B.profile_phases() if tuning["engine"] == 1 else None
    out = {"workload": "64 MFIM instances {32..128}^2 x 16, V ~ U[-2,2], seed 3", "cells": cells,
           "steps": K, "value": ws * cells * K / (t / 1e3) / 1e6, "unit": UNIT, "ms_per_step": t / K,
           "precision": "mixed" if precision == ferrox.MIXED else "fp64", "engine": engine,
           "vcycles_per_step_mean": float(np.mean([s1[i]["cycles"] - s0[i]["cycles"] for i in range(len(inst))])) / K,
           "tuning": tuning, "l2": "working set ~270 MB > L2 (no flush)",
           "phase_breakdown_one_step": None if phases is None else
           {k: {"ms": round(v[0], 4), "launches": v[1]} for k, v in phases.items()}}
    B.close()
    return out


# --------------------------------------------------------------- oracle on CPU -------

def _oracle_steps(budget_s, max_steps=None):
    import numpy as np

    import oracle
    from oracle import tdgl
    from paper_2210_15668_gb300 import inputs as I
    cfg = I.mfim_sweep()
    geom = cfg["geom"]
    pl = oracle.planes(geom)
    P = I.random_polarization(geom, cfg["seed"])
    v = cfg["sweep"][0]
    phi = tdgl.solve_poisson(P, np.zeros(P.shape[1:]), pl, geom, 0.0, v)   # Step 0
    cells = P[0].size
    n = 0
    t0 = time.perf_counter()
    while True:
        P, phi = tdgl.step(P, phi, pl, geom, cfg["dt"], 0.0, v)
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s or (max_steps and n >= max_steps):
            break
    return cells, n, el


def cpu_model():
    """CPU model name of this host (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _oracle_replica(job):
    """One spawned process: wait for the common start time, then run oracle steps for
    the budget (or max_steps).  Returns (cells, steps, elapsed s)."""
    budget_s, max_steps, warm, t_start = job
    if warm:
        _oracle_steps(1e9, max_steps=warm)
    while time.time() < t_start:
        time.sleep(0.001)
    return _oracle_steps(budget_s, max_steps=max_steps)


def oracle_all_cores(budget_s, max_steps=None, warm=0, cores=None):
    """The oracle on every host core at once: one independent replica of the same
    workload per core (spawned processes, one BLAS/OpenMP thread each), all started
    together; throughput = all replicas' cell-steps over the slowest replica's time."""
    import multiprocessing as mp
    cores = cores or host_cores()
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        t_start = time.time() + 12.0 + 2.0 * warm       # after every replica's import and warm-up
        res = pool.map(_oracle_replica, [(budget_s, max_steps, warm, t_start)] * cores)
    cells = res[0][0]
    n_tot = sum(r[1] for r in res)
    el = max(r[2] for r in res)
    return cells, n_tot, el, cores, min(r[1] for r in res)


ORACLE_NOTE = ("numpy FP64 oracle, exact FFT/tridiagonal Poisson solve (a different algorithm "
               "from the GPU multigrid)")


def cpu_baseline(budget_s):
    cells, n, el = _oracle_steps(budget_s)
    one = {"value": cells * n / el / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{n} oracle steps of mfim_256x256x32 at -2 V from Step 0 ({el:.1f} s; "
                     f"{ORACLE_NOTE}; one core)"}
    cells, n_tot, el_all, cores, n_min = oracle_all_cores(budget_s)
    return {"value": cells * n_tot / el_all / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} replicas (one per host core, spawned processes) of oracle steps of "
                      f"mfim_256x256x32 at -2 V from Step 0, {n_tot} steps in total (>= {n_min} each) "
                      f"in {el_all:.1f} s; {ORACLE_NOTE}",
            "cpu_model": cpu_model(), "nproc": os.cpu_count(), "single_core": one}


def bench_config(ws, args=None):
    """The workload record of the 256x256x32 line (the same for both arms)."""
    from paper_2210_15668_gb300 import inputs as I
    cfg = I.mfim_sweep()
    g = cfg["geom"]
    c = {"workload": "mfim_256x256x32 Q-V sweep (first steps at -2 V), seed 1",
         "cells": g["nx"] * g["ny"] * I.nz_of(g), "tol": 1e-10, "order": 1, "precision": "fp64",
         "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{ws}"}
    if args is not None:
        c.update(precision=args.precision, guess=args.guess, nu1=args.nu1, nu2=args.nu2, inner=args.inner)
    return c


def run_reference(args, ws, rank):
    if rank != 0:
        return
    # every host core runs one replica: W warm-up steps, then K timed steps each
    # (bounded: K and W are capped so the run ends within a few minutes)
    K = max(1, min(args.steps, 30))
    W = max(1, min(args.warmup, 3))
    cells, n_tot, el, cores, n_min = oracle_all_cores(1e9, max_steps=K, warm=W)
    value = cells * n_tot / el / 1e6
    cfg = bench_config(ws, args)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K,
            "warmup": W, "ms_per_step": el / K * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{cores} replicas x {K} oracle steps of the workload in {el:.1f} s "
                                       f"(after {W} warm-up steps each); {ORACLE_NOTE}",
                             "cpu_model": cpu_model(), "nproc": os.cpu_count()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_nn_forward(args):
    """Event-timed forwards of the warm-start network (random weights) on the level-2
    grids of the 256x256x32 stack (64 x 64 x 8) and of the 512x512x128 stack
    (128 x 128 x 32), from a seeded input, with the convolutions on the tcgen05
    kernel and on the mma.sync kernel."""
    import torch
    from paper_2210_15668_gb300 import ferrox
    out = {}
    for D, H, W in ((8, 64, 64), (32, 128, 128)):
        net = ferrox.NN(D, H, W, seed=3)
        g = torch.Generator(device="cuda").manual_seed(0)
        x = torch.randn(D * H * W, 16, device="cuda", dtype=torch.float32, generator=g)
        res = {}
        for tc in (True, False):
            net.use_tensor_memory(tc)
            for _ in range(args.warmup):
                net.forward(x)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(args.steps):
                net.forward(x)
            b.record()
            torch.cuda.synchronize()
            res["tcgen05" if tc else "mma_sync"] = a.elapsed_time(b) / args.steps * 1e3
        info = net.kernel_info()
        net.use_tensor_memory(True)
        res["tc_convs"] = net.kernel_info()["tc_forward"]
        res["fault"] = info["fault"]
        out[f"{D}x{H}x{W}"] = res
        net.close()
    print(json.dumps({"nn_forward_us": out, "forwards": args.steps}))


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed", "fp64_defect"], default="fp64",
                    help="fp64: V-cycles on phi (residual norm fused into the restriction); "
                         "fp64_defect: FP64 V-cycles on the correction equation; mixed: FP32 "
                         "V-cycles in FP64 defect correction")
    ap.add_argument("--workload", default="mfim_256x256x32",
                    help="mfim_256x256x32 (the benchmark) or mfim_NXxNYxNZ (profiling copies)")
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--inner", type=int, default=1, help="V-cycles per outer (FP64) iteration")
    ap.add_argument("--nu1", type=int, default=2, help="pre-smoothing sweeps per level")
    ap.add_argument("--nu2", type=int, default=2, help="post-smoothing sweeps per level")
    ap.add_argument("--guess", type=int, choices=[0, 1], default=0,
                    help="initial potential of each solve: 0 previous (paper), 1 extrapolated")
    ap.add_argument("--learned", action="store_true",
                    help="attach a network trained on the 256^2 x 32 MFIM and 256^2 x 64 MFISM snapshots")
    ap.add_argument("--nn-snapshots", type=int, default=300)
    ap.add_argument("--nn-train-on", default="mfim_256x256x32,mfism_256x256x64",
                    help="workloads whose snapshots train the --learned network (comma list)")
    ap.add_argument("--nn-epochs", type=int, default=20)
    ap.add_argument("--batch-steps", type=int, default=50)
    ap.add_argument("--no-mfism", action="store_true", help="skip the 256x256x64 and 512x512x128 MFISM keys")
    ap.add_argument("--mfism-nn-snapshots", type=int, default=1000,
                    help="snapshots per training workload for the 512x512x128 learned form")
    ap.add_argument("--mfism-nn-epochs", type=int, default=8)
    ap.add_argument("--nn-forward", action="store_true",
                    help="time only the network forward on the 64x64x8 level of the benchmark "
                         "stack (--steps forwards; for profiling the convolution kernels)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    ws, rank, local = dist_env()
    if args.nn_forward:
        run_nn_forward(args)
    elif args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
