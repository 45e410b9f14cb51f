#!/usr/bin/env python
"""Benchmark of the SMP topological-charge-density path on one GB300.

Workload (a "step"): q(x) and Q for every site of the 8^3 x 16 quantised-flux
configuration (Q = 2, noise 0.1, random gauge transform), symmetric
multi-probing r_min = 4, Normal mode: 256 colour classes x 12 = 3072 sources,
each a 14-shift multi-shift CG to relative residual 1e-10 (kappa = 0.21,
14-pole Zolotarev), then the gamma_5 contraction and Q.

Metric: q(x) sites/s = sites of the lattice / step time.
  value : mixed-precision batched path, all 3072 sources in one batch, inputs
          resident on the GPU: FP64-accurate (float-float) iterations until
          ||r|| < 1e-3 ||b||, then FP32 iterations; shifted vectors, scalars and
          reductions in FP64, so every shift stops at the same 1e-10 residual
          as the FP64 path;
  e2e   : the same call with host buffers: gauge field uploaded from pinned
          host memory and q(x) read back every step;
  fp32_reliable : FP32 iterations with FP64 reliable updates (faster, but
          its shifted systems keep an FP32 error floor);
  fp64_plain / fp64_batched : the FP64 path one source at a time / batched,
          timed on a sample of classes and scaled to all classes;
  roofline : the dominant solver kernel's algorithmic bytes / CUDA-event time
          against the measured HBM bandwidth; its arithmetic rate against the
          measured FP32 (or FP64) peak as the secondary `alu` entry;
  cpu_baseline : the FP64 oracle on the host cores on one class (12 sources).

The timed steps run as a user runs them (CUDA graphs on, no per-launch
events); one further step with per-launch CUDA events gives the kernel times
of the roofline, and one with the true_residual option the FP64 true residual.
The Zolotarev interval comes from the GPU Lanczos estimate
(smpq_measure_spectrum), timed as setup.

Multi-GPU (torchrun, N ranks): every rank evaluates its own configuration
(independent problems, no collective on the data path) -> weak scaling.
`--impl reference` times the CPU oracle on the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CONFIG = "flux8x16"
# algorithmic arithmetic per site and source of one launch, in FP32 operations:
# float-float D_W = 8 hops x (36 unnormalised additions x 8 ops + 12 real parts
# of three-term complex dot products x 64 ops) + 24 renormalisations x 6 ops
# = 8592, plus the epilogue (1368 for t = D_W p with norms, 1824 for the r update)
DF64_OPS_A = 8592 + 1368
DF64_OPS_B = 8592 + 1824
# FP64 D_W: 1320 flop hopping + 24 (kappa scale) + 24 (norm) / + 72 (update and norm)
FP64_FLOP_A = 1320 + 48
FP64_FLOP_B = 1320 + 96
R_MIN, MODE = 4, 0
KAPPA = 0.21


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        hbm = d.get("hbm_gbs") or d.get("hbm_GBs")
        if hbm:
            return float(hbm), "measured"
    return 6800.0, "fallback"


def _src_hash(kernel=""):
    """Hash of the files that define a solver kernel (wilson.cuh, df64.cuh,
    device.cuh, msolve.cu, and stage.cuh for the staged FP32 kernels `*_st`):
    traffic figures taken on other sources are void."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1901_02211_gb300", "csrc")
    files = ["df64.cuh", "device.cuh", "msolve.cu", "wilson.cuh"] + (["stage.cuh"] if "_st[" in kernel else [])
    for f in files:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def _traffic(kernel, B):
    """DRAM bytes per launch from the committed ncu summary, if taken on this source."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel)
    if not e or e.get("src_hash") != _src_hash(kernel):
        return None
    # scale a smaller capture to this launch by the sources processed
    return float(e["dram_bytes_per_launch"]) * B / float(e["B"])


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = "/tmp/smpq_clocks_%d.csv" % os.getpid()

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "samples": len(sm),
                "reasons": sorted(reasons)}


def config_for_rank(rank, name=CONFIG):
    """The configuration a rank evaluates: rank 0 the named one, rank k > 0 an
    independent configuration of the same shape and recipe with other seeds
    (independent problems: no data-path collective between ranks)."""
    from synth import CONFIGS, make_config
    if rank == 0:
        return make_config(name)
    p = dict(CONFIGS[name])
    p["seed_noise"] += 100 * rank
    p["seed_gauge"] += 100 * rank
    CONFIGS["%s_r%d" % (name, rank)] = p
    return make_config("%s_r%d" % (name, rank))


def max_over_ranks(value, device="cpu"):
    """Max of a per-rank float over the process group (the timing rule)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_oracle_sample(U, dims, a, b, n_classes=1, tol=1e-10, rmin=R_MIN):
    """FP64 oracle on `n_classes` colour classes (12 sources each); returns (sites/s, sites, sec, threads)."""
    from oracle import native, probing, qx, zolotarev
    c0, c, q, _ = zolotarev.zolotarev(14, a, b)
    colour, n = probing.color_sites(dims, rmin, MODE)
    classes = list(range(n_classes))
    t0 = time.perf_counter()
    qv, st = qx.smp_qx(U, dims, KAPPA, (c0, c, q), colour, n, tol=tol, colours=classes, batch_colours=n_classes)
    dt = time.perf_counter() - t0
    sites = int(np.isin(colour, classes).sum())
    return sites / dt, sites, dt, native.threads()


def _oracle_interval(name, U, dims):
    """Zolotarev interval for the CPU legs: the oracle's ARPACK spectrum, stored
    by tests/golden/make_spectra.py when there is one, else computed here."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", "spectra.json")) as f:
            sp = json.load(f)[name]
        return 0.98 * sp["lmin2"], 1.02 * sp["lmax2"]
    except KeyError:
        from oracle import spectrum
        lo, hi = spectrum.h2_extremes(U, dims, KAPPA, tol=1e-8)
        return 0.98 * lo, 1.02 * hi


def run_reference(args):
    """The oracle (plain FP64 CPU code) as the reference arm: each step is one
    colour class (12 sources and its sites) of the workload, on all host cores.
    value = the sites of that sample per second it took; ms_per_step = the
    measured time of one sample step (a whole-lattice step would take
    N_p times as long: that extrapolation is labelled, not reported as the step)."""
    ws, rank, local = _dist()
    if rank != 0:
        return
    from oracle import native
    from synth import make_config
    native.build()
    cfg = make_config(args.config)
    U, dims = cfg["U"], cfg["dims"]
    a, b = _oracle_interval(args.config, U, dims)
    V = int(np.prod(dims))
    n_cls = args.rmin ** 4
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state; bounded steps only
    vals, secs = [], []
    for _ in range(args.steps):
        v, sites, dt, thr = cpu_oracle_sample(U, dims, a, b, 1, rmin=args.rmin)
        vals.append(v)
        secs.append(dt)
    value = float(np.median(vals))
    line = {
        "impl": "reference", "metric": "q(x) sites/s", "value": value, "unit": "sites/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * float(np.median(secs)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": _workload_name(args),
                   "sample": "each step: 1 colour class (12 sources, %d of %d sites)" % (sites, V),
                   "whole_lattice_step_ms_extrapolated": 1000.0 * V / value},
        "cpu_baseline": {"value": value, "unit": "sites/s", "cores": thr, "kind": "oracle",
                         "sample": "1 of %d colour classes per step (12 sources, %d sites), FP64, tol 1e-10"
                                   % (n_cls, sites)},
        "e2e": {"value": value, "unit": "sites/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _alu_peaks(dev):
    """Measured FP32 (packed two-lane, the form the float-float kernels issue)
    and FP64 multiply-add lane rates of this GPU (smpq_alu_peak)."""
    from paper_1901_02211_gb300 import smpq
    try:
        return {"fp32_lane_ops_per_s": smpq.smpq_alu_peak(dev, smpq.ALU_FP32X2),
                "fp32_scalar_lane_ops_per_s": smpq.smpq_alu_peak(dev, smpq.ALU_FP32),
                "fp64_fma_per_s": smpq.smpq_alu_peak(dev, smpq.ALU_FP64)}
    except Exception as e:  # reported, never invented
        return {"error": str(e)}


def _kernel_table(prec, stats, V, B, peak_hbm, peak_kind, alu):
    """Per solver kernel: average CUDA-event time per launch (profiled step),
    algorithmic bytes per launch (spinor fields read and written + links, as in
    the module docstring of msolve.cu) against the measured HBM bandwidth, and
    for the FP64-accurate kernels their arithmetic against the measured ALU peak."""
    from paper_1901_02211_gb300 import smpq
    link32, link64 = 4 * 9 * 8, 4 * 9 * 16
    b_vecs = 6 if prec == smpq.SMPQ_FP32 else 4  # t, p, r (+ x_lo) read, r (+ x_lo) written
    half = prec in (smpq.SMPQ_FP16N, smpq.SMPQ_BF16N)
    lo = {smpq.SMPQ_FP16N: "fp16n", smpq.SMPQ_BF16N: "bf16n"}.get(prec, "fp32")
    st_ = "_st" if stats[-1].get("staged") and lo == "fp32" else ""  # neighbours staged in shared memory
    kern = {}
    for key, ms_k, n_k, esz_k, nvec in (
            ("k_apply_a%s[%s]" % (st_, lo), "dslash_ms", "dslash_launches", 8, 2),
            ("k_apply_b%s[%s]" % (st_, lo), "update_ms", "update_launches", 8, b_vecs),
            ("k_apply_a[fp64-accurate]", "dslash_hi_ms", "dslash_hi_launches", 16, 2),
            ("k_apply_b[fp64-accurate]", "update_hi_ms", "update_hi_launches", 16, 4)):
        tot = sum(x[ms_k] for x in stats)
        n = sum(x[n_k] for x in stats)
        if not n or tot <= 0:
            continue
        if half and esz_k == 8:
            # half-format p and t (52 bytes per site and source with the norm),
            # FP32 r and x_lo (96 bytes each, read and written in k_apply_b),
            # reconstruct-12 links (96 bytes per site)
            nbytes = V * B * (2 * 52 if key.startswith("k_apply_a") else 2 * 52 + 4 * 96) + V * 96
        else:
            nbytes = V * B * nvec * 12 * esz_k + V * (link32 if esz_k == 8 else link64)
        ms = tot / n
        k = dict(ms=ms, n=n, share_ms=tot / len(stats), bytes=nbytes, bound="hbm", unit="GB/s", peak=peak_hbm,
                 peak_source=peak_kind, achieved=nbytes / (ms / 1000.0) / 1e9)
        if esz_k == 16 and prec == smpq.SMPQ_MIXED and "fp32_lane_ops_per_s" in alu:  # float-float
            ops = V * B * (DF64_OPS_A if key.startswith("k_apply_a") else DF64_OPS_B)
            pk = alu["fp32_lane_ops_per_s"] / 1e12
            k["alu"] = dict(achieved=ops / (ms / 1000.0) / 1e12, peak=pk, unit="T FP32 lane-ops/s",
                            frac=ops / (ms / 1000.0) / 1e12 / pk, algorithmic=ops,
                            peak_source="measured (smpq_alu_peak, packed FFMA2 probe)")
        elif esz_k == 16 and "fp64_fma_per_s" in alu:  # native FP64
            fl = V * B * (FP64_FLOP_A if key.startswith("k_apply_a") else FP64_FLOP_B)
            pk = 2 * alu["fp64_fma_per_s"] / 1e12
            k["alu"] = dict(achieved=fl / (ms / 1000.0) / 1e12, peak=pk, unit="TFLOP/s (FP64)",
                            frac=fl / (ms / 1000.0) / 1e12 / pk, algorithmic=fl,
                            peak_source="measured (smpq_alu_peak, DFMA probe, 2 flop each)")
        kern[key] = k
    return kern


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1901_02211_gb300 import Session, smpq

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream().cuda_stream

    cfg = config_for_rank(rank, args.config)
    U, dims = cfg["U"], cfg["dims"]
    V = int(np.prod(dims))
    if args.dslash_only:  # profiling entry: the stand-alone D_W formats alone, no solve
        s = Session(device=dev, stream=stream)
        s.load_gauge(dims, U)
        print(json.dumps({"workload": "%dx%dx%dx%d %s, stand-alone D_W" % (tuple(dims) + (args.config,)),
                          "dslash": _dslash_formats(s, V, args.dslash_columns)}), flush=True)
        s.close()
        return
    prec = {"fp32": smpq.SMPQ_FP32, "fp64": smpq.SMPQ_FP64, "mixed": smpq.SMPQ_MIXED, "fp16n": smpq.SMPQ_FP16N,
            "bf16n": smpq.SMPQ_BF16N}[args.precision]

    s = Session(device=dev, stream=stream, precision=prec, tol=1e-10, rhs_block=0, iters_per_check=10,
                use_graphs=1, profile=0, switch_residual=args.switch, autotune=0 if args.no_autotune else 1)
    s.load_gauge(dims, U)
    # setup, timed on its own: the Zolotarev interval from the GPU Lanczos estimate
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lo, hi = s.measure_spectrum(args.lanczos)
    spectrum_s = time.perf_counter() - t0
    a, b = 0.98 * lo, 1.02 * hi
    s.set_spectrum(a, b)
    n_classes = s.build_sources(args.rmin, MODE)
    q_re = torch.zeros(V, dtype=torch.float64, device="cuda")
    q_im = torch.zeros(V, dtype=torch.float64, device="cuda")

    sub = list(range(args.classes)) if args.classes else None
    V_step = V if sub is None else V * len(sub) // n_classes  # sites whose q(x) one step produces

    def step():
        if sub is None:
            return smpq.smpq_compute_qx(s.ctx, q_re, q_im)
        st = smpq.smpq_compute_qx_classes(s.ctx, sub, q_re, q_im)
        return st["Q"], st

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    stats = []
    with Clocks(dev) as clk:
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        # the NVTX range names the timed steps for a profiler's launch list
        # (ncu --nvtx --nvtx-include smpq_timed_steps/)
        torch.cuda.nvtx.range_push("smpq_timed_steps")
        for _ in range(args.steps):
            Q, st = step()
            stats.append(st)
        torch.cuda.nvtx.range_pop()
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    if ws > 1:
        ms = max_over_ranks(ms, "cuda")
    value = ws * V_step / (ms / 1000.0)
    clocks = clk.summary()
    launches = sum(x["kernel_launches"] for x in stats)
    q_out = {"headline": (q_re + 1j * q_im).cpu().numpy()} if sub is None else {}

    # one more step with CUDA events around every D_W launch (graphs off): the
    # kernel times of the roofline; then one with the FP64 true residual
    s.set_options(profile=1)
    Qp, stp = step()
    s.set_options(profile=0, true_residual=1)
    Qt, stt = step()
    enforced = None
    if prec == smpq.SMPQ_MIXED and sub is None and not args.no_baselines:
        # the variant that drives the base system to a true residual below tol
        s.set_options(true_residual=2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Qe, ste = step()
        te = time.perf_counter() - t0
        q_out["mixed_base_residual_enforced"] = (q_re + 1j * q_im).cpu().numpy()
        enforced = {"value": V_step / te, "unit": "sites/s", "iterations": ste["max_iterations"],
                    "true_resid_base": ste["true_resid"], "Q": Qe, "abs_dQ_vs_headline": abs(Qe - Q),
                    "note": "true_residual = 2: after every shift converged, one residual replacement and a CG "
                            "restart of the base shift until its true residual is below tol"}
    s.set_options(true_residual=0)
    B = stats[-1]["n_rhs"] // max(1, stats[-1]["n_batches"])
    peak_hbm, peak_kind = _peaks()
    alu = _alu_peaks(dev)
    kern = _kernel_table(prec, [stp], V, B, peak_hbm, peak_kind, alu)
    dom = max(kern, key=lambda k: kern[k]["share_ms"])
    traffic = _traffic(dom, B)
    esz = 8 if prec == smpq.SMPQ_FP32 else 16

    e2e_val = None
    if args.no_e2e:
        pass
    else:
        e2e_val = _e2e(args, s, dims, U, V, a, b, prec, dev, stream, ws)
    out = _baselines(args, rank, dims, U, V, a, b, n_classes, dev, stream, q_out) if rank == 0 else {}
    if rank == 0 and not args.no_extra:
        out["uneven_batch"] = {"bf16n": _uneven(args, smpq.SMPQ_BF16N, dev, stream),
                               "mixed": _uneven(args, smpq.SMPQ_MIXED, dev, stream)}
    if rank == 0 and not args.no_extra:
        out["c3_16x32"] = _c3_record(args, dev, stream)
        out["c5_32x64"] = _c5_record(args, dev, stream)
    if rank == 0 and not args.no_baselines and args.low_modes > 0 and sub is None:
        q_ref = (q_re + 1j * q_im).cpu().numpy()
        out["low_mode_projection"] = _low_modes(args, dims, U, V, a, b, prec, dev, stream, q_ref)
    out["spectrum"] = {"lmin2": a, "lmax2": b, "lanczos_lmin2": lo, "lanczos_lmax2": hi, "setup_s": spectrum_s,
                       "source": "GPU Lanczos (smpq_measure_spectrum, %d steps), widened 0.98/1.02" % args.lanczos}
    out["alu_peaks"] = alu
    if enforced is not None:
        out["mixed_base_residual_enforced"] = enforced
    out["sm_count"] = torch.cuda.get_device_properties(dev).multi_processor_count
    if rank == 0 and not args.no_dslash:
        out["dslash"] = _dslash_formats(s, V, B)
    if rank == 0:
        _report(args, ws, V, ms, value, prec, B, esz, clocks, e2e_val, U, launches, dom, kern, traffic, stats, stp,
                stt, out, sub)
    s.close()
    if ws > 1:
        dist.destroy_process_group()


def _dslash_formats(s, V, B, reps=20):
    """Stand-alone D_W (smpq_time_dslash) on the workload's B columns in every
    storage format: CUDA-event time per launch on the context's stream and
    algorithmic bytes (spinor in + out per site and column, links once) against
    the measured HBM bandwidth."""
    from paper_1901_02211_gb300 import smpq
    peak, kind = _peaks()
    res = {"columns": B, "reps": reps, "peak": peak, "peak_source": kind, "unit": "GB/s"}
    staging = s.options.staging
    for name, prec, stg in (("fp16n_recon12", smpq.SMPQ_FP16N, staging), ("bf16n_recon12", smpq.SMPQ_BF16N, staging),
                            ("fp32", smpq.SMPQ_FP32, 0), ("fp32_staged", smpq.SMPQ_FP32, 1),
                            ("fp64", smpq.SMPQ_FP64, staging)):
        s.set_options(staging=stg)  # FP32: neighbours staged in shared memory, or plain loads
        ms, nbytes = smpq.smpq_time_dslash(s.ctx, B, False, prec, reps)
        gbs = nbytes / (ms / 1000.0) / 1e9
        res[name] = {"avg_launch_ms": ms, "algorithmic_bytes": nbytes, "achieved": gbs, "frac": gbs / peak}
    s.set_options(staging=staging)
    return res


def _e2e(args, s, dims, U, V, a, b, prec, dev, stream, ws):
    """Same metric through host buffers: pinned gauge upload + q(x) read-back each step."""
    import torch

    from paper_1901_02211_gb300 import Session, smpq
    Upin = torch.from_numpy(np.ascontiguousarray(U)).pin_memory()
    hq_re = torch.zeros(V, dtype=torch.float64).pin_memory()
    hq_im = torch.zeros(V, dtype=torch.float64).pin_memory()
    s2 = Session(device=dev, stream=stream, precision=prec, tol=1e-10, rhs_block=0, iters_per_check=10,
                 use_graphs=1)
    s2.load_gauge(dims, Upin.numpy())
    s2.set_spectrum(a, b)
    s2.build_sources(args.rmin, MODE)

    def e2e_step():
        smpq.smpq_load_gauge(s2.ctx, dims, Upin)
        s2.set_spectrum(a, b)
        s2.build_sources(args.rmin, MODE)
        return smpq.smpq_compute_qx(s2.ctx, hq_re, hq_im)

    e2e_step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    t0 = time.perf_counter()
    n_e2e = max(1, args.steps)
    for _ in range(n_e2e):
        e2e_step()
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = max(e0.elapsed_time(e1), 1000 * (time.perf_counter() - t0)) / n_e2e
    s2.close()
    return ws * V / (e2e_ms / 1000.0)


def _low_modes(args, dims, U, V, a, b, prec, dev, stream, q_ref):
    """The same q(x) with the lowest eigenmodes of H_W treated exactly (GPU
    subspace iteration, then the Zolotarev interval shortened to
    [0.98 lambda_{k+1}^2, b]): setup time, throughput and the difference from
    the headline estimate."""
    import torch

    from paper_1901_02211_gb300 import Session, smpq
    k = args.low_modes
    s4 = Session(device=dev, stream=stream, precision=prec, tol=1e-10, rhs_block=0, iters_per_check=10,
                 use_graphs=1, switch_residual=args.switch)
    s4.load_gauge(dims, U)
    s4.set_spectrum(a, b)
    s4.build_sources(args.rmin, MODE)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev, res, it = s4.low_modes(k)
    setup = time.perf_counter() - t0
    s4.set_spectrum(0.98 * ev[k] ** 2, b)
    s4.compute_qx()
    torch.cuda.synchronize()
    n = max(1, args.steps)
    t0 = time.perf_counter()
    for _ in range(n):
        q, Q, st = s4.compute_qx()
    dt = (time.perf_counter() - t0) / n
    s4.close()
    return {"value": V / dt, "unit": "sites/s", "k": k, "lambda2_k_plus_1": float(ev[k] ** 2),
            "interval": [0.98 * float(ev[k] ** 2), b], "setup_s": setup, "filter_steps": it,
            "max_eig_residual": float(res.max()), "max_iterations": st["max_iterations"], "Q": Q,
            "max_abs_dq_vs_headline": float(np.abs(q - q_ref).max()),
            "note": "setup (the eigen-solve) is per gauge field and not in value"}


def _one_step(name, dims, U, r, prec, dev, stream, switch, max_iter=5000, classes=None, lanczos=300):
    """One untimed-setup, timed q(x) step of a configuration in one precision:
    GPU Lanczos interval (setup), then compute_qx (all classes or a subset)."""
    import torch

    from paper_1901_02211_gb300 import Session, smpq
    V = int(np.prod(dims))
    with Session(device=dev, stream=stream, precision=prec, tol=1e-10, rhs_block=0, iters_per_check=10,
                 use_graphs=1, switch_residual=switch, max_iter=max_iter) as s:
        s.load_gauge(dims, U)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lo, hi = s.measure_spectrum(lanczos)
        setup = time.perf_counter() - t0
        s.set_spectrum(0.98 * lo, 1.02 * hi)
        n_classes = s.build_sources(r, MODE)
        t0 = time.perf_counter()
        try:
            q, Q, st = s.compute_qx(classes=classes)
            err = None
        except smpq.SmpqError as e:
            err = str(e)
        dt = time.perf_counter() - t0
    if err is not None:
        return {"error": err, "seconds": dt, "lambda2_min": lo, "lambda2_max": hi, "max_iter": max_iter}
    nc = n_classes if classes is None else len(classes)
    rec = {"value": V * nc / n_classes / dt, "unit": "sites/s", "seconds": dt, "setup_lanczos_s": setup,
           "extrapolated": classes is not None and nc < n_classes,
           "sources": 12 * nc, "batches": st["n_batches"], "rhs_tile": st["rhs_tile"],
           "iterations": st["max_iterations"], "reliable_updates": st["reliable_updates"],
           "true_resid_base": st["true_resid"], "max_resid": st["max_resid"], "Q": Q,
           "abs_Q_minus_round": st["q_round_dev"], "max_im_q": st["max_im_q"],
           "lambda2_min": lo, "lambda2_max": hi}
    return rec


def _c3_record(args, dev, stream):
    """16^3 x 32 flux configuration (Q = -1, noise 0.15), r_min = 4: all 3072
    sources, one step in the mixed (headline) precision and one with FP16
    storage, per-site norms and reconstruct-12 links."""
    from paper_1901_02211_gb300 import smpq
    from synth import make_config
    cfg = make_config("flux16x32")
    out = {"workload": "16x16x16x32 flux Q=%d noise 0.15 + gauge transform, r_min=4, 256 classes x 12 = 3072 "
                       "sources x 14 shifts, tol 1e-10" % cfg["Q_closed"]}
    for key, prec in (("mixed", smpq.SMPQ_MIXED), ("fp16n", smpq.SMPQ_FP16N)):
        out[key] = _one_step("flux16x32", cfg["dims"], cfg["U"], 4, prec, dev, stream, args.switch)
    return out


def _c5_record(args, dev, stream):
    """32^3 x 64 stout-smoothed Haar configuration, r_min = 8: one colour class
    (12 sources, the batch the configuration names) in FP32 with FP64
    reliable updates; the throughput is that class's sites per second scaled
    to the lattice, labelled extrapolated.  On this rough field H_W is barely
    gapped (lambda^2_min about 5e-5): the iteration cap is bounded, and a solve
    that reaches it is reported with the residual it reached.  Q of one class
    is a partial sum over its sites, not an integer: reported, not asserted."""
    from paper_1901_02211_gb300 import smpq
    from synth import make_config
    t0 = time.perf_counter()
    cfg = make_config("stout32x64")
    gen = time.perf_counter() - t0
    rec = _one_step("stout32x64", cfg["dims"], cfg["U"], 8, smpq.SMPQ_FP32, dev, stream, args.switch,
                    max_iter=args.c5_max_iter, classes=[0])
    rec["generation_s"] = gen
    rec["workload"] = ("32x32x32x64 Haar seed 5001 + 20 stout steps rho 0.1, r_min=8, class 0 of 4096 "
                       "(12 sources), FP32 + FP64 reliable updates, tol 1e-10, max_iter %d" % args.c5_max_iter)
    return rec


def _uneven(args, prec, dev, stream):
    """The uneven batch: three lattices of different size and scheme (8^3x16 r = 2
    Q = 1, 12^3x24 r = 4 Q = 2, 16^3x32 r = 4 Q = 3), one context each, in one
    smpq_compute_qx_batch call: every CG iteration is the same three launches
    for all three lattices.  Sites of all three per second."""
    import torch

    from paper_1901_02211_gb300 import Session, smpq
    from synth import make_config
    lattices = (("flux8x16_b", 2), ("flux12x24", 4), ("flux16x32_b", 4))
    sessions, re_, im_, sites, names = [], [], [], 0, []
    t0 = time.perf_counter()
    for name, r in lattices:
        cfg = make_config(name)
        s4 = Session(device=dev, stream=stream, precision=prec, tol=1e-10, iters_per_check=10, use_graphs=1,
                     switch_residual=args.switch)
        s4.load_gauge(cfg["dims"], cfg["U"])
        s4.measure_spectrum(300)
        s4.build_sources(r, MODE)
        V = int(np.prod(cfg["dims"]))
        sessions.append(s4)
        re_.append(torch.zeros(V, dtype=torch.float64, device="cuda"))
        im_.append(torch.zeros(V, dtype=torch.float64, device="cuda"))
        sites += V
        names.append("%s r=%d (V=%d, Q=%d)" % (name, r, V, cfg["Q_closed"]))
    setup = time.perf_counter() - t0
    ctxs = [s4.ctx for s4 in sessions]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Qs, st = smpq.smpq_compute_qx_batch(ctxs, re_, im_)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    for s4 in sessions:
        s4.close()
    return {"value": sites / dt, "unit": "sites/s", "seconds": dt, "setup_s": setup, "lattices": names, "Q": Qs,
            "abs_Q_minus_round": [x["q_round_dev"] for x in st], "rhs": [x["n_rhs"] for x in st],
            "rounds": st[0]["n_batches"], "rhs_tile": st[0]["rhs_tile"],
            "iterations": [x["max_iterations"] for x in st], "true_resid_base": [x["true_resid"] for x in st],
            "launch": "one solve for the three lattices: each CG iteration is 3 kernel launches covering all of "
                      "them; sources in rounds sized to device memory; GPU Lanczos intervals (setup)"}


def _baselines(args, rank, dims, U, V, a, b, n_classes, dev, stream, q_out=None):
    """Comparison paths on the same GPU.  fp64_batched runs every class: its
    q(x) on the whole lattice is the FP64 reference that the other paths' q(x)
    and Q are compared with (q_out: name -> whole-lattice q(x) of the timed
    path and its variants)."""
    import torch

    from paper_1901_02211_gb300 import Session, smpq
    out = {}
    q32 = None
    if not args.no_baselines:
        # FP64 one-source-at-a-time path and FP64 batched path on a sample of classes
        sample = list(range(0, n_classes, n_classes // 2))[:2]
        if args.precision != "fp32":
            s3 = Session(device=dev, stream=stream, precision=smpq.SMPQ_FP32, tol=1e-10, rhs_block=0,
                         iters_per_check=10, use_graphs=1)
            s3.load_gauge(dims, U)
            s3.set_spectrum(a, b)
            s3.build_sources(args.rmin, MODE)
            s3.compute_qx()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            q32, Qs, st3 = s3.compute_qx()
            dt = time.perf_counter() - t0
            s3.close()
            out["fp32_reliable"] = {"value": V / dt, "unit": "sites/s", "extrapolated": False,
                                    "note": "FP32 iterations + FP64 reliable updates of the base system; the "
                                            "shifted systems keep an FP32 floor (max |dq| ~1e-7 vs the oracle)",
                                    "max_iterations": st3["max_iterations"], "reliable_updates": st3["reliable_updates"]}
        for key, blk in (("fp64_plain", 1), ("fp64_batched", 0)):
            s3 = Session(device=dev, stream=stream, precision=smpq.SMPQ_FP64, tol=1e-10, rhs_block=blk,
                         iters_per_check=10, use_graphs=1)
            s3.load_gauge(dims, U)
            s3.set_spectrum(a, b)
            s3.build_sources(args.rmin, MODE)
            cls = sample if blk == 1 else list(range(n_classes))
            s3.compute_qx(classes=cls[:1])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            q, Qs, st3 = s3.compute_qx(classes=cls)
            dt = time.perf_counter() - t0
            s3.close()
            per_class = dt / len(cls)
            full = len(cls) == n_classes
            out[key] = {"value": V / (per_class * n_classes), "unit": "sites/s", "extrapolated": not full,
                        "sample": "%d of %d classes (%d sources), %.3f s" % (len(cls), n_classes, 12 * len(cls), dt),
                        "max_iterations": st3["max_iterations"]}
            if full:
                # the whole lattice in FP64: the reference for the other paths' q(x) and Q
                out[key]["Q"] = Qs
                cmp = dict(q_out or {})
                if q32 is not None:
                    cmp["fp32_reliable"] = q32
                out[key]["vs_fp64_whole_lattice"] = {
                    name: {"max_abs_dq": float(np.abs(qq - q).max()),
                           "abs_dQ": abs(float(qq.real.sum() - q.real.sum()))} for name, qq in cmp.items()}
        # ablation of the star support: the shifted directions on every site
        # (14 full-lattice vectors per source) against the restricted path, on
        # the same sample of classes and in the same precision
        prec = {"fp32": smpq.SMPQ_FP32, "fp64": smpq.SMPQ_FP64, "mixed": smpq.SMPQ_MIXED, "fp16n": smpq.SMPQ_FP16N,
            "bf16n": smpq.SMPQ_BF16N}[args.precision]
        cls = list(range(0, n_classes, max(1, n_classes // 16)))[:16]
        res = {}
        for full in (0, 1):
            s3 = Session(device=dev, stream=stream, precision=prec, tol=1e-10, rhs_block=0, iters_per_check=10,
                         use_graphs=1, switch_residual=args.switch, full_support=full)
            s3.load_gauge(dims, U)
            s3.set_spectrum(a, b)
            s3.build_sources(args.rmin, MODE)
            s3.compute_qx(classes=cls[:1])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            q, Qs, st3 = s3.compute_qx(classes=cls)
            dt = time.perf_counter() - t0
            s3.close()
            res[full] = (V / (dt / len(cls) * n_classes), q, dt)
        colour, _ = smpq.smpq_colour_sites(dims, args.rmin, MODE)
        mask = np.isin(colour, cls)
        out["support_ablation"] = {
            "restricted": res[0][0], "full_support": res[1][0], "unit": "sites/s", "extrapolated": True,
            "sample": "%d of %d classes (%d sources), %.3f s restricted / %.3f s full" % (
                len(cls), n_classes, 12 * len(cls), res[0][2], res[1][2]),
            "max_abs_dq": float(np.abs(res[0][1][mask] - res[1][1][mask]).max())}
        if not args.no_cpu:
            oa, ob = _oracle_interval(args.config, U, dims)
            v, sites, dt, thr = cpu_oracle_sample(U, dims, oa, ob, 1, rmin=args.rmin)
            out["cpu_baseline"] = {"value": v, "unit": "sites/s", "cores": thr, "kind": "oracle",
                                   "sample": "1 of %d colour classes (12 sources, %d sites), FP64 tol 1e-10, %.1f s"
                                             % (n_classes, sites, dt)}
    return out


def _workload_name(args):
    from synth import CONFIGS
    p = CONFIGS[args.config]
    d = p["dims"]
    n_cls = (args.rmin ** 4)
    if "stout" in p:
        links = "Haar seed %d + %d stout steps rho %g" % (p["seed"], p["stout"][1], p["stout"][0])
    else:
        links = "flux Q=%d noise %g + gauge transform" % (p["k"], p["eps"])
    return ("%dx%dx%dx%d %s, SMP r_min=%d mode 0, %d classes x 12 = %d sources x 14 shifts, tol 1e-10"
            % (d[0], d[1], d[2], d[3], links, args.rmin, n_cls, 12 * n_cls))


def _report(args, ws, V, ms, value, prec, B, esz, clocks, e2e_val, U, launches, dom, kern, traffic, stats, stp,
            stt, out, sub):
    from paper_1901_02211_gb300 import smpq
    st = stats[-1]
    k = kern[dom]
    roof = {"bound": "hbm", "kernel": dom, "achieved": k["achieved"], "peak": k["peak"], "unit": "GB/s",
            "frac": k["achieved"] / k["peak"], "peak_source": k["peak_source"], "traffic": traffic,
            "traffic_over_algorithmic": None if traffic is None else traffic / k["bytes"],
            "algorithmic_per_launch": k["bytes"], "avg_launch_ms": k["ms"], "launches": k["n"],
            "timing": "CUDA events around every launch of one profiled step (graphs off), on the launch stream"}
    if "alu" in k:
        roof["alu"] = k["alu"]
    n_iter = max(1, stp["max_iterations"])
    line = {
        "metric": "q(x) sites/s", "value": value, "unit": "sites/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {smpq.SMPQ_FP32: "f32", smpq.SMPQ_FP64: "f64", smpq.SMPQ_MIXED: "f64+f32",
                                  smpq.SMPQ_FP16N: "f16+f32", smpq.SMPQ_BF16N: "bf16+f32"}[prec],
        "data": "synthetic",
        "config": {"workload": _workload_name(args),
                   "precision": {smpq.SMPQ_FP32: "FP32 dslash/vectors + FP64 reliable updates",
                                 smpq.SMPQ_FP16N: "FP16 p, t with per-site norms, reconstruct-12 links, FP32 "
                                                  "r and arithmetic, FP64 reliable updates",
                                 smpq.SMPQ_BF16N: "BF16 p, t with per-site norms, reconstruct-12 links, FP32 "
                                                  "r and arithmetic, FP64 reliable updates",
                                 smpq.SMPQ_FP64: "FP64",
                                 smpq.SMPQ_MIXED: "FP64-accurate until ||r|| < %g ||b||, then FP32 (shifted vectors too)"
                                 % args.switch}[prec],
                   "batch": B, "rhs_tile": int(st.get("rhs_tile", 0)),
                   "l2": "inputs larger than L2 (each solver vector %.1f GB)" % (V * 12 * B * esz / 1e9),
                   "graphs": "CUDA graphs, %d iterations per host check" % 10,
                   "parallelism": "replicas" if ws > 1 else "single"},
        "clocks": clocks,
        "e2e": None if e2e_val is None else {
            "value": e2e_val, "unit": "sites/s", "h2d_bytes_per_step": int(U.nbytes),
            "d2h_bytes_per_step": int(2 * V * 8 + 16)},
        "gpu_launches": int(launches),
        "launches_per_iteration": (stp["kernel_launches"] / n_iter) if n_iter else None,
        "roofline": roof,
        "roofline_all": {kk: {"bound": v["bound"], "achieved": v["achieved"], "peak": v["peak"], "unit": v["unit"],
                              "frac": v["achieved"] / v["peak"], "avg_launch_ms": v["ms"], "launches": v["n"],
                              **({"alu_frac": v["alu"]["frac"]} if "alu" in v else {})}
                         for kk, v in kern.items()},
        "solver": {"iterations": st["max_iterations"], "reliable_updates": st["reliable_updates"],
                   "max_resid": st["max_resid"], "true_resid_base": stt["true_resid"],
                   "true_resid_note": "|b - (H^2 + s0) x| / |b| of the smallest shift recomputed with FP64 "
                                      "accuracy after the solve (mixed, FP32, half: the last residual replacement; "
                                      "FP64: x accumulated in a verification step)",
                   "Q": st["Q"], "abs_Q_minus_round": st["q_round_dev"], "max_im_q": st["max_im_q"],
                   "profiled_step_ms": stp["total_ms"], "timed_step_ms": ms,
                   "kernel_ms_per_step": {kk: v["share_ms"] for kk, v in kern.items()},
                   "kernel_avg_launch_ms": {kk: v["ms"] for kk, v in kern.items()},
                   "launch_shape": {"rhs_tile": st["rhs_tile"], "tiles_per_block_hi": st["tiles_per_block_hi"],
                                    "tiles_per_block_lo": st["tiles_per_block_lo"],
                                    "cols_per_thread": st["cols_per_thread"], "staged_fp32": st["staged"]}},
    }
    if sub is not None:
        line["config"]["workload"] += " (profiling subset: first %d classes)" % len(sub)
    line.update(out)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="smpq", choices=["smpq", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp32", "fp64", "mixed", "fp16n", "bf16n"])
    ap.add_argument("--no-baselines", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-dslash", action="store_true",
                    help="skip the stand-alone D_W timing in every storage format")
    ap.add_argument("--dslash-only", action="store_true",
                    help="time only the stand-alone D_W in every storage format (no solve)")
    ap.add_argument("--dslash-columns", type=int, default=3072, help="--dslash-only: right-hand sides")
    ap.add_argument("--switch", type=float, default=1e-3, help="SMPQ_MIXED: FP64 -> FP32 switch residual")
    ap.add_argument("--config", default=CONFIG, help="synthetic configuration (synth.CONFIGS)")
    ap.add_argument("--rmin", type=int, default=R_MIN, help="SMP r (Normal mode)")
    ap.add_argument("--classes", type=int, default=0, help="profiling: only the first N colour classes")
    ap.add_argument("--low-modes", type=int, default=20,
                    help="also time the variant with this many low modes of H_W exact (0: skip)")

    ap.add_argument("--lanczos", type=int, default=300, help="Lanczos steps of the spectrum setup")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the records of the 16^3x32 and 32^3x64 configurations and of the uneven batch")
    ap.add_argument("--c5-max-iter", type=int, default=6000, help="iteration cap of the 32^3x64 record")
    ap.add_argument("--no-autotune", action="store_true",
                    help="widest RHS tile that divides the batch, without timing the candidates")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
