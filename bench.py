#!/usr/bin/env python
"""Benchmark: eeFU imaginary-time Trotter steps (and CTM sweeps) per second.

One step = one second-order Trotter step of the exact-environment full update
(five gate layers x, y, z, y, x; each builds the gated composite, runs a fixed
number of CTM sweeps, forms the metric and runs the ALS bond update) followed
by the observables (three gamma-mapped CTMRGs of the un-gated state with a
fixed number of sweeps, E/site and sublattice magnetisations read back).

Workload: Kitaev point K=1, J=0, D=4, chi=64, dbeta=0.01, seeded synthetic
start (beta=0 product state plus 5% N(0,1) noise, seed = rank).  Multi-GPU:
independent replicas per rank (weak scaling, no collective on the data path).

    python bench.py [--gpus N --steps K --warmup W --prec fp32 --impl ours|reference]
"""
import argparse
import math
import json
import os
import statistics
import tempfile
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import kh_inputs  # noqa: E402

METRIC = "CTM sweeps/s and eeFU Trotter steps/s at (D,χ); TC TFLOP/s vs peak; err vs FP64"
WORKLOAD = "kitaev_D4_chi64"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="tf32x3")
    ap.add_argument("--proj-fp64", type=int, default=1,
                    help="1 (default): the projector SVD in FP64 in the single-precision modes; 0: in FP32")
    ap.add_argument("--ctm-sweeps", type=int, default=4, help="CTM sweeps per gate layer")
    ap.add_argument("--obs-sweeps", type=int, default=2, help="CTM sweeps per mapping in the observables")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-check", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the FP64 and (D, chi) = (6, 144) lines measured after the main one")
    ap.add_argument("--e2e-steps", type=int, default=0, help="default: = --steps")
    ap.add_argument("--kernel", default="", choices=["", "tc_gemm", "site_layered"],
                    help="profiling mode: run one library kernel instead of the bench (tc_gemm on --size^3 "
                         "operands; site_layered: the layered site contraction of --D, --chi, p = 16)")
    ap.add_argument("--size", type=int, default=4096)
    ap.add_argument("--D", type=int, default=4)
    ap.add_argument("--chi", type=int, default=64)
    return ap.parse_args()


def workload():
    w = dict(kh_inputs.WORKLOADS[WORKLOAD])
    return w


def sweeps_per_step(a):
    return 5 * a.ctm_sweeps + 3 * a.obs_sweeps


# ----------------------------------------------------------------- distributed

def dist_setup(a):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        pg = dist
    return rank, world, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, x):
    if pg is None:
        return x
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.path = os.path.join(os.environ.get("KH_BENCH_CLOCKS_DIR", tempfile.gettempdir()),
                                 "bench_clocks_%d.csv" % gpu_index)
        self.idx = gpu_index

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
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
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names[1:], parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------- ours

def flush_l2(buf):
    buf.add_(1.0)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


def _peak(bound, prec, pk, pk_src):
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    if bound == "tensor":
        # kernels timed inside a long step: the sustained (power-capped) bf16 figure
        bf = pk.get("bf16_tflops_sustained", pk["bf16_tflops"])
        if prec == "bf16":
            return bf, "bf16 sustained, %s (MEASURED_PEAKS.json)" % pk_src
        return bf * 1.1 / 2.25, "tf32 = bf16 sustained %s x 1.1/2.25 nominal ratio" % pk_src
    if prec == "fp64":
        return 1.25, "nominal FP64 1.25 TFLOP/s"
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12, "FP32 CUDA-core FMA peak 152 SM x 128 x 2 x %.0f MHz" % sm_mhz


def roofline_entry(cat, c, bound, prec, pk, pk_src):
    if c["launches"] == 0 or c["ms"] <= 0:
        return None
    per_launch_flops = c["flops"] / c["launches"]
    per_launch_s = c["ms"] * 1e-3 / c["launches"]
    achieved = per_launch_flops / per_launch_s / 1e12
    peak, src = _peak(bound, prec, pk, pk_src)
    out = {"bound": bound, "kernel": cat, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
           "frac": achieved / peak, "traffic": None, "peak_source": src,
           "flops_per_launch": per_launch_flops,
           "launches": c["launches"], "avg_launch_us": per_launch_s * 1e6}
    if bound == "tensor" and prec == "tf32x3":
        out["mma_passes"] = 3      # achieved counts the 2MNK algorithmic flops once
    return out


def roofline_for(prec, prof, pk, pk_src):
    """`roofline`: the enlarged-corner step of a CTM move (the two corners
    C E E (T, T) of a move, row a3 of the hot path), the contraction the
    method spends its flops on: achieved = its algorithmic flops per move
    (2 (2 chi^3 D^2 + 2 chi^3 D^4 + 4 p chi^2 D^6), the layered count whatever
    form runs) / its average duration per move, against the tensor-core peak
    of the contraction precision (the CUDA-core peak for FP32 / FP64).
    Companion entries: the half-system product (a4), the absorption (a6), the
    layered site contraction alone (the ket-then-bra kernel inside a3 and a6,
    4 p chi^2 D^6 flops per launch) and the CholQR2 orthonormalisation of the
    projector subspace (latency-bound, against the CUDA-core peak).  `traffic` is null: these are categories of
    several launches, and no DRAM counters of the current kernels are stored
    with the benchmark."""
    tc = prec in ("tf32", "tf32x3", "bf16")
    bounds = {"corners": "tensor" if tc else "alu", "half_system_product": "tensor" if tc else "alu",
              "absorb": "tensor" if tc else "alu", "site_layer": "tensor" if tc else "alu", "cholqr_orth": "alu"}
    out = {}
    for cat, b in bounds.items():
        c = prof.get(cat)
        if c and c["flops"] > 0 and c["launches"] > 0:
            out[cat] = roofline_entry(cat, c, b, prec, pk, pk_src)
    return out


def step_flops(D, chi, sweeps, p=16):
    """Algorithmic flops of the CTM sweeps of one step by the per-move model
    F_move = 8 chi^3 D^4 + 12 p chi^2 D^6 + 2 chi^3 D^6 (4 moves per sweep)."""
    f_move = 8.0 * chi ** 3 * D ** 4 + 12.0 * p * chi ** 2 * D ** 6 + 2.0 * chi ** 3 * D ** 6
    return 4.0 * f_move * sweeps


class Workload:
    """One context of the library with the benchmark's step: a Trotter step
    (fixed CTM sweeps per layer) followed by the observables (fixed sweeps per
    mapping), on its own stream."""

    def __init__(self, g, dev, D, chi, prec, a, w, seed, proj_fp64=0, site_form=0):
        import torch
        self.g, self.dev, self.a, self.w = g, dev, a, w
        self.D, self.chi, self.prec = D, chi, prec
        self.A0, self.B0 = kh_inputs.perturbed_product_state(D, seed=seed, eps=0.05)
        self.stream = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(self.stream):
            # the library's defaults per precision (single precision: cut 1e-4 s_1,
            # two subspace iterations per move)
            self.ctx = g.Context(D, chi, prec, device=dev, stream=self.stream,
                                 proj_fp64=proj_fp64 if prec != "fp64" else 0, site_form=site_form)
            self.ctx.set_state(torch.as_tensor(self.A0, device=dev), torch.as_tensor(self.B0, device=dev))
        self.Hs = [g.bond_hamiltonian(gm, w["J"], w["K"]) for gm in "xyz"]

    def step(self):
        a, w = self.a, self.w
        self.ctx.eefu_trotter_step(w["J"], [w["K"]] * 3, w["dbeta"], ctm_max_sweeps=a.ctm_sweeps,
                                   ctm_min_sweeps=a.ctm_sweeps, ctm_tol=-1.0, info=False)
        return self.ctx.observables(self.Hs, ctm_max_sweeps=a.obs_sweeps, ctm_min_sweeps=a.obs_sweeps,
                                    ctm_tol=-1.0)

    def timed(self, steps, warmup, flush=None):
        """Warm-up, then `steps` steps each bracketed by CUDA events on the
        context's stream (L2 flushed before each, outside the events).
        Returns (total ms, last observables)."""
        import torch
        for _ in range(warmup):
            self.step()
        torch.cuda.synchronize(self.dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        last = None
        for i in range(steps):
            if flush is not None:
                with torch.cuda.stream(self.stream):
                    flush_l2(flush)
            ev[i][0].record(self.stream)
            last = self.step()
            ev[i][1].record(self.stream)
        torch.cuda.synchronize(self.dev)
        return sum(s.elapsed_time(e) for s, e in ev), last

    def close(self):
        self.ctx.close()


def site_form_name(prec, site_form, D, p=16):
    tc = prec in ("tf32", "tf32x3", "bf16")
    if site_form == 2 and D * D <= 2 * p:
        return "double-layer operand (D^2 x D^2 index formed)"
    if site_form == 0 and not tc and D * D <= 2 * p:
        return "double-layer operand (D^2 x D^2 index formed)"
    return "layered ket-then-bra, tensor cores, intermediate on chip" if tc else "layered ket-then-bra, CUDA cores"


def variant(g, dev, a, w, D, chi, prec, steps, warmup, flush, proj_fp64=0, site_form=0):
    """A second configuration measured in the same run (one replica, same
    step definition): steps/s and its CTM-sweep flop rate."""
    wl = Workload(g, dev, D, chi, prec, a, w, seed=0, proj_fp64=proj_fp64 if prec != "fp64" else 0,
                  site_form=site_form)
    ms, last = wl.timed(steps, warmup, flush)
    wl.close()
    ms_step = ms / steps
    sw = sweeps_per_step(a)
    return {"config": {"D": D, "chi": chi, "prec": prec, "projector_svd": "fp64" if (proj_fp64 or prec == "fp64")
                       else "fp32", "site_contraction": site_form_name(prec, site_form, D),
                       "J": w["J"], "K": w["K"], "dbeta": w["dbeta"],
                       "ctm_sweeps_per_layer": a.ctm_sweeps, "obs_sweeps_per_mapping": a.obs_sweeps},
            "value": 1e3 / ms_step, "unit": "steps/s", "steps": steps, "warmup": warmup, "ms_per_step": ms_step,
            "ctm_sweeps_per_s": 1e3 / ms_step * sw,
            "ctm_sweep_tflops": step_flops(D, chi, sw) / (ms_step * 1e-3) / 1e12,
            "E_site": last["E_site"] if last else None}


def batch_variant(g, dev, a, w, D, chi, prec, steps, nprob=16, proj_fp64=0):
    """Many coupling angles at once (eefu_evolve_batch): nprob problems with
    phi_i = 2 pi i / nprob (J = cos phi, K = 2 sin phi) advanced concurrently,
    each step = the benchmark's Trotter step + observables.  Timed on the host
    clock around the batch call (it returns when every problem's work has
    completed), after a one-step warm-up batch.  value = nprob x steps / time."""
    import torch
    stream = torch.cuda.current_stream(dev)
    ctxs = []
    for i in range(nprob):
        A0, B0 = kh_inputs.perturbed_product_state(D, seed=i, eps=0.05)
        c = g.Context(D, chi, prec, device=dev, stream=torch.cuda.Stream(device=dev),
                      proj_fp64=proj_fp64 if prec != "fp64" else 0)
        c.set_state(torch.as_tensor(A0, device=dev), torch.as_tensor(B0, device=dev))
        ctxs.append(c)
    phis = [2.0 * math.pi * i / nprob for i in range(nprob)]
    J = [math.cos(p) for p in phis]
    K = [[2.0 * math.sin(p)] * 3 for p in phis]
    kw = dict(ctm_max_sweeps=a.ctm_sweeps, ctm_min_sweeps=a.ctm_sweeps, ctm_tol=-1.0, obs_max_sweeps=a.obs_sweeps,
              obs_min_sweeps=a.obs_sweeps, obs_tol=-1.0)
    g.evolve_batch(ctxs, J, K, w["dbeta"], 1, 1, **kw)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    trajs = g.evolve_batch(ctxs, J, K, w["dbeta"], steps, 1, **kw)
    dt = time.perf_counter() - t0
    for c in ctxs:
        c.close()
    return {"config": {"D": D, "chi": chi, "prec": prec, "problems": nprob,
                       "couplings": "phi_i = 2 pi i / %d, J = cos phi, K = 2 sin phi" % nprob,
                       "projector_svd": "fp64" if (proj_fp64 or prec == "fp64") else "fp32",
                       "ctm_sweeps_per_layer": a.ctm_sweeps, "obs_sweeps_per_mapping": a.obs_sweeps,
                       "timing": "host clock around one eefu_evolve_batch call"},
            "value": nprob * steps / dt, "unit": "steps/s (all problems)", "steps": steps,
            "ms_per_batch_step": dt / steps * 1e3,
            "E_site_first_last": [trajs[0][-1]["E_site"], trajs[-1][-1]["E_site"]]}


def mixed_batch_variant(g, dev, a, w, prec, steps, proj_fp64=0):
    """The batched shape of many couplings at several sizes: phi in {0, 2 pi/3,
    4 pi/3} x (D, chi) in {(4, 64), (5, 100), (6, 144)}, nine problems advanced
    together by one eefu_evolve_batch call (host clock around it, after a
    one-step warm-up batch).  Reports the wall time of one batch step and the
    aggregate Trotter steps/s."""
    import torch
    sizes = [(4, 64), (5, 100), (6, 144)]
    phis = [2.0 * math.pi * i / 3 for i in range(3)]
    ctxs, J, K = [], [], []
    for D, chi in sizes:
        for i, phi in enumerate(phis):
            A0, B0 = kh_inputs.perturbed_product_state(D, seed=i, eps=0.05)
            c = g.Context(D, chi, prec, device=dev, stream=torch.cuda.Stream(device=dev),
                          proj_fp64=proj_fp64 if prec != "fp64" else 0)
            c.set_state(torch.as_tensor(A0, device=dev), torch.as_tensor(B0, device=dev))
            ctxs.append(c)
            J.append(math.cos(phi))
            K.append([2.0 * math.sin(phi)] * 3)
    kw = dict(ctm_max_sweeps=a.ctm_sweeps, ctm_min_sweeps=a.ctm_sweeps, ctm_tol=-1.0, obs_max_sweeps=a.obs_sweeps,
              obs_min_sweeps=a.obs_sweeps, obs_tol=-1.0)
    g.evolve_batch(ctxs, J, K, w["dbeta"], 1, 1, **kw)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    g.evolve_batch(ctxs, J, K, w["dbeta"], steps, 1, **kw)
    dt = time.perf_counter() - t0
    for c in ctxs:
        c.close()
    n = len(ctxs)
    return {"config": {"prec": prec, "problems": n, "sizes (D, chi)": sizes, "phi": "0, 2 pi/3, 4 pi/3 per size",
                       "projector_svd": "fp64" if (proj_fp64 or prec == "fp64") else "fp32",
                       "ctm_sweeps_per_layer": a.ctm_sweeps, "obs_sweeps_per_mapping": a.obs_sweeps,
                       "timing": "host clock around one eefu_evolve_batch call"},
            "value": n * steps / dt, "unit": "steps/s (all problems)", "steps": steps,
            "ms_per_batch_step": dt / steps * 1e3}


def run_ours(a, rank, world, local, pg):
    import torch
    import paper_1906_02220_gb300 as g

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    w = workload()
    D, chi = w["D"], w["chi"]
    wl = Workload(g, dev, D, chi, a.prec, a, w, seed=rank, proj_fp64=a.proj_fp64)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(a.warmup):
        wl.step()
    torch.cuda.synchronize(dev)
    barrier(pg)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = g.launch_count()
    wl.ctx.profile_start()
    t_ms, last = wl.timed(a.steps, 0, flush)
    prof = wl.ctx.profile_stop()
    launches = g.launch_count() - launches0
    clk = clocks.stop()
    barrier(pg)
    torch.cuda.synchronize(dev)
    t_max = max_over_ranks(pg, t_ms)
    value = a.steps * world / (t_max * 1e-3)

    # end to end through the public API with host buffers
    ne = a.e2e_steps or a.steps
    hA = torch.empty((2, 2, D, D, D), dtype=torch.float64, pin_memory=True)
    hB = torch.empty_like(hA)
    dA, dB = wl.ctx.get_state()
    hA.copy_(dA)
    hB.copy_(dB)
    torch.cuda.synchronize(dev)
    barrier(pg)
    t0 = time.perf_counter()
    for _ in range(ne):
        with torch.cuda.stream(wl.stream):
            dA.copy_(hA, non_blocking=True)
            dB.copy_(hB, non_blocking=True)
        wl.ctx.set_state(dA, dB)
        wl.step()
        dA, dB = wl.ctx.get_state()
        hA.copy_(dA)
        hB.copy_(dB)
    torch.cuda.synchronize(dev)
    te = time.perf_counter() - t0
    te = max_over_ranks(pg, te)
    state_bytes = 2 * 4 * D ** 3 * 8
    e2e = {"value": ne * world / te, "unit": "steps/s", "h2d_bytes_per_step": state_bytes,
           "d2h_bytes_per_step": state_bytes + 12 * 8}

    out = None
    if rank == 0:
        pk, pk_src = peaks()
        roofs = roofline_for(a.prec, prof, pk, pk_src)
        err = None
        if not a.no_fp64_check and a.prec != "fp64":
            err = fp64_check(a, g, dev, wl.A0, wl.B0, w, wl.Hs, last, a.warmup + a.steps)
        variants = []
        if not a.no_variants and world == 1:
            # the plain FP64 GPU form of the same workload, and the largest
            # single-precision configurations (D, chi) = (6, 144), (8, 144)
            variants.append(variant(g, dev, a, w, D, chi, "fp64", 2, 3, flush))
            variants.append(variant(g, dev, a, w, D, chi, a.prec, 3, 3, flush, proj_fp64=1 - a.proj_fp64))
            variants.append(variant(g, dev, a, w, 6, 144, a.prec, 2, 3, flush, proj_fp64=a.proj_fp64))
            # the largest bond dimension, D = 8 (n = chi D^2 = 9216), at the largest chi of the
            # one-CTA projector solvers
            variants.append(variant(g, dev, a, w, 8, 144, a.prec, 2, 3, flush, proj_fp64=a.proj_fp64))
            # the same workload with the double-layer site operand (the D^2 index formed)
            variants.append(variant(g, dev, a, w, D, chi, a.prec, 3, 3, flush, proj_fp64=a.proj_fp64, site_form=2))
            # BF16 contractions (layered site contraction on kind::f16)
            variants.append(variant(g, dev, a, w, D, chi, "bf16", 3, 3, flush, proj_fp64=a.proj_fp64))
            # sixteen coupling angles at once
            variants.append(batch_variant(g, dev, a, w, D, chi, a.prec, 3, 16, proj_fp64=a.proj_fp64))
            # three couplings at each of three sizes at once
            variants.append(mixed_batch_variant(g, dev, a, w, a.prec, 2, proj_fp64=a.proj_fp64))
        cpu = None if (a.no_cpu_baseline or world > 1) else cpu_baseline(a, w, wl.A0, wl.B0)   # N = 1 only
        sw = sweeps_per_step(a)
        try:
            # plaquette flux of the final state (Sec. V), from the z mapping's
            # observables environment; outside the timed region
            t0 = time.perf_counter()
            wv = wl.ctx.flux("z")
            flux = {"value": wv, "mapping": "z", "ms": (time.perf_counter() - t0) * 1e3,
                    "note": "state after all steps; not timed"}
        except Exception as e:                      # reported, never fatal to the bench line
            flux = {"error": str(e)}
        out = {
            "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": t_max / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "fp64": "f64"}.get(a.prec, a.prec),
            "data": "synthetic (seeded perturbed beta=0 product state)",
            "config": {"workload": WORKLOAD, "D": D, "chi": chi, "J": w["J"], "K": w["K"], "dbeta": w["dbeta"],
                       "ctm_sweeps_per_layer": a.ctm_sweeps, "obs_sweeps_per_mapping": a.obs_sweeps,
                       "prec": a.prec, "projector_svd": "fp64" if (a.proj_fp64 or a.prec == "fp64") else "fp32",
                       "site_contraction": site_form_name(a.prec, 0, D),
                       "svd_cut": wl.ctx.cfg.svd_cut, "svd_iters_warm": wl.ctx.cfg.svd_iters_warm,
                       "parallelism": "replicas x%d" % world,
                       "l2": "flushed between timed steps (256 MB write outside the timed events)"},
            "ctm_sweeps_per_s": value * sw,
            "ctm_sweep_tflops": step_flops(D, chi, sw) / (t_max / a.steps * 1e-3) / 1e12,
            "E_site": last["E_site"] if last else None,
            "err_vs_fp64": err,
            "flux_W": flux,
            "roofline": roofs.get("corners"),
            "roofline_half_system_product": roofs.get("half_system_product"),
            "roofline_absorb": roofs.get("absorb"),
            "roofline_site_layer": roofs.get("site_layer"),
            "roofline_projector_orth": roofs.get("cholqr_orth"),
            "profile": prof,
            "variants": variants,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
        }
    wl.close()
    return out


def fp64_check(a, g, dev, A0, B0, w, Hs, last, nsteps):
    """|E_site(prec) - E_site(fp64)| / max(|E|, 1) after the same steps on the
    GPU FP64 path (a consistency check of the precisions at the bench's fixed
    sweep counts; the parity of each against the CPU oracle is the test
    suite's)."""
    import torch
    D, chi = w["D"], w["chi"]
    ctx = g.Context(D, chi, "fp64", device=dev, svd_cut=1e-12)
    ctx.set_state(torch.as_tensor(A0, device=dev), torch.as_tensor(B0, device=dev))
    r = None
    for _ in range(nsteps):
        ctx.eefu_trotter_step(w["J"], [w["K"]] * 3, w["dbeta"], ctm_max_sweeps=a.ctm_sweeps,
                              ctm_min_sweeps=a.ctm_sweeps, ctm_tol=-1.0, info=False)
        r = ctx.observables(Hs, ctm_max_sweeps=a.obs_sweeps, ctm_min_sweeps=a.obs_sweeps, ctm_tol=-1.0)
    ctx.close()
    return {"E_site_fp64": r["E_site"], "rel_err": abs(last["E_site"] - r["E_site"]) / max(abs(r["E_site"]), 1.0),
            "note": "E/site after the warm-up + timed steps vs the GPU FP64 path on the same start; "
                    "the timed run's e2e steps are not included"}


# ----------------------------------------------------------------- oracle (CPU)

def oracle_layer_seconds(a, w, A0, B0):
    """Time one gate layer of the oracle (composite, ctm_sweeps CTM sweeps,
    metric, ALS, gauge) at the bench workload."""
    from oracle import eefu, model
    prm = eefu.Params(D=w["D"], chi=w["chi"], J=w["J"], K=w["K"], ctm_tol=-1.0,
                      ctm_max_sweeps=a.ctm_sweeps, ctm_min_sweeps=a.ctm_sweeps, svd_cut=1e-12)
    st = eefu.State(A0, B0, prm)
    g = prm.gate("x", w["dbeta"] / 4)
    t0 = time.perf_counter()
    eefu.apply_gate(st, "x", g)
    return time.perf_counter() - t0


def cpu_baseline(a, w, A0, B0):
    t_layer = oracle_layer_seconds(a, w, A0, B0)
    scale = 5 + 3 * a.obs_sweeps / a.ctm_sweeps
    step_s = t_layer * scale
    return {"value": 1.0 / step_s, "unit": "steps/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "one gate layer (%d CTM sweeps + metric + ALS) of the bench workload, %.1f s wall, "
                      "extrapolated x%.2f to a full step (5 layers + 3 x %d observable sweeps)"
                      % (a.ctm_sweeps, t_layer, scale, a.obs_sweeps)}


def run_reference(a, rank, world):
    if rank != 0:
        return None
    w = workload()
    A0, B0 = kh_inputs.perturbed_product_state(w["D"], seed=0, eps=0.05)
    for _ in range(a.warmup):
        oracle_layer_seconds(a, w, A0, B0)
    ts = [oracle_layer_seconds(a, w, A0, B0) for _ in range(a.steps)]
    scale = 5 + 3 * a.obs_sweeps / a.ctm_sweeps
    step_s = statistics.mean(ts) * scale
    value = 1.0 / step_s
    cpu = {"value": value, "unit": "steps/s", "cores": os.cpu_count(), "kind": "oracle",
           "sample": "per step: one gate layer (%d CTM sweeps + metric + ALS), %.1f s on average, extrapolated "
                     "x%.2f to a full step (5 layers + 3 x %d observable sweeps); ms_per_step is that "
                     "extrapolation, the wall time of each timed sample is timed_s_per_step"
                     % (a.ctm_sweeps, statistics.mean(ts), scale, a.obs_sweeps)}
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "D": w["D"], "chi": w["chi"], "J": w["J"], "K": w["K"],
                       "dbeta": w["dbeta"], "ctm_sweeps_per_layer": a.ctm_sweeps,
                       "obs_sweeps_per_mapping": a.obs_sweeps, "prec": "fp64 (CPU oracle)"},
            "cpu_baseline": cpu, "timed_s_per_step": statistics.mean(ts), "extrapolation": scale,
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_kernel(a):
    """Profiling mode: the tensor-core contraction GEMM on size^3 operands
    (inputs larger than L2), or the layered site contraction of one corner
    (chi^2 blocks of D^2 x D^2, p = 16, in --prec), timed with CUDA events; one
    JSON line.  The times include the self-test's operand preparation."""
    import torch
    import paper_1906_02220_gb300 as g
    if a.kernel == "site_layered":
        gen = torch.Generator(device="cuda:0").manual_seed(0)
        D, nb = a.D, a.chi * a.chi
        T = torch.randn((16, D, D, D, D), dtype=torch.float64, device="cuda:0", generator=gen)
        Y = torch.randn((nb, D * D, D * D), dtype=torch.float64, device="cuda:0", generator=gen)
        npass = {"tf32x3": 3, "tf32": 1, "bf16": 16}[a.prec]
        t = []
        for i in range(a.warmup + a.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.selftest_site_layered(T, Y, 0, 0, npass)
            e1.record()
            torch.cuda.synchronize()
            if i >= a.warmup:
                t.append(e0.elapsed_time(e1))
        print(json.dumps({"kernel": "site_layered", "D": D, "chi": a.chi, "p": 16, "prec": a.prec,
                          "ms_incl_preparation": min(t), "flops": 4.0 * 16 * nb * D ** 6}))
        return
    n = a.size
    gen = torch.Generator(device="cuda:0").manual_seed(0)
    A = torch.randn((n, n), dtype=torch.float64, device="cuda:0", generator=gen)
    B = torch.randn((n, n), dtype=torch.float64, device="cuda:0", generator=gen)
    for _ in range(a.warmup):
        g.selftest_gemm(A, B, a.prec)
    t = []
    for _ in range(a.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.selftest_gemm(A, B, a.prec)
        e1.record()
        torch.cuda.synchronize()
        t.append(e0.elapsed_time(e1))
    print(json.dumps({"kernel": "tc_gemm", "prec": a.prec, "size": n, "ms_incl_conversions": min(t)}))


def main():
    a = parse()
    if a.kernel:
        run_kernel(a)
        return
    rank, world, local, pg = dist_setup(a)
    if a.impl == "reference":
        out = run_reference(a, rank, world)
    else:
        out = run_ours(a, rank, world, local, pg)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
