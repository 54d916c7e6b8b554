#!/usr/bin/env python
"""Benchmark: FWI fwd+adj grid-point updates per second on one GB300.

One step is one pass of the whole hot path over one batch: supergather
encoding of every posterior sample (host), the encoded misfit and velocity
gradient of every sample over all its supergathers (forward, residual,
adjoint, imaging; fwi_gradient), a preconditioned Langevin refinement step
(langevin_step_precond) and a DDPM re-noise draw (renoise).

The headline workload is the largest one, the 3D layered volume:
256 x 256 x 128 nodes at 20 m, 20-cell sponge (296 x 296 x 168 padded,
14.7 M points), 64 sources as 4 +-1-encoded supergathers of 16, 64 x 64
receivers, 5 Hz Ricker, dt 1.5 ms, 1500 steps, 8 posterior samples, FP32
wavefields with checkpointing.  The 2D thrust-belt batch (801 x 187 at 25 m,
100 sources, 400 receivers, 2000 steps, 16 samples x 5 supergathers of 20)
is timed as an extra, and so is the posterior-samples-per-hour comparison at
equal model RMSE on the thrust-belt geometry.

Metric: useful updates 2 x padded points x nt x wavefields per step / time.
Inputs (0.5 GB of wavefields per 3D time step, hundreds of GB of snapshots
per step) are far larger than L2, so no flush is needed between steps.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (the baseline arm; it is not a GPU implementation).
"""
import argparse
import json
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

WORKLOAD = "layered3d"
METRIC = "FWI fwd+adj Gpt/s (encoded gradient, grid-point updates/s)"
UNIT = "Gpt/s"
ORACLE_NT_3D = 40   # steps of the bounded 3D oracle sample (rate per step is what is reported)


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, timeout=10.0):
        """Blocks until nvidia-smi has printed its first sample: its start-up
        holds the driver for up to seconds, which must not fall inside the
        timed region."""
        t0 = time.time()
        while self.proc is not None and not self.lines and time.time() - t0 < timeout:
            time.sleep(0.05)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(value, dist=None, device="cpu"):
    """Largest per-rank value (the slowest replica's time); plain value on one rank."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, ms_max):
    """Whole-job rate: every replica's units over the slowest replica's time."""
    return units_per_rank * world / (ms_max * 1e-3)


def bytes_per_update(nsg, ndim=2, fwd_pair=False, adj_pair=False):
    """Algorithmic HBM bytes per wavefield grid-point update of each step kernel.

    2D forward: read p^n, p^{n-1}, write p^{n+1} (12 B) + cc shared by the nsg
    supergathers of a sample (4/nsg B).  2D adjoint: read q^{k+1}, q^{k+2},
    p^{k-1}, write q^k (16 B) + cc and the imaging accumulator read+write
    shared by the supergathers (12/nsg B).  3D kernels with one wavefield per
    CTA: forward 16 B, adjoint 16 B + cc 4 B + accumulator read+write 8 B;
    with pair tiles (two supergathers per CTA) cc and the accumulator are
    shared by the pair: forward 12 + 4/2 B, adjoint 16 + 12/2 B.
    """
    if ndim == 3:
        return {"forward": 14.0 if fwd_pair else 16.0, "adjoint": 22.0 if adj_pair else 28.0}
    return {"forward": 12.0 + 4.0 / nsg, "adjoint": 16.0 + 12.0 / nsg}


def oracle_sample(w, nsg_sample, seed, nt=None):
    """FP64 oracle gradient for one sample over nsg_sample supergathers, on the
    first nt steps (all when None).  Returns (Gpt/s, seconds, workload run)."""
    import oracle as O
    wr = synth.WORKLOADS[w.name](nt=nt) if nt else w
    g = O.Grid.from_workload(wr)
    v = synth.initial_model(wr)
    d = synth.random_records(wr, seed, nshots=wr.ns)
    perm, wt = O.encode(seed, 0, wr.ns)
    sg = wr.sg_sizes[:nsg_sample]
    t = time.perf_counter()
    O.gradient(g, v, wr.src, wr.rec, d, perm, wt, sg, 1.0, scale=1.0)
    dt = time.perf_counter() - t
    return 2.0 * wr.padded_points * wr.nt * nsg_sample / dt / 1e9, dt, wr


def oracle_threads():
    """Threads the oracle's OpenMP loops use."""
    import oracle as O
    return O.threads()


def _oracle_sample_plan(w):
    """(supergathers, steps, description) of the bounded oracle sample of w."""
    if w.ndim == 3:
        return 1, ORACLE_NT_3D, ("%s: 1 sample x 1 supergather of %d shots, first %d of %d steps, fwd+adj+imaging, "
                                 "FP64; the rate per step is extrapolated to the full run"
                                 % (w.name, w.sg_sizes[0], ORACLE_NT_3D, w.nt))
    return 1, None, ("%s: 1 sample x 1 supergather of %d shots, full %d steps, fwd+adj+imaging, FP64"
                     % (w.name, w.sg_sizes[0], w.nt))


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = synth.WORKLOADS[args.workload]()
    nsg_sample, nt, sample = _oracle_sample_plan(w)
    for _ in range(args.warmup):
        oracle_sample(w, nsg_sample, 1, nt)
    vals, times = [], []
    for k in range(args.steps):
        v, dt, _ = oracle_sample(w, nsg_sample, 2 + k, nt)
        vals.append(v)
        times.append(dt)
    val = float(np.mean(vals))
    out = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": w.name, "sample": sample},
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle", "sample": sample},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def kernel_source_hash(src_name, root=None):
    """sha256 of a CUDA source with its comments and blank lines removed: the
    key of an ncu figure taken on that source, unchanged by edits to comments."""
    import hashlib
    import re
    src = open(os.path.join(root or ROOT, "paper_2512_12797_gb300", "csrc", src_name)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    code = "\n".join(line.rstrip() for line in src.splitlines() if line.strip())
    return hashlib.sha256(code.encode()).hexdigest()


def committed_traffic(kernel_name, ndim):
    """DRAM bytes per wavefield point update of the named step kernel from the
    committed ncu summary, if it was taken on the current kernel code (else None)."""
    import re
    src_name = "stencil3d.cu" if ndim == 3 else "stencil.cu"
    prof = "step3d_layered3d_traffic.md" if ndim == 3 else "step2d_thrust2d_traffic.md"
    try:
        key = kernel_source_hash(src_name)
        txt = open(os.path.join(ROOT, "profiles", prof)).read()
    except OSError:
        return None
    m = re.search(r"traffic-key %s code-sha256=([0-9a-f]+) forward_bytes_per_update=([0-9.]+) "
                  r"adjoint_bytes_per_update=([0-9.]+)" % re.escape(src_name), txt)
    if not m or m.group(1) != key:
        return None
    return float(m.group(3) if "ADJ" in kernel_name else m.group(2))


def gradient_run(P, torch, w, steps, warmup, e2e_steps, dist, dev, world, rank, local, budget=0, variants="",
                 clocks=True):
    """Times `steps` full hot-path steps of workload w on device-resident inputs
    (with per-phase events of the library), then `e2e_steps` through the public
    API with host buffers.  Returns the pieces of the JSON line."""
    nsamp, sg = w.nsamp, w.sg_sizes
    nsg = len(sg)
    B = nsamp * nsg
    ctx = P.FWI(w.grid_dict(), w.src, w.rec, B, budget)
    if variants:
        ctx.set_variants(*[int(x) for x in variants.split(",")])

    vel0 = synth.sample_models(w, nsamp, seed=100 + rank)
    d_obs_h = synth.random_records(w, 200 + rank)
    vel = torch.tensor(vel0, device=dev)
    d_obs = torch.tensor(d_obs_h, device=dev)
    xt = torch.zeros_like(vel)
    xprev = torch.zeros_like(vel)
    grad = torch.empty_like(vel)
    mom = torch.zeros_like(vel)
    misfit = torch.empty(nsamp, dtype=torch.float64, device=dev)
    sigma, eta = 1.0, 10.0
    beta = np.linspace(1e-4, 0.02, 1000)
    abar = np.cumprod(1 - beta)
    tlev = 300

    def encodings(it):
        e = [P.encode(1234 + s, it, w.ns) for s in range(nsamp)]
        return np.stack([a for a, _ in e]), np.stack([b for _, b in e])

    def step(it, vel_d, dobs_d):
        perm, wt = encodings(it)
        ctx.gradient(vel_d, perm, wt, sg, dobs_d, sigma, grad=grad, misfit=misfit)
        ctx.langevin_precond(vel_d, grad, mom, it + 1, eta, (2 * eta) ** 0.5, w.vmin, w.vmax, 77, it, eps=0.1)
        P.renoise(xt, vel_d, abar[tlev - 1], abar[tlev - 2], beta[tlev - 1], 78, it, out=xprev)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
            torch.cuda.synchronize()

    def timed(fn, nsteps, it0, sampler=None):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if sampler:
            sampler.start()
            sampler.wait_first()
        barrier()
        ev0.record()
        for k in range(nsteps):
            fn(it0 + k)
        ev1.record()
        barrier()
        clk = sampler.stop() if sampler else None
        ms = max_over_ranks(ev0.elapsed_time(ev1) / nsteps, dist, dev)
        return ms, clk

    for k in range(warmup):
        step(k, vel, d_obs)
    torch.cuda.synchronize()

    # device-resident timed region, with per-phase events of the library
    ctx.set_profiling(True)
    phase_ms = np.zeros(4)
    phase_launch = np.zeros(4, np.int64)

    def step_prof(it):
        step(it, vel, d_obs)
        ms_, ln = ctx.phase_times()   # synchronises on the last phase event
        phase_ms[:] += ms_
        phase_launch[:] += ln

    ms, clk = timed(step_prof, steps, 1000, ClockSampler(local) if clocks else None)
    ctx.set_profiling(False)
    plan = ctx.plan_info()
    var = ctx.variants()
    units = 2.0 * w.padded_points * w.nt * B
    value = job_throughput(units, world, ms) / 1e9

    # end to end through the public API with host buffers
    vel_h = torch.tensor(vel0).pin_memory()
    dobs_h = torch.tensor(d_obs_h).pin_memory()
    out_h = torch.empty_like(vel_h).pin_memory()
    mis_h = torch.empty(nsamp, dtype=torch.float64).pin_memory()
    # Double-buffered: step k+1's inputs are copied on a copy stream while step
    # k computes (they do not depend on its results); every step still copies
    # its own inputs and reads back its own result inside the timed region.
    vel_e = [torch.empty_like(vel) for _ in range(2)]
    dobs_e = [torch.empty_like(d_obs) for _ in range(2)]
    cstream = torch.cuda.Stream()
    ready = [torch.cuda.Event() for _ in range(2)]
    free = [torch.cuda.Event() for _ in range(2)]
    rng = {}

    def prefetch(it):
        b = it % 2
        cstream.wait_event(free[b])  # the step that used buffer b is done with it
        with torch.cuda.stream(cstream):
            vel_e[b].copy_(vel_h, non_blocking=True)
            dobs_e[b].copy_(dobs_h, non_blocking=True)
        ready[b].record(cstream)

    def step_e2e(it):
        b = it % 2
        if it == rng["first"]:
            prefetch(it)
        torch.cuda.current_stream().wait_event(ready[b])
        if it + 1 < rng["end"]:
            prefetch(it + 1)
        step(it, vel_e[b], dobs_e[b])
        out_h.copy_(vel_e[b], non_blocking=True)
        mis_h.copy_(misfit, non_blocking=True)
        free[b].record()

    rng.update(first=0, end=1)
    step_e2e(0)
    torch.cuda.synchronize()
    rng.update(first=2000, end=2000 + e2e_steps)
    ms_e2e, _ = timed(step_e2e, e2e_steps, 2000)
    e2e_value = job_throughput(units, world, ms_e2e) / 1e9
    h2d = vel_h.numel() * 4 + dobs_h.numel() * 4
    d2h = out_h.numel() * 4 + nsamp * 8

    # roofline of the dominant step kernel from the per-phase events.  A
    # multi-step launch (2D; the persistent 3D variants) runs all steps of a
    # phase (forward: nt steps; adjoint: the steps of a checkpoint segment),
    # otherwise every step is a launch; both are charged per step.
    bpu = bytes_per_update(nsg, w.ndim, "pairs" in var["forward_name"], "pairs" in var["adjoint_name"])
    nchunks = (nsamp + plan["samples_per_chunk"] - 1) // plan["samples_per_chunk"]
    fwd_steps = w.nt * nchunks * steps
    rec_steps = plan["recomputed_steps"] * nchunks * steps
    fwd_step_ms = phase_ms[0] / max(fwd_steps, 1)  # phase 0 also holds one expand launch per chunk
    # the adjoint phase also holds the recomputed forward steps: charge them the
    # forward steps' average time
    adj_only_ms = phase_ms[2] - rec_steps * fwd_step_ms
    adj_step_ms = adj_only_ms / max(w.nt * nchunks * steps, 1)
    per_step_pts = w.padded_points * plan["samples_per_chunk"] * nsg  # wavefield points of one step launch
    kd = "3d" if w.ndim == 3 else "2d"
    kern = {
        "step%s_kernel<ADJ>" % kd: {"ms": adj_step_ms, "bytes": bpu["adjoint"] * per_step_pts,
                                    "share": adj_only_ms / max(phase_ms.sum(), 1e-9)},
        "step%s_kernel<FWD>" % kd: {"ms": fwd_step_ms, "bytes": bpu["forward"] * per_step_pts,
                                    "share": (phase_ms[0] + phase_ms[2] - adj_only_ms) / max(phase_ms.sum(), 1e-9)},
    }
    # both step kernels together: algorithmic bytes of all their launches over
    # their total time (forward launches: first pass and recomputation)
    n_f, n_a = fwd_steps + rec_steps, w.nt * nchunks * steps
    kf, ka = kern["step%s_kernel<FWD>" % kd], kern["step%s_kernel<ADJ>" % kd]
    comb_gbs = (kf["bytes"] * n_f + ka["bytes"] * n_a) / ((kf["ms"] * n_f + ka["ms"] * n_a) * 1e-3) / 1e9
    combined = {"achieved": comb_gbs, "unit": "GB/s", "launch_steps": {"forward": n_f, "adjoint": n_a}}
    dom = max(kern, key=lambda k: kern[k]["share"])
    other = [k for k in kern if k != dom][0]
    peaks = _peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    achieved = kern[dom]["bytes"] / (kern[dom]["ms"] * 1e-3) / 1e9
    combined["frac"] = comb_gbs / peak
    other_gbs = kern[other]["bytes"] / (kern[other]["ms"] * 1e-3) / 1e9
    tpu = committed_traffic(dom, w.ndim)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": tpu * per_step_pts if tpu is not None else None,
                "traffic_unit": "bytes per launch (dram read + write per point update from ncu, profiles/%s, "
                                "x the launch's point updates)" % ("step3d_layered3d_traffic.md" if w.ndim == 3
                                                                   else "step2d_thrust2d_traffic.md"),
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy)" if peaks else "fallback",
                "bytes_per_update": bpu["adjoint" if "ADJ" in dom else "forward"],
                "point_updates_per_step": per_step_pts,
                "avg_step_ms": kern[dom]["ms"],
                "share_of_step": kern[dom]["share"],
                "steps_per_launch": {
                    "forward": w.nt if w.ndim == 2 or "multi-step" in var["forward_name"] else 1,
                    "adjoint": (min(plan["segment_len"], w.nt)
                                if w.ndim == 2 or "multi-step" in var["adjoint_name"] else 1)},
                "other_kernel": {"name": other, "achieved": other_gbs, "frac": other_gbs / peak,
                                 "avg_step_ms": kern[other]["ms"], "share_of_step": kern[other]["share"]},
                "both_step_kernels": combined}
    res = {"value": value, "ms": ms, "clocks": clk, "units": units, "plan": plan, "variants": var,
           "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                   "ms_per_step": ms_e2e, "steps": e2e_steps,
                   "overlap": "double-buffered inputs: step k+1's H2D on a copy stream during step k"},
           # library launches counted per phase, plus the two refinement-step
           # kernels and the re-noise kernel of every step
           "gpu_launches": int(phase_launch.sum() + steps * 3),
           "roofline": roofline,
           "phase_ms_per_step": {"forward": phase_ms[0] / steps, "residual": phase_ms[1] / steps,
                                 "adjoint": phase_ms[2] / steps, "finalize": phase_ms[3] / steps}}
    ctx.close()
    del vel_e, dobs_e, vel, d_obs
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return res


def sampler_at_equal_rmse(P, torch, dev, full_steps=6, max_enc_steps=120):
    """Posterior samples/hour at equal model RMSE (Sec. 2.4, eq. pde-count; the
    encoded sampler against plain full-shot Langevin) on the thrust-belt
    geometry: 4 posterior samples, observed data from the forward on the
    seeded truth plus 1 % Gaussian noise.  The full-shot chain (every shot
    its own solve) runs full_steps preconditioned Langevin steps; its final
    posterior-mean RMSE is the target; the encoded chain (5 supergathers of
    20, redrawn every step) runs until it reaches that RMSE."""
    from paper_2512_12797_gb300 import sampler as S
    w = synth.thrust2d()
    nsamp = 4
    ctx = P.FWI(w.grid_dict(), w.src, w.rec, nsamp * w.ns, 0)
    truth = torch.tensor(synth.true_model(w), device=dev)
    v0 = torch.tensor(synth.sample_models(w, nsamp, seed=7), device=dev)
    ident = np.arange(w.ns, dtype=np.int32)
    d_clean = ctx.forward(truth[None].contiguous(), ident, np.ones(w.ns, np.int8), [1] * w.ns)[0]
    gen = torch.Generator(device=dev).manual_seed(4)
    noise = 0.01 * float(d_clean.pow(2).mean().sqrt())
    d_obs = (d_clean + noise * torch.randn(d_clean.shape, device=dev, generator=gen)).contiguous()
    kw = dict(eta=15.0, vmin=w.vmin, vmax=w.vmax, sigma=noise, seed=3)
    # untimed first calls (autotuner, plans) of both shapes
    S.plain_langevin(ctx, v0, d_obs, truth, steps=1, **kw)
    S.plain_langevin(ctx, v0, d_obs, truth, steps=1, sg_sizes=w.sg_sizes, **kw)
    full = S.plain_langevin(ctx, v0, d_obs, truth, steps=full_steps, **kw)
    target = full["rmse"][-1]
    enc = S.plain_langevin(ctx, v0, d_obs, truth, steps=max_enc_steps, sg_sizes=w.sg_sizes, rmse_target=target, **kw)
    ctx.close()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()

    def arm(solves, seconds, steps, per_step):
        return {"solves_to_target": solves, "seconds_to_target": seconds, "steps_to_target": steps,
                "pde_solves_per_step_per_sample": per_step,
                "samples_per_hour_at_target": nsamp * 3600.0 / seconds if seconds else None}

    out = {"workload": "thrust2d geometry, %d posterior samples, 1 %% noise, preconditioned Langevin with matched "
                       "noise (eta 15 m/s)" % nsamp,
           "rmse_initial": full["rmse"][0], "rmse_target": target,
           "plain_langevin_full_shot": arm(full["solves"][-1], full["seconds"], full_steps, 2 * w.ns),
           "encoded": None, "samples_per_hour_ratio": None, "solve_ratio": None}
    if enc["reached"] is not None:
        r = enc["reached"]
        out["encoded"] = arm(r["solves"], r["seconds"], r["steps"], 2 * len(w.sg_sizes))
        out["samples_per_hour_ratio"] = (out["encoded"]["samples_per_hour_at_target"] /
                                         out["plain_langevin_full_shot"]["samples_per_hour_at_target"])
        out["solve_ratio"] = full["solves"][-1] / r["solves"]
    else:
        out["encoded_final_rmse"] = enc["rmse"][-1]
        out["encoded_steps_run"] = max_enc_steps
    return out


def prior_measurement(w, nsamp, ms_iter, peaks):
    """The learned prior's x0-hat prediction on this batch's models, on the
    tcgen05 kernels: time per call, the convolutions' algorithmic TFLOP/s
    (real input channels, not the zero-padded ones) against the measured BF16
    peak, and its cost next to one encoded Langevin iteration.  (Random
    weights: the arithmetic does not depend on them.)"""
    import torch
    from paper_2512_12797_gb300 import unet
    den = unet.UNetDenoiser(unet.init_params(0, out_scale=1.0))
    Hp, Wp = unet.tile_shape(w.nz, w.nx)
    flops = 0.0
    for name, cin, cout in unet.LAYERS:
        lev = {"e1": 0, "e2": 1, "ba": 2, "bb": 2, "d2": 1, "d1": 0}[name[:2]]
        flops += 2.0 * (Hp >> lev) * (Wp >> lev) * 9 * cin * cout
    flops = (flops + 2.0 * Hp * Wp * 64 * 32) * nsamp
    x_t = torch.randn((nsamp, w.nz, w.nx), device="cuda")
    for _ in range(3):
        den(x_t, 0.5)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    reps = 10
    for _ in range(reps):
        den(x_t, 0.5)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    peak = peaks["bf16_tflops"] if peaks else 1900.0
    return {"network": "U-Net 64/128/256, 3x3 convs on tcgen05 (BF16, FP32 accumulation)",
            "input": [nsamp, w.nz, w.nx], "padded": [Hp, Wp], "ms_per_call": ms,
            "conv_tflops": flops / (ms * 1e-3) / 1e12, "bf16_peak_tflops": peak,
            "frac_of_peak": flops / (ms * 1e-3) / 1e12 / peak,
            "share_of_langevin_iteration": ms / ms_iter,
            "note": "whole call incl. padding, pooling, upsampling and concatenation; FLOPs of the real channels"}


def native_arm(args):
    import torch
    import paper_2512_12797_gb300 as P

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    w = synth.WORKLOADS[args.workload](**({"nt": args.nt} if args.nt else {}))
    if args.samples:
        w.nsamp = args.samples
    budget = int(args.budget_gb * (1 << 30)) if args.budget_gb else 0
    e2e_steps = args.e2e_steps or (args.steps if w.ndim == 2 else max(3, args.steps // 4))
    r = gradient_run(P, torch, w, args.steps, args.warmup, e2e_steps, dist, dev, world, rank, local, budget,
                     args.variants)
    nsg = len(w.sg_sizes)
    B = w.nsamp * nsg
    peaks = _peaks()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        nsg_s, nt_s, sample = _oracle_sample_plan(w)
        cval, cdt, _ = oracle_sample(w, nsg_s, 3, nt_s)
        nthr = O.threads()
        # the same oracle on one thread, over a shorter run (the rate per step
        # does not depend on the number of steps)
        O.threads(1)
        try:
            sval, sdt, w1 = oracle_sample(w, 1, 4, min(w.nt, 500 if w.ndim == 2 else 8))
        finally:
            O.threads(nthr)
        cpu = {"value": cval, "unit": UNIT, "cores": nthr, "kind": "oracle", "sample": sample + " (%.1f s)" % cdt,
               "single_thread": {"value": sval, "unit": UNIT, "cores": 1,
                                 "sample": "%s: 1 sample x 1 supergather of %d shots, first %d steps (%.1f s)"
                                           % (w.name, w1.sg_sizes[0], w1.nt, sdt)}}

    out = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": r["ms"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded %s models, random records)" % w.name,
           "config": {"workload": w.name, "grid": list(w.shape), "h_m": w.hx, "nb": w.nb, "nt": w.nt,
                      "sources": w.ns, "receivers": w.nr, "samples": w.nsamp, "supergathers": w.sg_sizes,
                      "wavefields": B, "padded_points": w.padded_points,
                      "parallelism": "replicas" if world > 1 else "single-gpu",
                      "l2": "inputs larger than L2 (no flush)",
                      "checkpoint_plan": r["plan"],
                      "step_kernels": {"forward": r["variants"]["forward_name"],
                                       "adjoint": r["variants"]["adjoint_name"],
                                       "forward_index": r["variants"]["forward"],
                                       "adjoint_index": r["variants"]["adjoint"],
                                       "tuner_ms_forward": r["variants"]["forward_ms"],
                                       "tuner_ms_adjoint": r["variants"]["adjoint_ms"]}},
           "e2e": r["e2e"], "gpu_launches": r["gpu_launches"], "roofline": r["roofline"],
           "phase_ms_per_step": r["phase_ms_per_step"], "clocks": r["clocks"], "cpu_baseline": cpu}

    if world == 1 and args.extras and w.name != "thrust2d" and not args.nt and not args.samples:
        # the 2D thrust-belt batch: its own line's figures, fewer steps
        w2 = synth.thrust2d()
        r2 = gradient_run(P, torch, w2, args.extra_steps, 2, args.extra_steps, None, dev, 1, 0, local, clocks=False)
        out["thrust2d"] = {"value": r2["value"], "unit": UNIT, "ms_per_step": r2["ms"], "steps": args.extra_steps,
                           "config": {"grid": list(w2.shape), "nt": w2.nt, "samples": w2.nsamp,
                                      "supergathers": w2.sg_sizes, "plan": r2["plan"]},
                           "e2e": r2["e2e"], "roofline": r2["roofline"], "phase_ms_per_step": r2["phase_ms_per_step"],
                           "gpu_launches": r2["gpu_launches"]}
        ms2 = r2["ms"]
    else:
        w2, ms2 = (w, r["ms"]) if w.ndim == 2 else (None, None)
    if world == 1 and args.sampler:
        out["sampler"] = sampler_at_equal_rmse(P, torch, dev)
    if world == 1 and args.prior and w2 is not None:
        out["prior"] = prior_measurement(w2, w2.nsamp, ms2, peaks)
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(synth.WORKLOADS))
    ap.add_argument("--budget-gb", type=float, default=0.0, help="wavefield pool (0: most of free memory)")
    ap.add_argument("--e2e-steps", type=int, default=0, help="steps of the end-to-end timing (0: automatic)")
    ap.add_argument("--extras", type=int, default=1, help="also time the 2D thrust-belt batch")
    ap.add_argument("--extra-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sampler", type=int, default=1, help="also measure posterior samples/hr at equal RMSE")
    ap.add_argument("--prior", type=int, default=1, help="also time the learned prior's x0-hat prediction")
    ap.add_argument("--samples", type=int, default=0, help="override posterior samples (profiling runs)")
    ap.add_argument("--nt", type=int, default=0, help="override time steps (profiling runs)")
    ap.add_argument("--variants", default="", help="force step-kernel variants 'fwd,adj' (default: autotune)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    return native_arm(args)


if __name__ == "__main__":
    sys.exit(main())
