"""Benchmark of the WPCD hot path on one GB300 (or N, sharded by sample).

Headline workload: 16384 parameter samples x 20 channels J <= 6 (6 coupled),
N_WP = 150 (coupled blocks 300 x 300), 128 lab energies 1..350 MeV, mixed
precision (FP32 Jacobi + FP64 eigenpair refinement; resolvent, T and phases in
FP64), the seeded synthetic regulated Yukawa + contact potential.  One step =
the whole hot path over that batch: parameter sum + eigensolve of every
(sample, channel), energy plan, SWP boundaries + resolvent + T at the needed
bins, T at every requested energy, phase interpolation and the np total cross
section.

The same JSON line carries, beside the device-resident throughput: the same
step end to end through wpcd_solve_host (host buffers, copies timed), the
dominant kernel's roofline, the plain (one eigensolve per launch) and batched
FP64 paths on the same GPU, the mixed path's error against the FP64 path and
against the CPU oracle on a seeded subset, the 4096-sample x 15-channel
batched workload (FP64 eigensolve as specified, and mixed), the MI comparison
method, spin observables, a served Poisson request stream with N_WP in
{32, 64, 128, 256} (latency, the FP64 per-request latency, a saturation
sweep), and the oracle's CPU throughput.

``--impl reference`` times the FP64 CPU oracle on the host cores instead, on a
bounded sample of the headline workload per step.
"""
from __future__ import annotations

import argparse
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

from paper_2106_00454_gb300 import inputs as W  # noqa: E402

METRIC = "channel-solves/s and p50/p99 latency at <=1e-3 deg phase error vs plain FP64"
UNIT = "channel-solves/s"
# GB300 FP64 and FP32 rates: not in the measured-peaks file (it holds the HBM copy
# rate and cuBLAS bf16), so both are this project's own figures, labelled as such
FP64_PEAK_TFLOPS = 1.25
FP64_PEAK_NOTE = ("builder-derived: nominal GB300 FP64 rate (2 DFMA per clock per SM); "
                  "our DFMA probe measured 1.19 TFLOP/s")
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP32_PEAK_NOTE = ("builder-derived: 152 SM x 128 FP32 lanes x 2 flop x 2.07 GHz; "
                  "our FFMA probe measured 69-70 TFLOP/s")
L2_FLUSH_BYTES = 512 << 20   # > 129 MB L2
# k_jacobi_mixed DRAM bytes (read + write) per solve per matrix element inside the headline
# step, from the ncu capture of the workload's first 128 samples (profiles/
# traffic_mixed_20ch_nwp150_128samples.md: 1.460 GB + 2.602 GB per solve pass over
# 128 x (6 x 300^2 + 14 x 150^2) elements, L2 flushed between passes as in the timed steps):
# the FP64 H and eigenvectors handed to the refinement (16 B an element), the potential
# terms re-read after the flush and eigenvector columns evicted from the L2; it scales
# with the samples and with n^2
JACOBI_MIXED_DRAM_BYTES_PER_N2 = (1459650764.8 + 2601650176.0) / (128 * (6 * 300 * 300 + 14 * 150 * 150))
# the refinement phase's kernels (digit splits, tcgen05 digit products, update, sort), same
# capture: 39.52 GB + 22.56 GB per solve pass, against the algorithmic 24 B an element (H and
# X read, X written, FP64)
REFINE_DRAM_BYTES_PER_N2 = (39518831616.0 + 22560583270.4) / (128 * (6 * 300 * 300 + 14 * 150 * 150))
SAT_P99_BOUND_MS = 250.0     # the saturation sweep's latency bound
SERVE_MAX_QUEUE = 4096       # requests waiting at most (the server refuses beyond)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="wpcd", choices=["wpcd", "reference"])
    ap.add_argument("--workload", default="config4", choices=["config4", "config3"],
                    help="config4: 16384 x 20 ch, N_WP 150 (the headline); config3: 4096 x 15 ch, N_WP 40/64/100")
    ap.add_argument("--samples", type=int, default=0, help="samples per step (0: the workload's own)")
    ap.add_argument("--exec", default="batched", choices=["batched", "plain"])
    ap.add_argument("--prec", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--graphs", default="on", choices=["on", "off"],
                    help="replay repeated solves from CUDA graphs (off: kernel by kernel, e.g. for ncu launch lists)")
    ap.add_argument("--prof-steps", type=int, default=2, help="steps re-run kernel by kernel for per-kernel times")
    ap.add_argument("--check-samples", type=int, default=16,
                    help="samples re-solved by the FP64 path on the GPU to state the mixed path's error")
    ap.add_argument("--oracle-samples", type=int, default=2,
                    help="samples solved by the CPU oracle for the per-result error of both GPU paths")
    ap.add_argument("--fp64-batched-samples", type=int, default=64, help="slice for the batched FP64 baseline")
    ap.add_argument("--fp64-plain-samples", type=int, default=1, help="slice for the plain FP64 baseline")
    ap.add_argument("--sweep-samples", type=int, default=256, help="slice whose sweep counts give the executed work")
    ap.add_argument("--cpu-samples", type=int, default=4, help="oracle sample size for the CPU baseline")
    ap.add_argument("--ref-samples", type=int, default=2, help="oracle samples per step of --impl reference")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--one-iter-leg", type=int, default=1, help="time the opt-in single refinement iteration")
    ap.add_argument("--secondary", default="on", choices=["on", "off"],
                    help="the 4096 x 15-channel batched workload, MI comparison and spin observables")
    ap.add_argument("--serve-seconds", type=float, default=30.0,
                    help="length of the Poisson request stream for the latency figures (0 = skip serving)")
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-nwp", default="32,64,128,256")
    ap.add_argument("--sat-rates", default="250,500,1000,1500", help="saturation sweep: offered rates (req/s)")
    ap.add_argument("--sat-seconds", type=float, default=4.0)
    ap.add_argument("--mi-interp", type=int, default=32,
                    help="MI comparison method: interpolation energies (0 = skip the MI leg)")
    ap.add_argument("--mi-quad", type=int, default=96, help="MI momentum grid points per l-block")
    ap.add_argument("--mi-samples", type=int, default=1024, help="slice of the 4096-sample workload for MI")
    ap.add_argument("--angles", type=int, default=32,
                    help="spin observables (Saclay amplitudes, dsigma/dOmega) at this many angles (0 = skip)")
    return ap.parse_args()


def dist_init(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    lrank = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "wpcd" else "gloo"
        dist.init_process_group(backend)
    return ws, rank, lrank


def headline_workload(name, samples=0, sample_seed=None):
    if name == "config3":
        return W.workload_batched(n_samples=samples or 4096, sample_seed=sample_seed)
    return W.workload_mixed(n_samples=samples or 16384, sample_seed=sample_seed)


def rank_workload(samples, rank, workload="config4"):
    """This rank's shard of a weak-scaling job: the same channels, meshes and
    energies on every rank, its own block of parameter samples (rank 0's are
    the single-GPU workload's)."""
    return headline_workload(workload, samples, None if rank == 0 else W.SEED + 7919 * rank)


def workload_label(wl):
    if wl.name.startswith("batched_"):
        return f"{wl.name}_nwp40-64-100_{len(wl.e_lab)}E"
    return f"{wl.name}_{len(wl.e_lab)}E"


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, x, device=None):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        loaded = [x for x in sm if x > 0.5 * smax] or sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows)}


def measured_peak(key, fallback):
    """A peak from the measured-peaks file at the repo root, else the stated fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key]), f"measured ({key})"
    except (OSError, KeyError, ValueError):
        return fallback, "fallback"


def host_cpu():
    """The host CPU as /proc/cpuinfo names it, with the machine type and logical CPU count."""
    import platform
    name = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key, _, val = line.partition(":")
                key = key.strip().lower()
                if key in ("model name", "cpu model", "hardware") and val.strip():
                    name = val.strip()
                    break
                if key == "cpu part" and not name:  # Arm: the part number (0xd4f = Neoverse V2)
                    name = "Arm part " + val.strip()
    except OSError:
        pass
    return f"{name or platform.processor() or 'unknown'} ({platform.machine()}, {os.cpu_count()} logical CPUs)"


def oracle_solve(wl, idx):
    """The FP64 oracle on samples idx of the workload: (t, delta, sigma, seconds)."""
    import oracle
    oracle.build()
    meshes = [oracle.Mesh(n) for n in wl.nwp]
    Vts = [oracle.project_channel(m, ch.astuple(), wl.gen, wl.gen_params, wl.n_terms) for m, ch in
           zip(meshes, wl.channels)]
    t0 = time.perf_counter()
    t, d, s, rc = oracle.batch([c.astuple() for c in wl.channels], meshes, Vts, wl.coeffs[idx], wl.e_lab)
    sec = time.perf_counter() - t0
    assert rc == 0
    return t, d, s, sec


def cpu_baseline(wl, n_samples, steps=1):
    """Time the FP64 oracle on a bounded sample of the workload (host cores)."""
    import oracle
    times = []
    for _ in range(steps):
        *_, sec = oracle_solve(wl, list(range(n_samples)))
        times.append(sec)
    sec = statistics.median(times)
    return {"value": n_samples * len(wl.channels) / sec, "unit": UNIT, "cores": oracle.max_threads(),
            "kind": "oracle", "cpu": host_cpu(),
            "sample": f"first {n_samples} of {wl.n_samples} samples x {len(wl.channels)} channels, "
                      f"{len(wl.e_lab)} energies (projection excluded, as on the GPU)"}, sec


def run_reference(args, ws, rank):
    if rank != 0:
        return
    wl = headline_workload(args.workload, args.samples)
    for _ in range(args.warmup):
        cpu_baseline(wl, 1)
    cb, sec = cpu_baseline(wl, args.ref_samples, steps=args.steps)
    line = {"metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"{workload_label(wl)} (oracle on a {args.ref_samples}-sample slice per step)",
                       "samples_per_step": args.ref_samples, "channels": len(wl.channels), "n_E": len(wl.e_lab)},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def phase_err(wl, da, sa, db, sb):
    """Worst |d delta|, |d eps_J| (deg) and |d sigma| (mb) between two result sets."""
    comp = np.array([[1, 1 if ch.coupled else 0, 0] for ch in wl.channels], dtype=bool)
    coup = np.array([ch.coupled for ch in wl.channels], dtype=bool)
    dd = np.abs((da - db + 90.0) % 180.0 - 90.0) * comp[None, :, None, :]
    de = np.abs(da[..., 2] - db[..., 2])[:, coup] if coup.any() else np.zeros(1)
    return {"max_delta_err_deg": float(dd.max()), "max_eps_err_deg": float(de.max()),
            "max_sigma_err_mb": float(np.abs(sa - sb).max())}


def t_rel_err(wl, ta, tb):
    """Worst |dT| over a channel's energies relative to that channel's max |T|."""
    worst = 0.0
    for c in range(len(wl.channels)):
        sc = np.abs(tb[:, c]).max()
        worst = max(worst, float(np.abs(ta[:, c] - tb[:, c]).max() / sc))
    return worst


class Poisson:
    """Open-loop stream through wpcd_submit / wpcd_poll (continuous batching)."""

    def __init__(self, ctx, prec):
        self.ctx, self.prec = ctx, prec

    def run(self, reqs):
        ctx = self.ctx
        lat, pending, refused = [], [], 0
        t0 = time.perf_counter()

        def drain():
            keep = []
            for tk in pending:  # every pending ticket, not only the oldest
                res = ctx.poll(tk)
                if res is None:
                    keep.append(tk)
                else:
                    lat.append(res.latency_us)
                    ctx.release_result(tk)
            pending[:] = keep

        last = 0.0
        for r in reqs:
            while True:
                now = time.perf_counter() - t0
                if now >= r.arrival_s:
                    break
                if pending and now - last > 5e-4:  # at most one pass over the tickets per 0.5 ms
                    drain()
                    last = now
            out = ctx.submit(r.coeffs, r.e_lab, r.n_wp, self.prec, raise_on_error=False)
            if out < 0:
                refused += 1
                continue
            pending.append(out)
        for tk in pending:
            res = ctx.wait(tk, 600000)
            lat.append(res.latency_us)
            ctx.release_result(tk)
        wall = time.perf_counter() - t0
        lat = np.array(lat)
        return {"requests": len(reqs), "completed": int(lat.size), "refused": refused, "wall_s": wall,
                "achieved_req_per_s": lat.size / wall,
                "p50_ms": float(np.percentile(lat, 50) / 1e3) if lat.size else None,
                "p99_ms": float(np.percentile(lat, 99) / 1e3) if lat.size else None}


def serve_latency(args, lrank, prec):
    """Workload 5: a Poisson stream of requests (c, 16..256 sorted energies,
    N_WP from the list) against the server; then the saturation sweep and the
    per-request latency of requests served alone (FP64 and mixed)."""
    from paper_2106_00454_gb300 import api
    nwp = tuple(int(x) for x in args.serve_nwp.split(","))
    reqs = W.serving_requests(duration_s=args.serve_seconds, rate_hz=args.serve_rate, nwp_choices=nwp)
    chs = W.np_channels(4, extra_1s0_tz=True)
    ctx = api.Context(lrank)
    # admission control: at most SERVE_MAX_QUEUE requests wait; beyond that a submission is
    # refused (counted), so an offered rate above capacity sheds load instead of queueing forever
    ctx.serve_start(chs, W.GEN_YUKAWA, W.YUKAWA_PARAMS, W.N_TERMS_YUKAWA, list(nwp), max_batch=256, n_slots=4,
                    max_queue=SERVE_MAX_QUEUE)
    # warm every slot with every N_WP (allocations) before the timed streams
    warm = [ctx.submit(r.coeffs, r.e_lab, r.n_wp, prec) for r in reqs[:128]]
    for t in warm:
        ctx.wait(t, 600000)
        ctx.release_result(t)
    s0 = ctx.serve_stats()
    main = Poisson(ctx, prec).run(reqs)
    s1 = ctx.serve_stats()
    main.update({"offered_rate_hz": args.serve_rate, "n_wp": list(nwp), "channels": len(chs),
                 "channel_solves_per_s": main["completed"] * len(chs) / main["wall_s"],
                 "mean_batch": (s1["completed"] - s0["completed"]) / max(s1["batches"] - s0["batches"], 1),
                 "precision": "mixed" if prec == api.PREC_MIXED else "fp64",
                 "stream": f"{args.serve_seconds:g} s open loop, Poisson arrivals, every pending ticket polled",
                 "max_queue": SERVE_MAX_QUEUE})
    sat = []
    for k, rate in enumerate(float(x) for x in args.sat_rates.split(",") if x):
        rq = W.serving_requests(duration_s=args.sat_seconds, rate_hz=rate, seed=W.SEED + 101 * (k + 1),
                                nwp_choices=nwp)
        r = Poisson(ctx, prec).run(rq)
        r["offered_rate_hz"] = rate
        sat.append(r)
    ok = [r for r in sat if r["refused"] == 0 and r["p99_ms"] is not None and r["p99_ms"] <= SAT_P99_BOUND_MS
          and r["achieved_req_per_s"] >= 0.9 * r["offered_rate_hz"]]
    main["saturation"] = {"p99_bound_ms": SAT_P99_BOUND_MS, "seconds_per_rate": args.sat_seconds, "rates": sat,
                          "max_rate_within_bound_hz": max((r["offered_rate_hz"] for r in ok), default=None)}
    ctx.serve_stop()

    # requests served alone, one at a time: the plain per-request latency of each precision
    ctx.serve_start(chs, W.GEN_YUKAWA, W.YUKAWA_PARAMS, W.N_TERMS_YUKAWA, list(nwp), max_batch=1, n_slots=1)
    alone = {"fp64": {}, "mixed": {}}
    picks = {n: next(r for r in reqs if r.n_wp == n) for n in nwp}
    for name, pr in (("mixed", api.PREC_MIXED), ("fp64", api.PREC_FP64)):
        for n, r in picks.items():
            ctx.wait(ctx.submit(r.coeffs, r.e_lab, n, pr), 600000)  # warm (allocations, this N_WP)
            res = ctx.wait(ctx.submit(r.coeffs, r.e_lab, n, pr), 600000)
            alone[name][str(n)] = {"latency_ms": res.latency_us / 1e3, "n_E": int(r.e_lab.size),
                                   "status": int(res.status)}
    ctx.serve_stop()
    ctx.close()
    main["latency_fp64_plain"] = {"per_nwp": alone["fp64"],
                                  "note": "one request at a time through the server (batch of 1) on the FP64 path"}
    main["latency_mixed_alone"] = {"per_nwp": alone["mixed"], "note": "one request at a time on the mixed path"}
    return main


def jacobi_algorithmic_flops(wl, S):
    """(8/3) n^3 per channel-solve: the paper's count for a symmetric eigensolve (Sec. 4.2.1)."""
    return S * sum((8.0 / 3.0) * (n * (2 if ch.coupled else 1)) ** 3 for n, ch in zip(wl.nwp, wl.channels))


def device_steps(ctx, step, k, flush, stream, ws=1, profiled=False):
    """k device-timed steps (CUDA events on the launching stream), L2 flushed
    between them.  Unprofiled steps run as a caller runs them (CUDA-graph
    replays after the first two calls); profiled steps launch kernel by kernel
    with CUDA events around each launch."""
    import torch
    ctx.profile(profiled)
    evs = []
    barrier(ws)
    torch.cuda.synchronize()
    for _ in range(k):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    ctx.sync()
    prof = ctx.profile_read() if profiled else None
    ctx.profile(False)
    return [a.elapsed_time(b) for a, b in evs], prof


def secondary_batched(args, ctx, dev, flush, stream):
    """The 4096-sample x 15-channel batched workload: FP64 eigensolve (as the
    workload specifies) and mixed, device-timed; the MI comparison method on a
    slice; spin observables from the mixed step's phases."""
    import torch

    from paper_2106_00454_gb300 import api
    wl = W.workload_batched(n_samples=4096)
    md = api.Model(ctx, wl)
    S, nch, nE = wl.n_samples, len(wl.channels), len(wl.e_lab)
    cf = torch.tensor(wl.coeffs, dtype=torch.float64, device=dev)
    e = torch.tensor(wl.e_lab, dtype=torch.float64, device=dev)
    d = torch.empty((S, nch, nE, 3), dtype=torch.float64, device=dev)
    s = torch.empty((S, nE), dtype=torch.float64, device=dev)
    out = {"workload": workload_label(wl), "samples": S, "channels": nch, "n_E": nE, "n_wp": wl.nwp}
    for name, prec, warm, k in (("mixed", api.PREC_MIXED, 3, 5), ("fp64", api.PREC_FP64, 2, 1)):
        def step():
            ctx.solve(md.vset, cf, S, e, None, d, s, prec=prec)
        for _ in range(warm):
            step()
        ms, _ = device_steps(ctx, step, k, flush, stream)
        m = statistics.mean(ms)
        out[name] = {"value": S * nch / (m * 1e-3), "unit": UNIT, "ms_per_step": m, "steps": k,
                     "dtype": "f32+f64" if prec == api.PREC_MIXED else "f64"}
    # leave the mixed step's phases in d / s for the comparisons below
    ctx.solve(md.vset, cf, S, e, None, d, s, prec=api.PREC_MIXED)
    ctx.sync()

    if args.mi_interp > 0:
        k = min(args.mi_samples, S)
        mid = ctx.mi_prepare(wl.channels, wl.gen, wl.gen_params, wl.n_terms, n_quad=args.mi_quad)
        e_int = torch.tensor(W.chebyshev_energies(args.mi_interp), dtype=torch.float64, device=dev)
        dmi = torch.empty((k, nch, nE, 3), dtype=torch.float64, device=dev)
        smi = torch.empty((k, nE), dtype=torch.float64, device=dev)
        cfk = cf[:k].contiguous()
        ctx.mi_solve(mid, cfk, k, e_int, e, None, dmi, smi)  # warm-up
        ctx.sync()
        ms, _ = device_steps(ctx, lambda: ctx.mi_solve(mid, cfk, k, e_int, e, None, dmi, smi), 1, flush, stream)
        ctx.release(mid)
        dd = np.abs((dmi.cpu().numpy() - d[:k].cpu().numpy() + 90.0) % 180.0 - 90.0)[..., :2]
        sel = wl.e_lab > 5.0
        sw = s[:k].cpu().numpy()
        rel_s = np.abs(smi.cpu().numpy() - sw)[:, sel] / np.abs(sw[:, sel])
        out["mi_comparison"] = {
            "method": "matrix inversion (Sec. 2.1) at Chebyshev interpolation energies, linear in T_lab (Sec. 6)",
            "n_interp": args.mi_interp, "n_quad": args.mi_quad, "samples": k, "ms_per_step": ms[0],
            "value": k * nch / (ms[0] * 1e-3), "unit": UNIT,
            "max_phase_diff_to_wpcd_deg": float(dd[:, :, sel].max()),
            "max_sigma_rel_diff_to_wpcd": float(rel_s.max()),
            "note": "method difference (WPCD N_WP 40-100 vs MI N_Q grid and interpolation), not an error bound"}

    if args.angles > 0:
        th = torch.linspace(0.0, np.pi, args.angles, dtype=torch.float64, device=dev)
        ab = torch.empty((S, nE, args.angles, 5, 2), dtype=torch.float64, device=dev)
        dsg = torch.empty((S, nE, args.angles), dtype=torch.float64, device=dev)
        ctx.saclay(wl.channels, d, S, e, th, ab, dsg)  # warm-up
        ms, _ = device_steps(ctx, lambda: ctx.saclay(wl.channels, d, S, e, th, ab, dsg), 3, flush, stream)
        sp_t = statistics.mean(ms)
        # optical theorem against the step's sigma_tot: (2 pi / p) Im(a + b)(0) [fm^2 -> mb]
        p_e = np.sqrt(938.918309 * wl.e_lab / 2.0) / 197.3269804
        abn = ab.cpu().numpy()
        opt = 2 * np.pi / p_e[None, :] * (abn[:, :, 0, 0, 1] + abn[:, :, 0, 1, 1]) * 10.0
        sn = s.cpu().numpy()
        out["spin_observables"] = {"observables": "Saclay amplitudes a-e and dsigma/dOmega (App. A)",
                                   "angles": args.angles, "ms_per_step": sp_t,
                                   "points_per_s": S * nE * args.angles / (sp_t * 1e-3),
                                   "optical_theorem_max_rel_dev": float(np.max(np.abs(opt - sn) / sn))}
    md.release()
    return out


def run_wpcd(args, ws, rank, lrank):
    import torch

    from paper_2106_00454_gb300 import api, build
    if rank == 0:
        build.build()
    barrier(ws)
    torch.cuda.set_device(lrank)
    dev = f"cuda:{lrank}"
    ctx = api.Context(lrank)
    ctx.set_graphs(args.graphs == "on")
    if args.exec == "plain":
        ctx.set_exec(api.EXEC_PLAIN)
    # weak scaling: every rank owns its own block of samples (independent seeds)
    wl = rank_workload(args.samples, rank, args.workload)
    prec = api.PREC_MIXED if args.prec == "mixed" else api.PREC_FP64
    # the projection: FP64 for the FP64 legs; the N_WP = 150 workload's mixed path also
    # projects in reduced precision (angle integrals on the tensor cores)
    t0 = time.perf_counter()
    md64 = api.Model(ctx, wl)
    proj = {"fp64_ms": (time.perf_counter() - t0) * 1e3}
    md = md64
    if prec == api.PREC_MIXED and args.workload == "config4":
        t0 = time.perf_counter()
        md = api.Model(ctx, wl, proj_prec=api.PREC_MIXED)
        proj["mixed_ms"] = (time.perf_counter() - t0) * 1e3
        worst = 0.0
        for c in range(len(wl.channels)):
            a, b = ctx.vset_get(md64.vset, c), ctx.vset_get(md.vset, c)
            for tt in range(a.shape[0]):
                sc = np.max(np.abs(a[tt]))
                if sc > 0:
                    worst = max(worst, float(np.max(np.abs(a[tt] - b[tt])) / sc))
        proj["max_rel_diff_mixed_vs_fp64"] = worst
        proj["note"] = ("wall time of mesh + projection of the 20-channel set (once per set, outside the step); "
                        "mixed: Yukawa angle integrals as a BF16 three-term tensor-core contraction")
    S, nch, nE = wl.n_samples, len(wl.channels), len(wl.e_lab)
    cf = torch.tensor(wl.coeffs, dtype=torch.float64, device=dev)
    e = torch.tensor(wl.e_lab, dtype=torch.float64, device=dev)
    t = torch.empty((S, nch, nE, 2, 2, 2), dtype=torch.float64, device=dev)
    d = torch.empty((S, nch, nE, 3), dtype=torch.float64, device=dev)
    s = torch.empty((S, nE), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(lrank)

    def step():
        ctx.solve(md.vset, cf, S, e, t, d, s, prec=prec)

    for _ in range(args.warmup):
        step()
    ctx.sync()

    launches0 = ctx.kernel_launches()
    graphs0 = ctx.graph_stats()
    with Clocks(lrank) as clk:
        step_ms, _ = device_steps(ctx, step, args.steps, flush, stream, ws)
        launches = ctx.kernel_launches() - launches0
        graphs1 = ctx.graph_stats()
    # per-launch kernel times for the phase breakdown and the roofline (kernel by kernel)
    kp = max(1, min(args.steps, args.prof_steps))
    prof_step_ms, prof = device_steps(ctx, step, kp, flush, stream, ws, profiled=True)
    ms = statistics.mean(step_ms)
    ms_max = max_over_ranks(ws, ms, dev)
    barrier(ws)
    value = ws * S * nch / (ms_max * 1e-3)

    # end to end through the host entry point: copies in and out inside the timed region
    def pinned(shape, src=None):
        a = torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
        if src is not None:
            a[...] = src
        return a

    # pinned host buffers, as a serving front end holds them: the copies run at the link's rate
    ch_, eh = pinned(wl.coeffs.shape, wl.coeffs), pinned(wl.e_lab.shape, wl.e_lab)
    th = pinned((S, nch, nE, 2, 2, 2))
    dh = pinned((S, nch, nE, 3))
    sh = pinned((S, nE))
    for _ in range(2):  # the second call captures the CUDA graph the timed calls replay
        ctx.solve_host(md.vset, ch_, S, eh, th, dh, sh, prec=prec)
    e2e_ms = []
    with Clocks(lrank) as clk_e2e:
        for _ in range(max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.solve_host(md.vset, ch_, S, eh, th, dh, sh, prec=prec)
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e = statistics.mean(e2e_ms)
    e2e_max = max_over_ranks(ws, e2e, dev)
    h2d = wl.coeffs.nbytes + wl.e_lab.nbytes
    d2h = th.nbytes + dh.nbytes + sh.nbytes
    del th, dh, sh

    line = None
    if rank == 0:
        dn, sn, tn = d.cpu().numpy(), s.cpu().numpy(), t.cpu().numpy().view(np.complex128).reshape(S, nch, nE, 2, 2)

        # the mixed path against the FP64 path on the same GPU (a slice) and both against the oracle
        accuracy, acc_oracle = None, None
        d6 = s6 = od = os_ = None
        ko = 0
        k = min(args.check_samples, S)
        if k > 0:
            t64 = torch.empty((k, nch, nE, 2, 2, 2), dtype=torch.float64, device=dev)
            d64 = torch.empty((k, nch, nE, 3), dtype=torch.float64, device=dev)
            s64 = torch.empty((k, nE), dtype=torch.float64, device=dev)
            ctx.solve(md64.vset, cf[:k].contiguous(), k, e, t64, d64, s64, prec=api.PREC_FP64)
            ctx.sync()
            d6, s6 = d64.cpu().numpy(), s64.cpu().numpy()
            t6 = t64.cpu().numpy().view(np.complex128).reshape(k, nch, nE, 2, 2)
            if prec == api.PREC_MIXED:
                accuracy = {"samples_checked": k, "reference": "FP64 path on the same GPU",
                            **phase_err(wl, dn[:k], sn[:k], d6, s6), "max_T_rel_err": t_rel_err(wl, tn[:k], t6)}
            ko = min(args.oracle_samples, k)
            if ko > 0:
                idx = list(range(ko))
                ot, od, os_, osec = oracle_solve(wl, idx)
                acc_oracle = {"samples": ko, "channels": nch, "n_E": nE, "oracle_seconds": osec,
                              "reference": "FP64 CPU oracle (own Jacobi, plain C), the first samples",
                              "headline_path": {**phase_err(wl, dn[:ko], sn[:ko], od, os_),
                                                "max_T_rel_err": t_rel_err(wl, tn[:ko], ot)},
                              "fp64_path": {**phase_err(wl, d6[:ko], s6[:ko], od, os_),
                                            "max_T_rel_err": t_rel_err(wl, t6[:ko], ot),
                                            "max_sigma_rel_err": float(np.max(np.abs(s6[:ko] - os_) / os_))},
                              "tolerances": {"mixed": "1e-3 deg, 0.01 mb", "fp64": "1e-10 rel T, 1e-8 deg"}}
            del t64, d64, s64

        # opt-in single FP64 refinement iteration on the headline workload: its time and its errors
        one_iter = None
        if prec == api.PREC_MIXED and args.one_iter_leg:
            ctx.set_refine_iters(1)
            t1 = torch.empty((S, nch, nE, 2, 2, 2), dtype=torch.float64, device=dev)
            d1 = torch.empty((S, nch, nE, 3), dtype=torch.float64, device=dev)
            s1 = torch.empty((S, nE), dtype=torch.float64, device=dev)

            def step1():
                ctx.solve(md.vset, cf, S, e, t1, d1, s1, prec=prec)
            for _ in range(2):
                step1()
            ms1, _ = device_steps(ctx, step1, 1, flush, stream)
            ctx.set_refine_iters(2)
            d1n, s1n = d1.cpu().numpy(), s1.cpu().numpy()
            one_iter = {"refine_iterations": 1, "value": S * nch / (ms1[0] * 1e-3), "unit": UNIT,
                        "ms_per_step": ms1[0],
                        "note": "opt-in (WPCD_OPT_REFINE_ITERS = 1), not within the 0.01 mb cross-section bar "
                                "on every sample; the headline uses 2"}
            if accuracy is not None:
                one_iter["vs_fp64_gpu"] = phase_err(wl, d1n[:k], s1n[:k], d6, s6)
            if acc_oracle is not None:
                one_iter["vs_oracle"] = phase_err(wl, d1n[:ko], s1n[:ko], od, os_)
            del t1, d1, s1

        # same-GPU FP64 baselines: batched (one launch per size bucket) and plain (one solve per launch)
        base = {}
        for name, ns, mode in (("baseline_batched_fp64", args.fp64_batched_samples, api.EXEC_BATCHED),
                               ("baseline_plain_fp64", args.fp64_plain_samples, api.EXEC_PLAIN)):
            ns = min(ns, S)
            if ns <= 0:
                continue
            cfs = cf[:ns].contiguous()
            dd = torch.empty((ns, nch, nE, 3), dtype=torch.float64, device=dev)
            ss = torch.empty((ns, nE), dtype=torch.float64, device=dev)
            ctx.set_exec(mode)

            def fstep():
                ctx.solve(md64.vset, cfs, ns, e, None, dd, ss, prec=api.PREC_FP64)
            reps = 2 if mode == api.EXEC_BATCHED else 1
            for _ in range(reps):  # warm-up (allocations; the batched path's graph capture)
                fstep()
            ctx.sync()
            fms, _ = device_steps(ctx, fstep, reps, flush, stream)
            ctx.set_exec(api.EXEC_PLAIN if args.exec == "plain" else api.EXEC_BATCHED)
            fm = statistics.mean(fms)
            base[name] = {"value": ns * nch / (fm * 1e-3), "unit": UNIT, "ms_per_call": fm, "samples": ns,
                          "channel_solves": ns * nch, "dtype": "f64",
                          "exec": "one eigensolve launch per (sample, channel)" if mode == api.EXEC_PLAIN
                          else "one launch per size bucket, CUDA graph"}
            del dd, ss
        if base:
            base["headline_over_batched_fp64"] = value / base["baseline_batched_fp64"]["value"] \
                if "baseline_batched_fp64" in base else None
            base["headline_over_plain_fp64"] = value / base["baseline_plain_fp64"]["value"] \
                if "baseline_plain_fp64" in base else None

        # the dominant kernel (the eigensolver: the single kernel with the largest share of the step)
        sum_n3 = sum((n * (2 if c.coupled else 1)) ** 3 for n, c in zip(wl.nwp, wl.channels))
        eig_ms, eig_n = prof["eigen"]
        ref_ms, ref_n = prof["refine"]
        big = [n * (2 if c.coupled else 1) for n, c in zip(wl.nwp, wl.channels)]
        jac = {"kernel": "k_jacobi_f64" if prec == api.PREC_FP64 else "k_jacobi_mixed", "bound": "alu",
               "flops_per_step": S * (8.0 / 3.0) * sum_n3,
               "flops_note": "(8/3) n^3 per channel-solve, the paper's symmetric-eigensolve count (Sec. 4.2.1)",
               "ms_per_step": eig_ms / kp, "launches_per_step": eig_n / kp, "matrix_sizes": sorted(set(big)),
               "peak": FP64_PEAK_TFLOPS if prec == api.PREC_FP64 else FP32_PEAK_TFLOPS,
               "peak_source": FP64_PEAK_NOTE if prec == api.PREC_FP64 else FP32_PEAK_NOTE,
               "timing": ("CUDA events around each eigensolver launch (one kernel per launch), over "
                          f"{kp} further steps launched kernel by kernel")}
        if args.exec == "batched" and args.sweep_samples > 0:
            # executed eigensolver work from the sweep count of every solve of a slice:
            # a round updates the packed matrix in ~n^2/8 quads of 16 flop and rotates
            # n/2 eigenvector column pairs at 4n flop, n - 1 rounds a sweep: <= 4 n^3 a sweep
            ks = min(args.sweep_samples, S)
            eid = ctx.diag(md.vset, cf[:ks].contiguous(), ks, prec=prec)
            sweeps = torch.zeros((ks, nch), dtype=torch.int32, device=dev)
            ctx.diag_status(eid, sweeps)
            ctx.sync()
            sw = np.clip(sweeps.cpu().numpy(), 0, None).astype(np.float64)
            ctx.release(eid)
            nvec = np.array(big, dtype=np.float64)
            ex = float((sw * 4.0 * nvec[None, :] ** 3).sum()) * (S / ks)
            ach = ex / (jac["ms_per_step"] * 1e-3) / 1e12
            jac["executed"] = {"flops_per_step": ex, "achieved": ach, "frac": ach / jac["peak"],
                               "sweeps_mean": float(sw.mean()), "sweeps_max": int(sw.max()),
                               "note": f"upper bound: sweeps x 4 n^3 per solve, sweeps of the first {ks} samples"}
        ref, ref_traffic = None, None
        if ref_n:
            if ctx.refine_engine == api.REFINE_TENSOR:
                # Ozaki products: 6 balanced 8-bit digits per operand, the 21 digit pairs of
                # weight >= 2^-40 (p + q <= 5), each a 2 n^3 BF16 tensor-core product
                peak, src = measured_peak("bf16_tflops_sustained", 1700.0)
                ref = {"kernel": "refinement phase (k_oz_gemm_tc tcgen05 BF16 digit products, digit splits, "
                                 "FP64 update and eigenpair sort)", "bound": "tensor",
                       "flops_per_step": S * 8 * 21 * 2.0 * sum_n3,
                       "flops_note": "8 products (2 iterations x H X, X^T Y, X^T X, X (I + E)) x 21 digit pairs "
                                     "x 2 n^3 BF16 flop",
                       "peak": peak, "peak_source": src}
            else:
                ref = {"kernel": "refinement phase (k_bgemm64 FP64 products and FP64 update kernels)",
                       "bound": "alu", "flops_per_step": S * 16.0 * sum_n3,
                       "flops_note": "two refinement iterations of four 2 n^3 products: 16 n^3 flop",
                       "peak": FP64_PEAK_TFLOPS, "peak_source": FP64_PEAK_NOTE}
            ref.update({"ms_per_step": ref_ms / kp, "launches_per_step": ref_n / kp,
                        "timing": "CUDA events around the whole phase (several kernels per launch)"})
            if ctx.refine_engine == api.REFINE_TENSOR and args.workload == "config4" and all(v <= 304 for v in big):
                ref_traffic = REFINE_DRAM_BYTES_PER_N2 * S * sum(v * v for v in big) / ref["launches_per_step"]
        for r in (jac, ref):
            if r:
                r["achieved"] = r["flops_per_step"] / (r["ms_per_step"] * 1e-3) / 1e12
                r["unit"] = "TFLOP/s"
                r["frac"] = r["achieved"] / r["peak"]
                r["traffic"] = None
        if ref_traffic is not None and prec == api.PREC_MIXED:
            ref["traffic"] = ref_traffic
            ref["traffic_note"] = ("ncu capture of the workload's first 128 samples (567 B of DRAM traffic per "
                                   "matrix element per solve against the algorithmic 24 B: the BF16 digit slices of "
                                   "every operand and the FP64 intermediates go through HBM), scaled by the step's "
                                   "sum of n^2; bytes per phase launch")
        if prec == api.PREC_MIXED and args.workload == "config4" and jac["launches_per_step"] > 0 \
                and all(v <= 304 for v in big):
            # DRAM bytes per launch: the capture's bytes per matrix element times the step's
            # sum of n^2 over its solves, over the step's Jacobi launches
            jac["traffic"] = JACOBI_MIXED_DRAM_BYTES_PER_N2 * S * sum(v * v for v in big) / jac["launches_per_step"]
            jac["traffic_note"] = ("ncu capture of the workload's first 128 samples (37.1 B of DRAM traffic per "
                                   "matrix element per solve against the algorithmic 16 B), scaled by the step's "
                                   "sum of n^2; bytes per launch")

        clocks = clk.summary()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == api.PREC_FP64 else "f32+f64", "data": "synthetic",
            "config": {"workload": workload_label(wl), "samples": S, "channels": nch, "n_E": nE,
                       "projection": "tensor-core angle integrals" if md is not md64 else "fp64",
                       "n_wp": sorted(set(wl.nwp)), "exec": args.exec, "precision": args.prec,
                       "cuda_graphs": args.graphs, "l2": "flushed between timed steps (512 MB write)",
                       "parallelism": f"replicas{ws}"},
            "roofline": jac,
            "roofline_secondary": ref,
            "phases_ms_per_step": {kk: v[0] / kp for kk, v in prof.items()},
            "projection": proj,
            "ms_per_step_kernel_by_kernel": statistics.mean(prof_step_ms),
            "cuda_graphs": {"captures": graphs1["captures"],
                            "replays_in_timed_steps": graphs1["replays"] - graphs0["replays"]},
            "e2e": {"value": ws * S * nch / (e2e_max * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_max,
                    "ms_each": [round(x, 2) for x in e2e_ms], "clocks": clk_e2e.summary()},
            "gpu_launches": launches,
            "autotune": ctx.tuning(),
            "accuracy_vs_fp64": accuracy,
            "accuracy_vs_oracle": acc_oracle,
            "mixed_one_refinement_iteration": one_iter,
            **base,
            "clocks": clocks,
        }
    if md is not md64:
        md.release()
    md64.release()
    del t, d, s
    if rank == 0:
        if args.secondary == "on":
            line["batched_4096x15ch"] = secondary_batched(args, ctx, dev, flush, stream)
        if args.serve_seconds > 0:
            line["latency"] = serve_latency(args, lrank, prec)
        if not args.no_cpu_baseline:
            cb, _ = cpu_baseline(wl, args.cpu_samples)
            line["cpu_baseline"] = cb
        print(json.dumps(line), flush=True)
    ctx.close()


def main():
    args = parse()
    ws, rank, lrank = dist_init(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_wpcd(args, ws, rank, lrank)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
