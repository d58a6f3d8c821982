"""Benchmark of the WPCD hot path on one GB300 (or N, sharded by sample).

One step = the whole hot path over one batch: parameter sum + eigensolve of
every (sample, channel), energy plan, SWP boundaries + resolvent + T at the
needed bins, T at every requested energy, phase interpolation and the np
total cross section.  Workload: 4096 parameter samples x 15 channels (J <= 4
plus a T_z = +-1 copy of 1S0), N_WP per channel from {40, 64, 100} (coupled
80/128/200), 128 lab energies 1..350 MeV, FP64 (seeded synthetic inputs).

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the host cores instead, on a bounded sample of the same workload.
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
FP64_PEAK_TFLOPS = 1.25      # nominal GB300 FP64 rate (MEASURED_PEAKS.json holds no FP64 figure)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # FP32 FMA lanes x clock
JACOBI_MIXED_DRAM_BYTES_1024 = 2.06e9  # k_jacobi_mixed, one step of the 1024-sample batched workload
L2_FLUSH_BYTES = 512 << 20   # > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="wpcd", choices=["wpcd", "reference"])
    ap.add_argument("--samples", type=int, default=4096)
    ap.add_argument("--exec", default="batched", choices=["batched", "plain"])
    ap.add_argument("--prec", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--graphs", default="on", choices=["on", "off"],
                    help="replay repeated solves from CUDA graphs (off: kernel by kernel, e.g. for ncu launch lists)")
    ap.add_argument("--check-samples", type=int, default=64,
                    help="samples re-solved in FP64 to state the mixed path's phase error")
    ap.add_argument("--cpu-samples", type=int, default=24, help="oracle sample size for the CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=5.0,
                    help="length of the Poisson request stream for the latency figures (0 = skip)")
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-nwp", default="32,64,128")
    ap.add_argument("--mi-interp", type=int, default=32,
                    help="MI comparison method: interpolation energies (0 = skip the MI leg)")
    ap.add_argument("--mi-quad", type=int, default=96, help="MI momentum grid points per l-block")
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


def rank_workload(samples, rank):
    """This rank's shard of a weak-scaling job: the same channels, meshes and
    energies on every rank, its own block of parameter samples."""
    return W.workload_batched(n_samples=samples, sample_seed=W.SEED + 7919 * rank)


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


def cpu_baseline(wl, n_samples, steps=1):
    """Time the FP64 oracle on a bounded sample of the workload (host cores)."""
    import oracle
    oracle.build()
    meshes = [oracle.Mesh(n) for n in wl.nwp]
    Vts = [oracle.project_channel(m, ch.astuple(), wl.gen, wl.gen_params, wl.n_terms) for m, ch in
           zip(meshes, wl.channels)]
    sub = wl.coeffs[:n_samples]
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        _, _, _, rc = oracle.batch([c.astuple() for c in wl.channels], meshes, Vts, sub, wl.e_lab)
        times.append(time.perf_counter() - t0)
        assert rc == 0
    sec = statistics.median(times)
    return {"value": n_samples * len(wl.channels) / sec, "unit": UNIT, "cores": oracle.max_threads(),
            "kind": "oracle", "cpu": host_cpu(),
            "sample": f"first {n_samples} of {wl.n_samples} samples x {len(wl.channels)} channels, "
                      f"{len(wl.e_lab)} energies (projection excluded, as on the GPU)"}, sec


def run_reference(args, ws, rank):
    if rank != 0:
        return
    wl = W.workload_batched(n_samples=args.samples)
    for _ in range(args.warmup):
        cpu_baseline(wl, max(1, args.cpu_samples // 4))
    cb, sec = cpu_baseline(wl, args.cpu_samples, steps=args.steps)
    line = {"metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"{wl.name} (oracle on a {args.cpu_samples}-sample slice)",
                       "samples_per_step": args.cpu_samples, "channels": len(wl.channels), "n_E": len(wl.e_lab)},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def serve_latency(args, lrank, prec):
    """Open-loop Poisson stream through wpcd_submit / wpcd_poll (continuous batching)."""
    from paper_2106_00454_gb300 import api
    nwp = tuple(int(x) for x in args.serve_nwp.split(","))
    reqs = W.serving_requests(duration_s=args.serve_seconds, rate_hz=args.serve_rate, nwp_choices=nwp)
    chs = W.np_channels(4, extra_1s0_tz=True)
    ctx = api.Context(lrank)
    ctx.serve_start(chs, W.GEN_YUKAWA, W.YUKAWA_PARAMS, W.N_TERMS_YUKAWA, list(nwp), max_batch=256, n_slots=4)
    # warm the slots (allocations) with a short burst before the timed stream
    warm = [ctx.submit(r.coeffs, r.e_lab, r.n_wp, prec) for r in reqs[:64]]
    for t in warm:
        ctx.wait(t)
        ctx.release_result(t)
    lat, pending, refused = [], [], 0
    t0 = time.perf_counter()
    for r in reqs:
        while time.perf_counter() - t0 < r.arrival_s:
            pass
        out = ctx.submit(r.coeffs, r.e_lab, r.n_wp, prec, raise_on_error=False)
        if out < 0:
            refused += 1
            continue
        pending.append(out)
        while pending:
            res = ctx.poll(pending[0])
            if res is None:
                break
            lat.append(res.latency_us)
            ctx.release_result(pending.pop(0))
    for t in pending:
        res = ctx.wait(t, 600000)
        lat.append(res.latency_us)
        ctx.release_result(t)
    wall = time.perf_counter() - t0
    stats = ctx.serve_stats()
    ctx.serve_stop()
    ctx.close()
    lat = np.array(lat)
    return {"requests": len(reqs), "completed": int(lat.size), "refused": refused, "offered_rate_hz": args.serve_rate,
            "n_wp": list(nwp), "channels": len(chs), "wall_s": wall, "achieved_req_per_s": lat.size / wall,
            "channel_solves_per_s": lat.size * len(chs) / wall,
            "p50_ms": float(np.percentile(lat, 50) / 1e3) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99) / 1e3) if lat.size else None,
            "mean_batch": stats["completed"] / max(stats["batches"], 1), "precision": args.prec}


def jacobi_algorithmic_flops(wl, S):
    """(8/3) n^3 per channel-solve: the paper's count for a symmetric eigensolve (Sec. 4.2.1)."""
    return S * sum((8.0 / 3.0) * (n * (2 if ch.coupled else 1)) ** 3 for n, ch in zip(wl.nwp, wl.channels))


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
    wl = rank_workload(args.samples, rank)
    md = api.Model(ctx, wl)
    S, nch, nE = wl.n_samples, len(wl.channels), len(wl.e_lab)
    cf = torch.tensor(wl.coeffs, dtype=torch.float64, device=dev)
    e = torch.tensor(wl.e_lab, dtype=torch.float64, device=dev)
    t = torch.empty((S, nch, nE, 2, 2, 2), dtype=torch.float64, device=dev)
    d = torch.empty((S, nch, nE, 3), dtype=torch.float64, device=dev)
    s = torch.empty((S, nE), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(lrank)

    prec = api.PREC_MIXED if args.prec == "mixed" else api.PREC_FP64

    def step():
        ctx.solve(md.vset, cf, S, e, t, d, s, prec=prec)

    for _ in range(args.warmup):
        step()
    ctx.sync()

    def timed(profiled):
        """K device-timed steps, L2 flushed between them.  Unprofiled steps run as
        the caller runs them (CUDA-graph replays after the warm-up); profiled steps
        launch kernel by kernel with CUDA events around each launch."""
        ctx.profile(profiled)
        evs = []
        barrier(ws)
        torch.cuda.synchronize()
        for _ in range(args.steps):
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

    launches0 = ctx.kernel_launches()
    graphs0 = ctx.graph_stats()
    with Clocks(lrank) as clk:
        step_ms, _ = timed(False)
        launches = ctx.kernel_launches() - launches0
        graphs1 = ctx.graph_stats()
        # per-launch kernel times for the phase breakdown and the roofline
        prof_step_ms, prof = timed(True)
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
    ch, eh = pinned(wl.coeffs.shape, wl.coeffs), pinned(wl.e_lab.shape, wl.e_lab)
    th = pinned((S, nch, nE, 2, 2, 2))
    dh = pinned((S, nch, nE, 3))
    sh = pinned((S, nE))
    for _ in range(2):  # the second call captures the CUDA graph the timed calls replay
        ctx.solve_host(md.vset, ch, S, eh, th, dh, sh, prec=prec)
    e2e_ms = []
    with Clocks(lrank) as clk_e2e:
        for _ in range(max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.solve_host(md.vset, ch, S, eh, th, dh, sh, prec=prec)
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e = statistics.mean(e2e_ms)
    e2e_max = max_over_ranks(ws, e2e, dev)
    h2d = wl.coeffs.nbytes + wl.e_lab.nbytes
    d2h = th.nbytes + dh.nbytes + sh.nbytes

    # the mixed path's phase / cross-section error against plain FP64 on the GPU
    accuracy = None
    if prec == api.PREC_MIXED and args.check_samples > 0:
        k = min(args.check_samples, S)
        d64 = torch.empty((k, nch, nE, 3), dtype=torch.float64, device=dev)
        s64 = torch.empty((k, nE), dtype=torch.float64, device=dev)
        ctx.solve(md.vset, cf[:k].contiguous(), k, e, None, d64, s64, prec=api.PREC_FP64)
        ctx.sync()
        dm, d6 = d[:k].cpu().numpy(), d64.cpu().numpy()
        comp = np.array([[1, 1 if ch.coupled else 0, 1 if ch.coupled else 0] for ch in wl.channels], dtype=bool)
        diff = np.abs((dm - d6 + 90.0) % 180.0 - 90.0)
        diff[..., 2] = np.abs(dm[..., 2] - d6[..., 2])
        diff = diff * comp[None, :, None, :]
        accuracy = {"samples_checked": k, "max_phase_err_deg": float(diff.max()),
                    "max_sigma_err_mb": float(np.abs(s[:k].cpu().numpy() - s64.cpu().numpy()).max()),
                    "reference": "FP64 path on the same GPU"}

    # the paper's comparison method on the same GPU: MI solves at Chebyshev
    # interpolation energies, phases interpolated in T_lab (Sec. 2.1, Sec. 6)
    mi = None
    if args.mi_interp > 0:
        mid = ctx.mi_prepare(wl.channels, wl.gen, wl.gen_params, wl.n_terms, n_quad=args.mi_quad)
        e_int = torch.tensor(W.chebyshev_energies(args.mi_interp), dtype=torch.float64, device=dev)
        dmi = torch.empty((S, nch, nE, 3), dtype=torch.float64, device=dev)
        smi = torch.empty((S, nE), dtype=torch.float64, device=dev)
        ctx.mi_solve(mid, cf, S, e_int, e, None, dmi, smi)  # warm-up
        ctx.sync()
        mi_ms = []
        for _ in range(2):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.mi_solve(mid, cf, S, e_int, e, None, dmi, smi)
            b.record(stream)
            torch.cuda.synchronize()
            mi_ms.append(a.elapsed_time(b))
        ctx.sync()
        ctx.release(mid)
        dd = np.abs((dmi.cpu().numpy() - d.cpu().numpy() + 90.0) % 180.0 - 90.0)[..., :2]
        sel = wl.e_lab > 5.0
        rel_s = np.abs(smi.cpu().numpy() - s.cpu().numpy())[:, sel] / np.abs(s.cpu().numpy()[:, sel])
        mi_t = statistics.mean(mi_ms)
        mi = {"method": "matrix inversion (Sec. 2.1) at Chebyshev interpolation energies, linear in T_lab (Sec. 6)",
              "n_interp": args.mi_interp, "n_quad": args.mi_quad, "ms_per_step": mi_t,
              "value": S * nch / (mi_t * 1e-3), "unit": UNIT,
              "max_phase_diff_to_wpcd_deg": float(dd[:, :, sel].max()),
              "max_sigma_rel_diff_to_wpcd": float(rel_s.max()),
              "note": "method difference (WPCD N_WP 40-100 vs MI N_Q grid and interpolation), not an error bound"}

    # spin observables (App. A) from the step's phases: M-matrix, Saclay amplitudes, dsigma/dOmega
    spin = None
    if args.angles > 0:
        th = torch.linspace(0.0, np.pi, args.angles, dtype=torch.float64, device=dev)
        ab = torch.empty((S, nE, args.angles, 5, 2), dtype=torch.float64, device=dev)
        dsg = torch.empty((S, nE, args.angles), dtype=torch.float64, device=dev)
        ctx.saclay(wl.channels, d, S, e, th, ab, dsg)  # warm-up
        sp_ms = []
        for _ in range(3):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.saclay(wl.channels, d, S, e, th, ab, dsg)
            b.record(stream)
            torch.cuda.synchronize()
            sp_ms.append(a.elapsed_time(b))
        sp_t = statistics.mean(sp_ms)
        # optical theorem against the step's sigma_tot: (2 pi / p) Im(a + b)(0) [fm^2 -> mb]
        p_e = np.sqrt(938.918309 * wl.e_lab / 2.0) / 197.3269804
        abn = ab.cpu().numpy()
        opt = 2 * np.pi / p_e[None, :] * (abn[:, :, 0, 0, 1] + abn[:, :, 0, 1, 1]) * 10.0
        spin = {"observables": "Saclay amplitudes a-e and dsigma/dOmega (App. A)", "angles": args.angles,
                "ms_per_step": sp_t, "points_per_s": S * nE * args.angles / (sp_t * 1e-3),
                "optical_theorem_max_rel_dev": float(np.max(np.abs(opt - s.cpu().numpy()) / s.cpu().numpy()))}

    sum_n3 = sum((n * (2 if ch.coupled else 1)) ** 3 for n, ch in zip(wl.nwp, wl.channels))
    eig_ms, eig_n = prof["eigen"]
    ref_ms, ref_n = prof["refine"]
    jac = {"kernel": "k_jacobi_f64" if prec == api.PREC_FP64 else "k_jacobi_mixed", "bound": "alu",
           "flops_per_step": S * (8.0 / 3.0) * sum_n3,
           "flops_note": "(8/3) n^3 per channel-solve, the paper's symmetric-eigensolve count (Sec. 4.2.1)",
           "ms_per_step": eig_ms / args.steps, "launches_per_step": eig_n / args.steps,
           "peak": FP64_PEAK_TFLOPS if prec == api.PREC_FP64 else FP32_PEAK_TFLOPS,
           "peak_source": ("nominal GB300 FP64 rate (measured 1.19 TFLOP/s with a DFMA probe)" if prec == api.PREC_FP64
                           else "FP32 FMA rate from unit counts: 152 SM x 128 lanes x 2 flop x 2.07 GHz")}
    if args.exec == "batched":
        # executed eigensolver work, from the sweep count of every solve (the eigensolver's
        # status): a round updates the packed matrix in ~n^2/8 quads of 16 flop and rotates
        # n/2 eigenvector column pairs at 4n flop, n - 1 rounds a sweep, so <= 4 n^3 per
        # sweep (an upper bound: pairs below the rotation threshold are skipped)
        eid = ctx.diag(md.vset, cf, S, prec=prec)
        sweeps = torch.zeros((S, nch), dtype=torch.int32, device=dev)
        ctx.diag_status(eid, sweeps)
        ctx.sync()
        sw = np.clip(sweeps.cpu().numpy(), 0, None).astype(np.float64)
        ctx.release(eid)
        nvec = np.array([n * (2 if ch.coupled else 1) for n, ch in zip(wl.nwp, wl.channels)], dtype=np.float64)
        ex = float((sw * 4.0 * nvec[None, :] ** 3).sum())
        ach = ex / (jac["ms_per_step"] * 1e-3) / 1e12
        jac["executed"] = {"flops_per_step": ex, "achieved": ach, "frac": ach / jac["peak"],
                           "sweeps_mean": float(sw.mean()), "sweeps_max": int(sw.max()),
                           "note": "upper bound: sweeps x 4 n^3 per solve"}
    ref = None
    if ref_n:
        if ctx.refine_engine == api.REFINE_TENSOR:
            # Ozaki products: 6 balanced 8-bit digits per operand, the 21 digit pairs of
            # weight >= 2^-40 (p + q <= 5), each a 2 n^3 BF16 tensor-core product
            peak, src = measured_peak("bf16_tflops_sustained", 1700.0)
            ref = {"kernel": "refinement phase (k_oz_gemm_tc tcgen05 BF16 digit products, digit splits, "
                             "FP64 update and eigenpair sort)", "bound": "tensor",
                   "flops_per_step": S * 8 * 21 * 2.0 * sum_n3,
                   "flops_note": "8 products (2 iterations x 4) x 21 digit pairs x 2 n^3 BF16 flop",
                   "peak": peak, "peak_source": src}
        else:
            ref = {"kernel": "refinement phase (k_bgemm64 FP64 products and FP64 update kernels)", "bound": "alu",
                   "flops_per_step": S * 16.0 * sum_n3,
                   "flops_note": "two refinement iterations of four 2 n^3 products: 16 n^3 flop",
                   "peak": FP64_PEAK_TFLOPS, "peak_source": "nominal GB300 FP64 rate"}
        ref.update({"ms_per_step": ref_ms / args.steps, "launches_per_step": ref_n / args.steps,
                    "timing": "CUDA events around the whole phase (several kernels per launch)"})
    jac["timing"] = ("CUDA events around each k_jacobi launch (one kernel per launch), over K further timed "
                     "steps launched kernel by kernel")
    for r in (jac, ref):
        if r:
            r["achieved"] = r["flops_per_step"] / (r["ms_per_step"] * 1e-3) / 1e12
            r["unit"] = "TFLOP/s"
            r["frac"] = r["achieved"] / r["peak"]
            r["traffic"] = None
    if prec == api.PREC_MIXED and jac["launches_per_step"] > 0 and wl.name.startswith("batched_"):
        # DRAM bytes of the mixed Jacobi launches of one step of this workload, from an ncu
        # capture at 1024 samples (dram__bytes_read.sum + dram__bytes_write.sum, all six buckets:
        # 2.06e9 B), scaled by the channel-solves (the FP64 H and eigenvectors handed to the
        # refinement, 16 n^2 B per solve, dominate), per launch like "achieved"
        jac["traffic"] = JACOBI_MIXED_DRAM_BYTES_1024 * (S / 1024.0) / jac["launches_per_step"]
        jac["traffic_note"] = "ncu capture at 1024 samples, scaled by channel-solves; bytes per launch"

    # the eigensolver launch is the single kernel with the largest share of the step
    dominant, secondary = jac, ref
    if rank == 0:
        clocks = clk.summary()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == api.PREC_FP64 else "f32+f64", "data": "synthetic",
            "config": {"workload": wl.name + "_nwp40-64-100_128E", "samples": S, "channels": nch, "n_E": nE,
                       "n_wp": wl.nwp, "exec": args.exec, "precision": args.prec, "cuda_graphs": args.graphs,
                       "l2": "flushed between timed steps (512 MB write)", "parallelism": f"replicas{ws}"},
            "roofline": dominant,
            "roofline_secondary": secondary,
            "phases_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
            "ms_per_step_kernel_by_kernel": statistics.mean(prof_step_ms),
            "cuda_graphs": {"captures": graphs1["captures"],
                            "replays_in_timed_steps": graphs1["replays"] - graphs0["replays"]},
            "e2e": {"value": ws * S * nch / (e2e_max * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_max,
                    "ms_each": [round(x, 2) for x in e2e_ms], "clocks": clk_e2e.summary()},
            "gpu_launches": launches,
            "autotune": ctx.tuning(),
            "accuracy_vs_fp64": accuracy,
            "clocks": clocks,
        }
        if mi is not None:
            line["mi_comparison"] = mi
        if spin is not None:
            line["spin_observables"] = spin
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
