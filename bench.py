#!/usr/bin/env python
"""Throughput of SAGE/EM direction-dependent calibration on GB300.

One step = one sc_calibrate_sage call on one job (predict every cluster,
then n_em SAGE sweeps of n_lm Levenberg-Marquardt iterations per cluster)
with the job's inputs resident in HBM.  The metric counts, per second,
visibilities x clusters x LM iterations:

    value = (B * T * F) * K * n_lm * n_em * steps * n_gpus / seconds

Default workload: SKA1-LOW scale, 512 stations (130816 baselines), 10
timeslots, 4 channels 140-160 MHz, 40 clusters x 100 sources, 5 SAGE sweeps x
10 LM iterations, mixed precision (float32 data and factorisation, float64
phase argument, Jones state and step refinement).  Inputs are synthetic,
shaped like the paper's 512-station dataset (paper §2).

With --gpus N (launched by torchrun) every rank calibrates its own job (an
independent sub-band, seed = rank): no collective on the data path, weak
scaling; the barrier and the max over ranks only frame the timing.
--impl reference times the FP64 CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1910_13908_gb300 import synth  # noqa: E402

METRIC = "vis·cluster/s per LM iter"
UNIT = "vis·cluster·iter/s"

WORKLOADS = {
    # name: (config, n_em, n_lm, description)
    "ska512": ("c4", 5, 10, "SKA1-LOW scale: 512 stations (130816 baselines), 10 timeslots, "
                            "4 channels 140-160 MHz, 40 clusters x 100 sources, 5 SAGE sweeps x 10 LM"),
    "precision128": ("c2", 3, 10, "128 stations (8128 baselines), 20 timeslots, 8 channels 140-160 MHz "
                                  "(spectral index -0.7), 10 clusters x 25 sources, 3 SAGE sweeps x 10 LM"),
    "lofar64": ("c1", 1, 10, "64 stations (2016 baselines), 10 timeslots, 1 channel at 150 MHz, "
                             "1 cluster x 20 sources, 10 LM"),
    "consensus16": ("consensus", 1, 10, "16 sub-bands tiling 115-185 MHz, each 128 stations (8128 baselines), "
                                        "10 timeslots, 2 channels, 10 clusters x 25 sources; Jones drifting "
                                        "linearly across the band; consensus ADMM on a 3-term frequency model, "
                                        "3 iterations of 1 SAGE sweep x 10 LM per band"),
    "serve500": ("c5", 3, 10, "Poisson-arriving calibration jobs: stations uniform in {64,128,256,384,512}, "
                              "clusters 1-40 x 25 sources, 5-20 timeslots, 1-8 channels 140-160 MHz, 3 SAGE "
                              "sweeps x 10 LM, continuous batching with HBM-footprint admission"),
    "chunks128": ("c2", 1, 10, "one 128-station sub-band (8128 baselines, 8 channels 140-160 MHz, 10 clusters x "
                               "25 sources) in 6 consecutive chunks of 20 timeslots, gains drifting between "
                               "chunks; each chunk 1 SAGE sweep x 10 LM warm-started from the previous chunk, "
                               "all chunks in one sc_calibrate_chunks call"),
    "batch64": ("c3", 3, 10, "64 sub-band jobs of 256 stations (32640 baselines), timeslots uniform in 5-40 "
                             "per job, 1 channel, 20 clusters x 50 sources, 3 SAGE sweeps x 10 LM, all jobs "
                             "in one sc_calibrate_batched call (lock step: one launch per LM stage for all "
                             "jobs)"),
}


def job_seed(rank: int, i: int = 0) -> int:
    """Seed of job i on rank `rank`: every rank calibrates its own, distinct
    sub-band jobs (no data is shared between ranks)."""
    return 1000 * rank + i


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The slowest rank's time: all_reduce(MAX) of one float (any backend)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sm_count() -> int:
    """Multiprocessors of the current CUDA device."""
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def fp32_peak_tflops(sm_mhz: float) -> float:
    """FP32 FMA peak: SMs x 128 lanes x 2 flops x SM clock (no measured FP32
    figure exists, so it is derived from the unit counts)."""
    return sm_count() * 128 * 2 * sm_mhz * 1e6 / 1e12


def fp32_peak_source(sm_mhz: float) -> str:
    return "FP32 FMA: %d SMs x 128 lanes x 2 flops x %.0f MHz" % (sm_count(), sm_mhz)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


# --- the FP64 CPU oracle on a bounded sample (cpu_baseline and --impl reference) -------------

def oracle_sample(n_lm=1, N=512, S=100, seed=0):
    """Times the oracle (as it stands) on a bounded sample of the workload:
    N stations, 1 timeslot, 1 channel, one cluster of S sources: prediction
    plus LM with n_lm trial steps.  Returns (units, seconds, description)."""
    import oracle as O
    spec = synth.JobSpec(N=N, T=1, F=1, K=1, S=S, f_lo=150e6, f_hi=150e6, seed=seed)
    uvw, f, sky = synth.station_uvw(spec), synth.freqs(spec), synth.sky(spec)
    Jt = synth.jones_true(spec)
    t0 = time.perf_counter()
    C = O.predict_coherencies(uvw, f, sky.l, sky.m, sky.flux, sky.alpha)
    V = O.model_vis(C, Jt[0]) + synth.noise(spec)
    O.lm_cluster(V, C, synth.identity_jones(1, N)[0], n_lm, eps_grad=0.0)
    dt = time.perf_counter() - t0
    units = spec.B * spec.T * spec.F * 1 * n_lm
    desc = ("oracle (numpy FP64) on %d stations x 1 timeslot x 1 channel, 1 cluster x %d sources: "
            "predict + LM with %d trial step(s); numpy elementwise work single-threaded, "
            "LAPACK Cholesky on the BLAS thread pool" % (N, S, n_lm))
    return units, dt, desc


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# --- clocks during the timed region ------------------------------------------------------------

class ClockSampler:
    """nvidia-smi clock and throttle samples every 200 ms while the timed
    region runs, written as CSV to $BENCH_CLOCKS_DIR (default: the system
    temporary directory) and summarised into the JSON line."""

    def __init__(self, index):
        self.proc = None
        folder = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(folder, "bench_clocks_%d.csv" % os.getpid())
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            c = [x.strip() for x in line.split(",")]
            if len(c) < 9:
                continue
            try:
                sm.append(float(c[1]))
                mx.append(float(c[2]))
            except ValueError:
                continue
            for n, v in zip(names, c[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --- our arm ---------------------------------------------------------------------------------------

def make_job(spec, prec, dev):
    """Device-resident inputs of one job.  The observed visibilities are
    simulated with the library's own prediction (true Jones, thermal noise);
    they are inputs here, not results."""
    import torch
    from paper_1910_13908_gb300 import sagecal as sc
    uvw = torch.as_tensor(synth.station_uvw(spec)).to(dev)
    freqs = torch.as_tensor(synth.freqs(spec)).to(dev)
    sky = synth.sky(spec)
    dsky = sc.DeviceSky.from_synth(sky, dev)
    shp = sc.Shape(spec.N, spec.T, spec.F, spec.K, spec.S)
    ws = sc.workspace(shp, prec, dev)
    C = sc.predict_coherencies(shp, uvw, freqs, dsky, prec, ws)
    Jt = torch.as_tensor(synth.jones_true(spec)).to(dev)
    p, q = np.triu_indices(spec.N, 1)
    cdt = C.dtype
    V = torch.zeros((spec.T, spec.B, spec.F, 2, 2), dtype=cdt, device=dev)
    for k in range(spec.K):
        G = (Jt[k, p] @ Jt[k, q].conj().transpose(-1, -2)).to(cdt)          # [B][2][2]
        V += C[k][..., None, None] * G[None, :, None]
    del C
    g = torch.Generator(device=dev)
    g.manual_seed(1234 + spec.seed)
    rdt = torch.float32 if cdt == torch.complex64 else torch.float64
    noise = torch.randn((*V.shape, 2), generator=g, device=dev, dtype=rdt) * spec.sigma
    V += torch.view_as_complex(noise)
    J0 = torch.as_tensor(synth.identity_jones(spec.K, spec.N)).to(dev)
    return dict(shape=shp, uvw=uvw, freqs=freqs, sky=dsky, V=V.contiguous(), J0=J0, ws=ws,
                sky_host=sky)


def roofline_for(kind, spec, prec, n_em, n_lm, launches, ms, pk, peak_src):
    """Algorithmic work of one launch of the dominant kernel kind."""
    from paper_1910_13908_gb300 import sagecal as sc
    P = 8 * spec.N
    Ppad = (P + 63) // 64 * 64
    vis = spec.B * spec.T * spec.F
    rs = 4 if prec == sc.SC_MIXED else 8
    avg_s = (ms / 1e3) / max(launches, 1)
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    if kind == "cholesky":
        work = P ** 3 / 3.0                         # flops of L L^T = A
        if prec == sc.SC_MIXED:
            peak = fp32_peak_tflops(sm_mhz)   # FP32 FMA lanes x 2 flops x clock
            return dict(bound="alu", achieved=work / avg_s / 1e12, peak=peak, unit="TFLOP/s",
                        peak_source=fp32_peak_source(sm_mhz))
        peak = 1.25
        return dict(bound="alu", achieved=work / avg_s / 1e12, peak=peak, unit="TFLOP/s",
                    peak_source="FP64 nominal 1.25 TFLOP/s")
    if kind == "lm_stats":
        work = vis * (4 * 2 * rs + 2 * rs)               # read the data (2x2 complex) + coherency, once per solve
        return dict(bound="hbm", achieved=work / avg_s / 1e9, peak=pk["hbm_gbs"], unit="GB/s",
                    peak_source=peak_src)
    if kind == "vis_pass":
        work = vis * (2 * 4 * 2 * rs + 2 * rs)           # read and write the running residual, read the coherency
        return dict(bound="hbm", achieved=work / avg_s / 1e9, peak=pk["hbm_gbs"], unit="GB/s",
                    peak_source=peak_src)
    if kind == "jhj_assemble":
        work = Ppad * (Ppad + 4) / 2 * rs               # lower triangle written
        return dict(bound="hbm", achieved=work / avg_s / 1e9, peak=pk["hbm_gbs"], unit="GB/s",
                    peak_source=peak_src)
    if kind == "tri_solve":
        work = Ppad * Ppad * rs                          # L read once forward, once backward (half each)
        return dict(bound="hbm", achieved=work / avg_s / 1e9, peak=pk["hbm_gbs"], unit="GB/s",
                    peak_source=peak_src)
    if kind == "coherency":
        work = 8.0 * vis * spec.S                        # one complex multiply-add per (source, vis)
        peak = fp32_peak_tflops(sm_mhz)
        return dict(bound="alu", achieved=work / avg_s / 1e12, peak=peak, unit="TFLOP/s",
                    peak_source=fp32_peak_source(sm_mhz))
    return dict(bound="latency", achieved=None, peak=None, unit=None)


def measure_residual_output(job, spec, prec, J, reps, pk, src, workload):
    """The output that follows calibration: the residual of all K clusters
    with the calibrated Jones, corrected towards cluster 0 (sc_residual_all),
    timed on its own after the calibration steps.  HBM-bound: per visibility
    it reads V and the K coherencies and writes R once."""
    import torch
    from paper_1910_13908_gb300 import sagecal as sc
    C = sc.predict_coherencies(job["shape"], job["uvw"], job["freqs"], job["sky"], prec, job["ws"])
    R = torch.empty_like(job["V"])
    for _ in range(2):
        sc.residual_all(job["shape"], job["V"], C, J, prec, job["ws"], corr=0, out=R)
    torch.cuda.synchronize()
    sc.profile_begin()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        _, cost = sc.residual_all(job["shape"], job["V"], C, J, prec, job["ws"], corr=0, out=R)
    e1.record()
    torch.cuda.synchronize()
    prof = sc.profile_end()
    status = sc.device_status(job["ws"])
    n, kms = prof["vis_pass"]
    rs = 4 if prec == sc.SC_MIXED else 8
    vis = spec.B * spec.T * spec.F
    work = vis * (8 * rs + 2 * rs * spec.K + 8 * rs)     # read V, read C of every cluster, write R
    avg_s = kms / 1e3 / max(n, 1)
    achieved = work / avg_s / 1e9
    del C, R
    return {"call": "sc_residual_all", "corr": 0, "launches": n,
            "avg_launch_us": round(avg_s * 1e6, 2), "call_ms": round(e0.elapsed_time(e1) / reps, 4),
            "vis_per_s": vis / avg_s, "bytes_per_launch": int(work),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / pk["hbm_gbs"], "traffic": NCU_TRAFFIC.get(("residual_all", workload)),
                         "peak_kind": src},
            "cost": float(cost.item()), "device_status": status}


FLOPS_PER_POL_TERM = 22      # per (source, vis): e_p conj(e_q) (6) + 4 complex-by-real FMAs (16)
FLOPS_PER_GAUSS_TERM = 10    # more per extended (source, vis): quadratic form (7) + attenuation (2) + 1


def measure_predict_full(job, spec, prec, reps, pk):
    """Polarised, Gaussian-extended prediction of every cluster
    (sc_predict_coherencies_full) on the workload's sky with Stokes Q, U, V
    and 30% of the sources Gaussian (synth.sky_pol), timed on its own.
    ALU-bound: one complex product, four complex FMAs and, for an extended
    source, one exponential per (source, vis)."""
    import torch
    from paper_1910_13908_gb300 import sagecal as sc
    sky = synth.sky_pol(spec)
    dsky = sc.DeviceSkyFull.from_synth(sky, job["V"].device)
    out = sc.predict_coherencies_full(job["shape"], job["uvw"], job["freqs"], dsky, prec, job["ws"])
    torch.cuda.synchronize()
    sc.profile_begin()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        sc.predict_coherencies_full(job["shape"], job["uvw"], job["freqs"], dsky, prec, job["ws"], out=out)
    e1.record()
    torch.cuda.synchronize()
    prof = sc.profile_end()
    status = sc.device_status(job["ws"])
    n, kms = prof["coherency"]
    vis = spec.B * spec.T * spec.F
    n_src = int(sky.offsets[-1])
    n_ext = int(np.count_nonzero((sky.maj != 0) | (sky.mnr != 0)))
    terms = vis * n_src                                   # (source, vis) pairs of one call
    flops = terms * FLOPS_PER_POL_TERM + vis * n_ext * FLOPS_PER_GAUSS_TERM
    kern_s = kms / 1e3 / max(reps, 1)                     # contraction time of one call (all clusters)
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    peak = fp32_peak_tflops(sm_mhz)
    del out
    return {"call": "sc_predict_coherencies_full", "clusters": sky.K, "sources": n_src, "extended": n_ext,
            "call_ms": round(e0.elapsed_time(e1) / reps, 4), "contraction_launches": n,
            "contraction_ms_per_call": round(kern_s * 1e3, 4), "source_terms_per_s": terms / kern_s,
            "roofline": {"bound": "alu", "achieved": flops / kern_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                         "frac": flops / kern_s / 1e12 / peak,
                         "peak_source": fp32_peak_source(sm_mhz),
                         "flops_per_term": FLOPS_PER_POL_TERM, "extra_flops_per_extended_term":
                         FLOPS_PER_GAUSS_TERM, "traffic": None},
            "device_status": status}


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one
# ncu capture of the float32 kernel as it stands (profiles/), by (kernel kind,
# workload); a kernel changed since its capture has no entry.
NCU_TRAFFIC = {
    ("cholesky", "ska512"): 38.4e6,     # k_chol<float>, order 4096; the factor stays in L2 between reads
    ("vis_pass", "ska512"): 321e6,      # k_pass_col32 (P_OLD | P_SUB | P_WRITE_R); part of R is read from L2
}


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1910_13908_gb300 import sagecal as sc
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    sc.lib()
    cfg, n_em, n_lm, desc = WORKLOADS[args.workload]
    spec = synth.config(cfg, seed=job_seed(rank))
    prec = sc.SC_FP64 if args.prec == "fp64" else sc.SC_MIXED
    job = make_job(spec, prec, dev)
    J = job["J0"].clone()
    costs = torch.zeros((spec.K,), dtype=torch.float64, device=dev)
    units = spec.B * spec.T * spec.F * spec.K * n_lm * n_em

    def step():
        J.copy_(job["J0"])
        sc.calibrate_sage(job["shape"], job["uvw"], job["freqs"], job["sky"], job["V"], J, prec,
                          job["ws"], n_em=n_em, n_lm=n_lm, refine_sweeps=args.refine, costs=costs)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if sc.device_status(job["ws"]) & 2:
        raise RuntimeError("device wait timed out during warm-up")
    barrier()
    torch.cuda.synchronize()
    flush = l2_flusher(job, dev)
    clocks = ClockSampler(local_rank)
    n0 = sc.launch_count()
    sc.profile_begin()
    ms = timed_steps(step, args.steps, flush)
    barrier()
    prof = sc.profile_end()
    n_launch = sc.launch_count() - n0
    clk = clocks.stop()
    ms = max_over_ranks(ms, world, dev)
    value = units * args.steps * world / (ms / 1e3)
    final_costs = costs.cpu().numpy().tolist()

    # the same step replayed from a captured CUDA graph, against direct calls,
    # both without the per-kernel timing events
    graph = None
    if not args.no_graph:
        graph = measure_graph(job, spec, prec, J, costs, n_em, n_lm, args, units, flush, world, dev)

    # end to end through the public API: host inputs (pinned) -> device -> result back
    e2e = None
    if not args.no_e2e:
        hV = job["V"].cpu().pin_memory()
        hu, hf = job["uvw"].cpu().pin_memory(), job["freqs"].cpu().pin_memory()
        hs = {k: getattr(job["sky"], k).cpu().pin_memory() for k in ("l", "m", "flux", "alpha")}
        hJ0 = job["J0"].cpu().pin_memory()
        hJ = torch.empty_like(hJ0).pin_memory()
        hc = torch.empty((spec.K,), dtype=torch.float64).pin_memory()
        dV, du, df = torch.empty_like(job["V"]), torch.empty_like(job["uvw"]), torch.empty_like(job["freqs"])
        ds = {k: torch.empty_like(v, device=dev) for k, v in hs.items()}
        dJ = torch.empty_like(job["J0"])
        dsky = sc.DeviceSky(ds["l"], ds["m"], ds["flux"], ds["alpha"], job["sky"].offsets, job["sky"].f0)
        bi = sum(t.numel() * t.element_size() for t in [hV, hu, hf, hJ0, *hs.values()])
        bo = hJ.numel() * hJ.element_size() + hc.numel() * hc.element_size()

        def e2e_step():
            dV.copy_(hV, non_blocking=True)
            du.copy_(hu, non_blocking=True)
            df.copy_(hf, non_blocking=True)
            for k in ds:
                ds[k].copy_(hs[k], non_blocking=True)
            dJ.copy_(hJ0, non_blocking=True)
            sc.calibrate_sage(job["shape"], du, df, dsky, dV, dJ, prec, job["ws"], n_em=n_em, n_lm=n_lm,
                              refine_sweeps=args.refine, costs=costs)
            hJ.copy_(dJ, non_blocking=True)
            hc.copy_(costs, non_blocking=True)
        e2e_step()
        torch.cuda.synchronize()
        barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ks = max(1, min(args.steps, 3))
        f0.record()
        for _ in range(ks):
            e2e_step()
        f1.record()
        torch.cuda.synchronize()
        ems = max_over_ranks(f0.elapsed_time(f1), world, dev)
        e2e = {"value": units * ks * world / (ems / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(bi),
               "d2h_bytes_per_step": int(bo), "steps": ks}

    # the plain FP64 GPU path and the mixed path on the same bounded sample
    fp64 = None
    if not args.no_fp64 and rank == 0:
        fp64 = compare_fp64(spec, dev, args)

    pk, src = peaks()
    resid = None
    if not args.no_residual:
        resid = measure_residual_output(job, spec, prec, J, 5, pk, src, args.workload)
    pol = None
    if not args.no_pol:
        pol = measure_predict_full(job, spec, prec, 3, pk)
    dominant = max(prof, key=lambda k: prof[k][1])
    n_dom, ms_dom = prof[dominant]
    roof = roofline_for(dominant, spec, prec, n_em, n_lm, n_dom, ms_dom, pk, src)
    if roof.get("achieved") is not None and roof.get("peak"):
        roof["frac"] = roof["achieved"] / roof["peak"]
    roof["kernel"] = dominant
    roof["launches"] = n_dom
    roof["avg_launch_us"] = 1e3 * ms_dom / max(n_dom, 1)
    roof["share_of_step"] = ms_dom / ms if ms > 0 else None
    roof["traffic"] = NCU_TRAFFIC.get((dominant, args.workload)) if args.prec == "mixed" else None
    roof["peak_kind"] = src
    breakdown = {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in prof.items() if v[0]}
    # the streaming kernels' own rooflines (HBM-bound)
    streaming = {}
    for k in ("lm_stats", "vis_pass"):
        if prof.get(k, (0, 0))[0]:
            r = roofline_for(k, spec, prec, n_em, n_lm, prof[k][0], prof[k][1], pk, src)
            r["frac"] = r["achieved"] / r["peak"]
            r["avg_launch_us"] = 1e3 * prof[k][1] / prof[k][0]
            r["launches"] = prof[k][0]
            r["traffic"] = NCU_TRAFFIC.get((k, args.workload)) if args.prec == "mixed" else None
            streaming[k] = r

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        u, dt, d = oracle_sample(n_lm=2)
        cpu = {"value": u / dt, "unit": UNIT, "cores": host_cores(), "kind": "oracle", "sample": d,
               "seconds": round(dt, 2)}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == sc.SC_MIXED else "f64",
        "data": "synthetic (seeded stations, sky, Jones and noise shaped like the paper's datasets)",
        "config": {"workload": args.workload, "description": desc, "stations": spec.N,
                   "baselines": spec.B, "timeslots": spec.T, "channels": spec.F, "clusters": spec.K,
                   "sources_per_cluster": spec.S, "n_em": n_em, "n_lm": n_lm,
                   "refine_sweeps": args.refine if prec == sc.SC_MIXED else 0,
                   "precision": args.prec, "parallelism": "one independent job per GPU (replicas)",
                   "l2": "inputs larger than L2 (coherency cache %.2f GB + visibilities %.2f GB per job)"
                         % (spec.K * spec.T * spec.B * spec.F * (8 if prec == sc.SC_MIXED else 16) / 1e9,
                            spec.T * spec.B * spec.F * (32 if prec == sc.SC_MIXED else 64) / 1e9)},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(n_launch),
        "clocks": clk,
        "fp64_gpu": fp64,
        "residual_output": resid,
        "predict_full": pol,
        "graph": graph,
        "kernel_ms": breakdown,
        "streaming": streaming,
        "final_costs_head": final_costs[:4],
    }
    if flush is not None:
        line["config"]["l2"] = ("inputs and workspace (%.1f MB) under twice L2: a %d MB buffer is written "
                                "between timed steps, outside the per-step events"
                                % (job_bytes(job) / 1e6, L2_FLUSH_MB))
    if rank == 0:
        print(json.dumps(line))


L2_BYTES = 129 * 2 ** 20
L2_FLUSH_MB = 512


def job_bytes(job):
    return sum(t.numel() * t.element_size() for t in (job["V"], job["uvw"], job["ws"]))


def l2_flusher(job, dev):
    """A function that evicts L2 by writing a buffer larger than it, when the
    job's inputs and workspace are not already larger than L2; else None."""
    if job_bytes(job) > 2 * L2_BYTES:
        return None
    import torch
    buf = torch.empty(L2_FLUSH_MB * 2 ** 20, dtype=torch.uint8, device=dev)
    return lambda: buf.fill_(1)


def timed_steps(step, n, flush):
    """Device time (ms) of n calls of step(), CUDA events on the current
    stream.  Without a flush: one event pair around all steps.  With one:
    L2 is flushed before every step, outside that step's event pair."""
    import torch
    torch.cuda.synchronize()
    if flush is None:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(n):
            step()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    for a, b in ev:
        flush()
        a.record()
        step()
        b.record()
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev)


def measure_graph(job, spec, prec, J, costs, n_em, n_lm, args, units, flush, world, dev):
    """Times direct sc_calibrate_sage calls and replays of the same call
    captured once as a CUDA graph (sc_graph_capture_sage), each over the
    same number of steps, and checks that a replay gives the direct call's
    result bit for bit."""
    import torch
    from paper_1910_13908_gb300 import sagecal as sc
    ks = max(1, min(args.steps, 3))

    def direct():
        J.copy_(job["J0"])
        sc.calibrate_sage(job["shape"], job["uvw"], job["freqs"], job["sky"], job["V"], J, prec,
                          job["ws"], n_em=n_em, n_lm=n_lm, refine_sweeps=args.refine, costs=costs)

    direct()
    torch.cuda.synchronize()
    J_ref, c_ref = J.clone(), costs.clone()
    ms_d = max_over_ranks(timed_steps(direct, ks, flush), world, dev)
    g = sc.capture_sage(job["shape"], job["uvw"], job["freqs"], job["sky"], job["V"], J, prec, job["ws"],
                        costs, n_em=n_em, n_lm=n_lm, refine_sweeps=args.refine)

    def replay():
        J.copy_(job["J0"])
        g.launch()

    replay()
    torch.cuda.synchronize()
    same = bool(torch.equal(J, J_ref) and torch.equal(costs, c_ref))
    n0 = sc.launch_count()
    ms_g = max_over_ranks(timed_steps(replay, ks, flush), world, dev)
    per_step = (sc.launch_count() - n0) // ks
    g.close()
    return {"value": units * ks * world / (ms_g / 1e3), "unit": UNIT, "ms_per_step": ms_g / ks,
            "direct_value": units * ks * world / (ms_d / 1e3), "direct_ms_per_step": ms_d / ks,
            "speedup_over_direct": ms_d / ms_g, "kernels_per_step": int(per_step), "steps": ks,
            "replay_equals_direct": same}


def run_batch(args, rank, world, local_rank):
    """One step = one sc_calibrate_batched call over 64 uneven jobs (lock
    step: one launch per LM stage for every job).  The same jobs enqueued
    job by job on their own streams (sc_calibrate_batch) are timed beside
    it."""
    import torch
    from paper_1910_13908_gb300 import sagecal as sc
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    cfg, n_em, n_lm, desc = WORKLOADS["batch64"]
    prec = sc.SC_FP64 if args.prec == "fp64" else sc.SC_MIXED
    n_jobs = args.jobs
    Ts = synth.uneven_time_chunks(n_jobs, 5, 40, seed=rank)
    jobs, J0s, units = [], [], 0
    for i in range(n_jobs):
        spec = synth.config("c3", seed=job_seed(rank, i))
        spec.T = int(Ts[i])
        job = make_job(spec, prec, dev)
        jobs.append(sc.Job(shape=job["shape"], uvw=job["uvw"], freqs=job["freqs"], sky=job["sky"], V=job["V"],
                           jones=job["J0"].clone(), costs=torch.zeros(spec.K, dtype=torch.float64, device=dev),
                           ws=job["ws"], stream=torch.cuda.Stream(dev)))
        J0s.append(job["J0"])
        units += spec.B * spec.T * spec.F * spec.K * n_lm * n_em
    bws = sc.batched_workspace(jobs, prec, dev)
    # the factorisation's task order, measured (untimed): staggered windows
    # against the interleave (a window above the whole merged list)
    window, tune_ms = sc.tune_batched(jobs, prec, bws, windows=(4, 16, 64, 1 << 20))
    if window == 1 << 20:
        window = 0                   # the interleave itself, without an order table
    torch.cuda.synchronize()

    def step(lockstep=True):
        for j, j0 in zip(jobs, J0s):
            j.jones.copy_(j0)
        torch.cuda.synchronize()
        if lockstep:
            sc.calibrate_batched(jobs, prec, bws, n_em=n_em, n_lm=n_lm, refine_sweeps=args.refine, window=window)
        else:
            sc.calibrate_batch(jobs, prec, n_em=n_em, n_lm=n_lm, refine_sweeps=args.refine)
        torch.cuda.synchronize()

    # the per-job-stream variant, for comparison (untimed warm-up, then one step)
    step(False)
    t0 = time.perf_counter()
    step(False)
    el_streams = time.perf_counter() - t0
    for _ in range(args.warmup):
        step()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clocks = ClockSampler(local_rank)
    n0 = sc.launch_count()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t0
    n_launch = sc.launch_count() - n0
    clk = clocks.stop()
    el = max_over_ranks(el, world, dev)
    value = units * args.steps * world / el
    pk, src = peaks()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == sc.SC_MIXED else "f64",
        "data": "synthetic",
        "config": {"workload": "batch64", "description": desc, "jobs": n_jobs,
                   "timeslots_per_job": [int(t) for t in Ts], "precision": args.prec,
                   "timing": "host wall clock around each batch call with device synchronisation on both "
                             "sides",
                   "batch_workspace_gb": bws.numel() / 1e9,
                   "stagger_window": window,
                   "tuner_ms_per_factorisation": {str(k): round(v, 3) for k, v in tune_ms.items()},
                   "l2": "inputs larger than L2"},
        "streams_variant": {"entry": "sc_calibrate_batch (each job on its own stream, "
                                     "CUDA_DEVICE_MAX_CONNECTIONS=%s)" % os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS"),
                            "value": units * world / max_over_ranks(el_streams, world, dev),
                            "ms_per_step": 1e3 * el_streams},
        "gpu_launches": int(n_launch), "clocks": clk, "peak_kind": src,
    }
    if rank == 0:
        print(json.dumps(line))


N_CHUNKS = 6
CHUNK_DRIFT = 0.05   # rad per chunk: per-station gain phase drift, x_s in [0, 1]


def run_chunks(args, rank, world, local_rank):
    """One step = one sc_calibrate_chunks call over N_CHUNKS consecutive time
    chunks of one sub-band, from identity gains, each chunk warm-started from
    the previous one.  Also reports, outside the timed region, each chunk's
    final cost against a cold start of the same budget and the noise floor."""
    import dataclasses
    import torch
    from paper_1910_13908_gb300 import sagecal as sc
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    sc.lib()
    cfg, n_em, n_lm, desc = WORKLOADS["chunks128"]
    prec = sc.SC_FP64 if args.prec == "fp64" else sc.SC_MIXED
    spec = synth.config(cfg, seed=job_seed(rank))
    n = N_CHUNKS
    full = dataclasses.replace(spec, T=n * spec.T)
    uvw = torch.as_tensor(synth.station_uvw(full)).to(dev)
    freqs = torch.as_tensor(synth.freqs(spec)).to(dev)
    dsky = sc.DeviceSky.from_synth(synth.sky(spec), dev)
    shp = sc.Shape(spec.N, spec.T, spec.F, spec.K, spec.S)
    ws = sc.workspace(shp, prec, dev)
    Jt = torch.as_tensor(synth.jones_true(spec)).to(dev)
    ph = torch.linspace(0.0, 1.0, spec.N, dtype=torch.float64, device=dev)[None, :, None, None]
    p, q = np.triu_indices(spec.N, 1)
    cdt = torch.complex64 if prec == sc.SC_MIXED else torch.complex128
    rdt = torch.float32 if prec == sc.SC_MIXED else torch.float64
    V = torch.zeros((n, spec.T, spec.B, spec.F, 2, 2), dtype=cdt, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(4321 + spec.seed)
    for i in range(n):
        C = sc.predict_coherencies(shp, uvw[i * spec.T:(i + 1) * spec.T].contiguous(), freqs, dsky, prec, ws)
        Ji = Jt * torch.exp(1j * CHUNK_DRIFT * i * ph)
        for k in range(spec.K):
            G = (Ji[k, p] @ Ji[k, q].conj().transpose(-1, -2)).to(cdt)
            V[i] += C[k][..., None, None] * G[None, :, None]
        del C
        V[i] += torch.view_as_complex(torch.randn((*V[i].shape, 2), generator=g, device=dev, dtype=rdt)
                                      * spec.sigma)
    J0 = torch.as_tensor(synth.identity_jones(spec.K, spec.N)).to(dev)
    J = J0.clone()
    units = spec.B * spec.T * spec.F * spec.K * n_lm * n_em * n
    out = {}

    def step():
        J.copy_(J0)
        out["r"] = sc.calibrate_chunks(shp, uvw, freqs, dsky, V, J, prec, ws, n_em=n_em, n_lm=n_lm,
                                       refine_sweeps=args.refine, want_history=True)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clocks = ClockSampler(local_rank)
    n0 = sc.launch_count()
    sc.profile_begin()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    prof = sc.profile_end()
    n_launch = sc.launch_count() - n0
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    value = units * args.steps * world / (ms / 1e3)
    warm = out["r"][2][:, -1].cpu().numpy()          # last cluster: the total residual after the sweep

    # end to end: host data and uvw in, every chunk's solution and costs out
    e2e = None
    if not args.no_e2e:
        hV, hu = V.cpu().pin_memory(), uvw.cpu().pin_memory()
        hH = torch.empty((n, spec.K, spec.N, 2, 2), dtype=torch.complex128).pin_memory()
        hC = torch.empty((n, spec.K), dtype=torch.float64).pin_memory()
        dV, du = torch.empty_like(V), torch.empty_like(uvw)
        bi = hV.numel() * hV.element_size() + hu.numel() * hu.element_size()
        bo = hH.numel() * hH.element_size() + hC.numel() * hC.element_size()

        def e2e_step():
            dV.copy_(hV, non_blocking=True)
            du.copy_(hu, non_blocking=True)
            J.copy_(J0)
            _, hist, costs = sc.calibrate_chunks(shp, du, freqs, dsky, dV, J, prec, ws, n_em=n_em, n_lm=n_lm,
                                                 refine_sweeps=args.refine)
            hH.copy_(hist, non_blocking=True)
            hC.copy_(costs, non_blocking=True)
        e2e_step()
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ks = max(1, min(args.steps, 3))
        f0.record()
        for _ in range(ks):
            e2e_step()
        f1.record()
        torch.cuda.synchronize()
        ems = max_over_ranks(f0.elapsed_time(f1), world, dev)
        e2e = {"value": units * ks * world / (ems / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(bi),
               "d2h_bytes_per_step": int(bo), "steps": ks}

    # cold starts with the same budget, outside the timed region
    cold = []
    for i in range(n):
        Jc = J0.clone()
        _, c = sc.calibrate_sage(shp, uvw[i * spec.T:(i + 1) * spec.T].contiguous(), freqs, dsky, V[i], Jc, prec,
                                 ws, n_em=n_em, n_lm=n_lm, refine_sweeps=args.refine)
        cold.append(float(c[-1].item()))
    chi2 = 8.0 * spec.B * spec.T * spec.F * spec.sigma ** 2   # noise energy of one chunk
    pk, src = peaks()
    dominant = max(prof, key=lambda k: prof[k][1])
    n_dom, ms_dom = prof[dominant]
    roof = roofline_for(dominant, spec, prec, n_em, n_lm, n_dom, ms_dom, pk, src)
    if roof.get("achieved") is not None and roof.get("peak"):
        roof["frac"] = roof["achieved"] / roof["peak"]
    roof.update(kernel=dominant, launches=n_dom, avg_launch_us=1e3 * ms_dom / max(n_dom, 1),
                share_of_step=ms_dom / ms if ms > 0 else None, traffic=None, peak_kind=src)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == sc.SC_MIXED else "f64",
        "data": "synthetic (seeded stations, sky, drifting Jones and noise)",
        "config": {"workload": "chunks128", "description": desc, "chunks": n, "timeslots_per_chunk": spec.T,
                   "stations": spec.N, "channels": spec.F, "clusters": spec.K, "n_em": n_em, "n_lm": n_lm,
                   "drift_rad_per_chunk": CHUNK_DRIFT, "precision": args.prec,
                   "l2": "inputs larger than L2 (visibilities %.2f GB)" % (V.numel() * V.element_size() / 1e9)},
        "roofline": roof, "e2e": e2e, "gpu_launches": int(n_launch), "clocks": clk,
        "warm_start": {"final_cost_warm": [float(x) for x in warm], "final_cost_cold": cold,
                       "noise_floor_chi2": chi2,
                       "note": "cost of the last cluster after each chunk's sweep = total residual energy"},
        "kernel_ms": {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in prof.items() if v[0]},
    }
    if rank == 0:
        print(json.dumps(line))


def serve_spec(i, seed=0):
    """Shape of serving job i (uniform draws from the serving workload)."""
    u = synth.uniform(seed, synth.TAG_JOBS + 2, 5, offset=5 * i)
    N = (64, 128, 256, 384, 512)[min(4, int(u[0] * 5))]
    K = 1 + min(39, int(u[1] * 40))
    T = 5 + min(15, int(u[2] * 16))
    F = 1 + min(7, int(u[3] * 8))
    return synth.JobSpec(N=N, T=T, F=F, K=K, S=25, f_lo=140e6, f_hi=160e6, seed=10000 + i)


def host_job_from_gpu(i, spec, prec, dev):
    """Host arrays of one serving job; its visibilities are simulated on the
    GPU with the library's prediction (an input, not a result)."""
    return staged_to_host(stage_job(i, spec, prec, dev))


def stage_job(i, spec, prec, dev):
    """One serving job's inputs, simulated on the device and kept there until
    the job arrives (no GPU work left for the arrival itself)."""
    job = make_job(spec, prec, dev)
    return dict(i=i, spec=spec, V=job["V"], sky=job["sky_host"])


def staged_to_host(st):
    """The job as it arrives: host arrays (the device copy of V is dropped)."""
    from paper_1910_13908_gb300 import serve
    spec, sky = st["spec"], st["sky"]
    V = st.pop("V").cpu().numpy()
    return serve.HostJob(st["i"], sc_shape(spec), synth.station_uvw(spec), synth.freqs(spec), sky.l, sky.m,
                         sky.flux, sky.alpha, [int(x) for x in sky.offsets], V, synth.identity_jones(spec.K, spec.N))


def sc_shape(spec):
    from paper_1910_13908_gb300 import sagecal as sc
    return sc.Shape(spec.N, spec.T, spec.F, spec.K, spec.S)


def run_serve(args, rank, world, local_rank):
    import queue
    import threading
    import torch
    from paper_1910_13908_gb300 import sagecal as sc, serve
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    cfg, n_em, n_lm, desc = WORKLOADS["serve500"]
    prec = sc.SC_FP64 if args.prec == "fp64" else sc.SC_MIXED
    n_jobs = args.jobs
    specs = [serve_spec(i, seed=rank) for i in range(n_jobs)]
    def work(sp):                                     # vis.cluster.iter of one job (a spec or a shape)
        return sp.N * (sp.N - 1) // 2 * sp.T * sp.F * sp.K * n_lm * n_em

    # capacity of the server: a probe of 48 jobs drawn from the same mix
    # (other seeds), all submitted at once, measured in work per second (the
    # probe's jobs are not the run's, so jobs/s would carry their size)
    def capacity(slots, jobs):
        srv = serve.Server(prec=prec, max_slots=slots, n_em=n_em, n_lm=n_lm, refine_sweeps=args.refine)
        srv.start()
        for hj in jobs:
            srv.submit(hj)
        srv.drain()
        span = srv.stats()["span_s"]
        srv.close()
        return sum(work(hj.shape) for hj in jobs) / span

    n_probe = min(48, n_jobs)
    probe_jobs = [host_job_from_gpu(100000 + i, serve_spec(100000 + i, seed=rank), prec, dev) for i in range(n_probe)]
    cap_single = capacity(1, probe_jobs)              # one job at a time
    cap_slots = capacity(args.slots, probe_jobs)      # the server's own overlap
    del probe_jobs
    mean_work = float(np.mean([work(sp) for sp in specs]))
    rate = args.rate if args.rate > 0 else 0.8 * cap_single / mean_work
    # every job's inputs are simulated on the device before the run (no
    # simulation competes with the server); a producer thread only copies
    # the next few jobs to the host ahead of their arrival
    staged = [stage_job(i, sp, prec, dev) for i, sp in enumerate(specs)]
    torch.cuda.synchronize(dev)
    q = queue.Queue(maxsize=8)

    def produce():
        s = torch.cuda.Stream(dev)
        with torch.cuda.stream(s):
            for i in range(n_jobs):
                q.put(staged_to_host(staged[i]))
    th = threading.Thread(target=produce, daemon=True)
    th.start()
    u = synth.uniform(rank, synth.TAG_JOBS + 3, n_jobs)
    gaps = -np.log(u) / rate
    arrivals = np.cumsum(gaps) - gaps[0]
    srv = serve.Server(prec=prec, max_slots=args.slots, n_em=n_em, n_lm=n_lm, refine_sweeps=args.refine)
    clocks = ClockSampler(local_rank)
    n0 = sc.launch_count()
    srv.start()
    i = 0
    while i < n_jobs or srv.step():
        while i < n_jobs and srv.now() >= arrivals[i]:
            srv.submit(q.get())
            i += 1
        srv.step()
        time.sleep(0.0005)
    st = srv.stats()
    n_launch = sc.launch_count() - n0
    clk = clocks.stop()
    # where the latency goes: waiting for admission (queueing) against being
    # on the device (service), and the tail by job size
    done = [(srv.results[j], specs[j]) for j in sorted(srv.results) if srv.results[j].outcome == "done"]
    wait = np.array([r.admitted - r.arrival for r, _ in done])
    service = np.array([r.finished - r.admitted for r, _ in done])
    lat = wait + service
    wjob = np.array([work(sp) for _, sp in done], dtype=np.float64)
    tail = lat >= np.percentile(lat, 95)
    breakdown = {
        "queue_wait_s": {"p50": float(np.percentile(wait, 50)), "p99": float(np.percentile(wait, 99))},
        "service_s": {"p50": float(np.percentile(service, 50)), "p99": float(np.percentile(service, 99))},
        "tail_5pct": {"mean_queue_wait_s": float(wait[tail].mean()), "mean_service_s": float(service[tail].mean()),
                      "mean_work_vs_median_job": float(wjob[tail].mean() / np.median(wjob)),
                      "stations": sorted(int(sp.N) for (r, sp), t in zip(done, tail) if t)},
        "latency_by_stations_p50_s": {str(n): float(np.median(lat[[sp.N == n for _, sp in done]]))
                                      for n in (64, 128, 256, 384, 512)
                                      if any(sp.N == n for _, sp in done)},
    }
    srv.close()
    units = sum(work(sp) for sp in specs)
    value = units / st["span_s"]
    line = {
        "metric": METRIC + "; serving p50/p99 solve latency", "value": value, "unit": UNIT, "n_gpus": world,
        "steps": 1, "warmup": 0, "ms_per_step": 1e3 * st["span_s"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if prec == sc.SC_MIXED else "f64", "data": "synthetic",
        "config": {"workload": "serve500", "description": desc, "jobs": n_jobs, "slots": args.slots,
                   "arrival_rate_hz": rate, "mean_job_work": mean_work,
                   "capacity_single_stream": cap_single, "capacity_%d_slots" % args.slots: cap_slots,
                   "capacity_unit": UNIT,
                   "offered_load_vs_%d_slots" % args.slots: rate * mean_work / cap_slots,
                   "rate_rule": ("0.8 x the measured single-stream capacity (%d jobs of the same mix, one at a "
                                 "time, in work per second) / the mean work of the %d jobs" % (n_probe, n_jobs))
                   if args.rate <= 0 else "given",
                   "inputs": "simulated on the device before the run; copied to the host just ahead of arrival"},
        "serving": {"p50_latency_s": st["p50_s"], "p99_latency_s": st["p99_s"], "mean_latency_s": st["mean_s"],
                    "jobs_per_s": st["jobs_per_s"], "failed_jobs": st["failed"],
                    "cancelled_jobs": st["cancelled"], "max_device_bytes_admitted": int(srv.max_used),
                    "budget_bytes": int(srv.mem_budget), "latency_breakdown": breakdown},
        "gpu_launches": int(n_launch), "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line))


def aligned_error(J, Jt):
    """max over stations of |J_p U - Jt_p|_F / |Jt_p|_F after the unitary U
    that best maps J onto Jt (orthogonal Procrustes by SVD): the solution's
    error with the gauge the unpolarised sky leaves free removed."""
    M = np.einsum("pji,pjk->ik", J.conj(), Jt)
    u, _, vh = np.linalg.svd(M)
    U = u @ vh
    return float(np.max(np.linalg.norm(J @ U - Jt, axis=(1, 2)) / np.linalg.norm(Jt, axis=(1, 2))))


def run_consensus(args, rank, world, local_rank):
    """Consensus across sub-bands: the bands' J-steps run at once on internal
    streams (a workspace of several band workspaces) or one after another."""
    import torch
    from paper_1910_13908_gb300 import sagecal as sc
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    _, n_em, n_lm, desc = WORKLOADS["consensus16"]
    prec = sc.SC_FP64 if args.prec == "fp64" else sc.SC_MIXED
    n_bands, n_poly, n_admm, rho = 16, 3, 3, 1.0e4
    spec = synth.JobSpec(N=128, T=10, F=2, K=10, S=25, seed=job_seed(rank))
    fr, centres = synth.sub_bands(spec, n_bands)
    basis = synth.frequency_basis(centres, n_poly)
    Jt = synth.jones_true_bands(spec, centres)                       # [n_bands][K][N][2][2]
    shp = sc.Shape(spec.N, spec.T, spec.F, spec.K, spec.S)
    uvw = torch.as_tensor(synth.station_uvw(spec)).to(dev)
    sky = synth.sky(spec)
    dsky = sc.DeviceSky.from_synth(sky, dev)
    cdt = torch.complex64 if prec == sc.SC_MIXED else torch.complex128
    rdt = torch.float32 if prec == sc.SC_MIXED else torch.float64
    ws1 = sc.workspace(shp, prec, dev)
    p, q = np.triu_indices(spec.N, 1)
    V = torch.zeros((n_bands, spec.T, spec.B, spec.F, 2, 2), dtype=cdt, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(4321 + spec.seed)
    for f in range(n_bands):                       # inputs: the library's prediction, true Jones, noise
        C = sc.predict_coherencies(shp, uvw, torch.as_tensor(fr[f]).to(dev), dsky, prec, ws1)
        Jf = torch.as_tensor(Jt[f]).to(dev)
        for k in range(spec.K):
            G = (Jf[k, p] @ Jf[k, q].conj().transpose(-1, -2)).to(cdt)
            V[f] += C[k][..., None, None] * G[None, :, None]
        V[f] += torch.view_as_complex(torch.randn((*V[f].shape, 2), generator=g, device=dev, dtype=rdt) * spec.sigma)
        del C
    del ws1
    dfr = torch.as_tensor(fr).to(dev)
    dbasis = torch.as_tensor(basis).to(dev)
    J0 = torch.as_tensor(np.broadcast_to(np.eye(2, dtype=complex), Jt.shape).copy()).to(dev)
    conc = n_bands
    ws = sc.consensus_workspace(shp, prec, conc, dev)

    def run(w, r):
        J = J0.clone()
        sc.calibrate_consensus(shp, uvw, dfr, dsky, V, dbasis, J, prec, w, r, n_admm=n_admm, n_em=n_em, n_lm=n_lm,
                               refine_sweeps=args.refine)
        return J

    def timed(w, r, k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(k):
            J = run(w, r)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k, J

    for _ in range(args.warmup):
        run(ws, rho)
    clocks = ClockSampler(local_rank)
    n0 = sc.launch_count()
    ms, J = timed(ws, rho, args.steps)
    n_launch = (sc.launch_count() - n0) // max(args.steps, 1)
    clk = clocks.stop()
    ms_seq, _ = timed(ws[: (sc.workspace_size(shp, prec) + 255) // 256 * 256], rho, 1)
    _, J_ind = timed(ws, 0.0, 1)                  # rho = 0: each band alone
    Jh, Jih = J.cpu().numpy(), J_ind.cpu().numpy()
    err = np.array([[aligned_error(Jh[f, k], Jt[f, k]) for k in range(spec.K)] for f in range(n_bands)])
    err_ind = np.array([[aligned_error(Jih[f, k], Jt[f, k]) for k in range(spec.K)] for f in range(n_bands)])
    units = n_bands * spec.B * spec.T * spec.F * spec.K * n_lm * n_em * n_admm
    line = {
        "metric": METRIC, "value": units * world / (ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if prec == sc.SC_MIXED else "f64", "data": "synthetic",
        "config": {"workload": "consensus16", "description": desc, "bands": n_bands, "stations": spec.N,
                   "baselines": spec.B, "timeslots": spec.T, "channels_per_band": spec.F, "clusters": spec.K,
                   "sources_per_cluster": spec.S, "n_poly": n_poly, "rho": rho, "n_admm": n_admm,
                   "concurrent_bands": conc, "l2": "inputs larger than L2 (%.2f GB of visibilities)"
                   % (V.numel() * V.element_size() / 1e9)},
        "consensus": {"ms_per_call_concurrent": ms, "ms_per_call_sequential": ms_seq,
                      "speedup_concurrent": ms_seq / ms,
                      "jones_error_consensus": {"median": float(np.median(err)), "max": float(err.max())},
                      "jones_error_independent": {"median": float(np.median(err_ind)), "max": float(err_ind.max())},
                      "error_measure": "max over stations of |J_p U - J_true,p| / |J_true,p| after Procrustes U, "
                                       "per band and cluster"},
        "gpu_launches": int(n_launch), "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line))


def compare_fp64(spec, dev, args):
    """vis.cluster/s per LM iteration of the plain FP64 GPU path and of the
    mixed path on one bounded sample of the same job: all stations,
    timeslots and channels, one cluster, one SAGE sweep of 10 LM iterations."""
    import torch
    from paper_1910_13908_gb300 import sagecal as sc
    sub = synth.JobSpec(**{**spec.__dict__, "K": 1})
    out = {}
    for name, prec in (("fp64", sc.SC_FP64), ("mixed", sc.SC_MIXED)):
        job = make_job(sub, prec, dev)
        J = job["J0"].clone()

        def go():
            J.copy_(job["J0"])
            sc.calibrate_sage(job["shape"], job["uvw"], job["freqs"], job["sky"], job["V"], J, prec, job["ws"],
                              n_em=1, n_lm=10, refine_sweeps=args.refine)
        go()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        go()
        e1.record()
        torch.cuda.synchronize()
        out[name] = sub.B * sub.T * sub.F * 10 / (e0.elapsed_time(e1) / 1e3)
        del job
        torch.cuda.empty_cache()
    return {"value": out["fp64"], "unit": UNIT, "mixed_same_sample": out["mixed"],
            "speedup_mixed_over_fp64": out["mixed"] / out["fp64"],
            "sample": "%d stations x %d timeslots x %d channels, 1 cluster x %d sources, 1 sweep x 10 LM "
                      "(predict included)" % (sub.N, sub.T, sub.F, sub.S)}


# --- reference arm: the FP64 CPU oracle -------------------------------------------------------------

def run_reference(args, rank, world):
    if rank != 0:
        return
    cfg, n_em, n_lm, desc = WORKLOADS[args.workload]
    for _ in range(args.warmup):
        oracle_sample(n_lm=1)
    tot_u, tot_t, d = 0, 0.0, ""
    for _ in range(args.steps):
        u, dt, d = oracle_sample(n_lm=1)
        tot_u += u
        tot_t += dt
    value = tot_u / tot_t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "description": desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": host_cores(), "sample": d},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ska512", choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--refine", type=int, default=1)
    ap.add_argument("--no-cpu", action="store_true", help="skip the timed oracle sample")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 GPU comparison")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end measurement")
    ap.add_argument("--no-graph", action="store_true", help="skip the CUDA-graph replay measurement")
    ap.add_argument("--no-pol", action="store_true",
                    help="skip the timed polarised, extended-source prediction (sc_predict_coherencies_full)")
    ap.add_argument("--no-residual", action="store_true",
                    help="skip the timed residual output (sc_residual_all) after the steps")
    ap.add_argument("--jobs", type=int, default=0, help="jobs of the batch64 (64) / serve500 (500) workloads")
    ap.add_argument("--slots", type=int, default=8, help="concurrent jobs of the serving workload")
    ap.add_argument("--rate", type=float, default=0.0, help="serving arrival rate (Hz); 0 = 0.8 x capacity")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        if args.workload == "batch64":
            args.jobs = args.jobs or 64
            run_batch(args, rank, world, local_rank)
        elif args.workload == "chunks128":
            run_chunks(args, rank, world, local_rank)
        elif args.workload == "serve500":
            args.jobs = args.jobs or 500
            run_serve(args, rank, world, local_rank)
        elif args.workload == "consensus16":
            run_consensus(args, rank, world, local_rank)
        else:
            run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
