"""Benchmark: emitting particle-steps/s of the photon-emission step on GB300.

Workload (default): the 1D Au configuration -- LP plane wave a0 = 270
(1e23 W/cm^2), Au 51+ slab 1 um thick at n_e = 50 n_c, 1e6 electrons with a
Maxwell-Juttner T = 1 MeV start, dt = T/100, 4000 steps, 256 x 256 tables.
One benchmark step = that whole job: all 1e6 electrons advanced through all
4000 steps of the hot path from the resident initial state (FP32 persistent
kernel, state in registers across the steps of a launch).

Lines printed (rank 0): one JSON object with the contract keys plus
  roofline      the dominant kernel (k_step_persistent<float>) against the FP32 pipe
  roofline_hbm  the one-step-per-launch form on a state larger than L2 against HBM
  fp64_plain    the plain FP64 path (one launch per step) on the same job
  cpu_baseline  the FP64 oracle on the host cores on a bounded sample
  e2e           the same metric through the public API with host buffers
`--impl reference` times the oracle alone on the same workload and metric.
"""
from __future__ import annotations

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

METRIC = "emitting particle-steps/s at 1 GB300 (FP32/batched vs FP64 plain); % HBM roofline; p99"
UNIT = "particle-steps/s"
# FP32 operations of one particle-step of the headline job, counted by ncu's SASS counters on one
# launch of the whole job (1e6 electrons x 4000 steps): 2 per FFMA, 4 per FFMA2, 1 per FADD/FMUL,
# 2 per FADD2/FMUL2, over the 4e9 particle-steps (profiles/k_step_pair__1d-au-a270-mj-1e6x4000__flops.md)
FLOP_PER_PSTEP_1D = 123.9
FLOP_COUNT_SOURCE = "ncu SASS counters on the headline launch (FFMA 2, FFMA2 4, FADD/FMUL 1, FADD2/FMUL2 2)"
# Algorithmic bytes of one particle-step when the state round-trips memory every step:
# read + write of x (float pair, 8 B), ux, uy, uz (f32) and tau (float pair, 8 B) in 1D;
# + y (float pair) in 2D.
BYTES_PER_PSTEP_1D = 56
BYTES_PER_PSTEP_2D = 72
# the same state with an uncompensated float position (x 4 B instead of the 8 B pair): the byte
# count the hot-path scope uses for its 60 % target
BYTES_PER_PSTEP_1D_PLAIN_X = 48
FP32_LANES_PER_SM = 128
# warp instructions per 64 electron-steps of the dominant kernel (one warp steps 64 electrons), from
# the same ncu capture of the headline launch; the kernel is bound by instruction issue (one warp
# instruction per scheduler per clock), which the roofline's `issue` entry reports beside the FP32 pipe.
# Counted before the optical-depth draw's renormalisation below U = 2^-10 entered the emission
# branch: a compare per emission (2.9e6 per job) and the rare renormalisation, about 2e-3
# instructions per particle-step, within the count's last digit.
NCU_WARP_INST_PER_64_ESTEPS = 279.1
SCHEDULERS_PER_SM = 4
# DRAM bytes (read + write) per electron and launch of the dominant kernel, from the same ncu
# capture of the headline launch (29.1 MB for 1e6 electrons: the state read once, the final state
# still in L2 at the end, the cold emission tables; profiles/k_step_pair__1d-au-a270-mj-1e6x4000__flops.md:
# 29.13 B); None once the kernel changes, as it has since (the optical-depth draw of the inlined
# emission branch), until the next capture.
NCU_TRAFFIC_BYTES_PER_ELECTRON = None
# DRAM bytes (read + write) per electron of one launch of the one-step form, from an ncu capture of
# one launch on 8e6 electrons (386.7 MB: 28 B read, 20.3 B written -- the rest of the 28 B still
# dirty in L2 when the kernel ends), scaled by the electron count of the measured workload
# (profiles/k_step_pair_stream__1d-au-a270-mj-8e6-K1__full.md: 48.34 B); None once the kernel
# changes, as it has since (the same emission branch), until the next capture.
NCU_STREAM_TRAFFIC_BYTES_PER_ELECTRON = None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def hbm_peak_gbs(d):
    for k in ("hbm_gbs", "hbm_GBs", "hbm_copy_gbs", "hbm"):
        if k in d and isinstance(d[k], (int, float)):
            return float(d[k])
    for v in d.values():
        if isinstance(v, dict):
            for k in ("hbm_gbs", "gbs"):
                if k in v:
                    return float(v[k])
    return 6800.0


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
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
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


_ORACLE_TABLES = {}


def cpu_baseline(cfg, n_sample, steps, threads):
    """FP64 oracle (test infrastructure) on a strided id sample of the same workload."""
    import oracle as O
    tp = {("photon_min" if k == "photon_min_mc2" else k): v for k, v in cfg["tables"].items()}
    key = (tuple(sorted(tp.items())), tuple(cfg["Z"]))
    if key not in _ORACLE_TABLES:
        _ORACLE_TABLES[key] = O.Tables(O.table_params(**tp), list(cfg["Z"]))
    ot = _ORACLE_TABLES[key]
    run = dict(cfg["run"])
    run["iz"] = list(cfg["Z"]).index(run["Z"])
    rp = O.run_params(**run)
    ids = np.arange(0, cfg["n"], max(cfg["n"] // n_sample, 1))[:n_sample]
    st = O.init(ot, rp, ids)
    t0 = time.perf_counter()
    O.run(ot, rp, ids, st, 0, steps, capacity=1 << 20, threads=threads)
    dt = time.perf_counter() - t0
    return len(ids) * steps / dt, len(ids), dt


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--steps-per-launch", type=int, default=0)
    ap.add_argument("--skip-cpu-baseline", action="store_true")
    ap.add_argument("--skip-extras", action="store_true", help="only the headline measurement")
    ap.add_argument("--particles", type=int, default=0, help="override N (profiling runs only)")
    ap.add_argument("--job-steps", type=int, default=0, help="override steps per job (profiling runs only)")
    ap.add_argument("--profile-pic", action="store_true",
                    help="profiling run only: one PE_PIC_1D job (--particles, --job-steps) of the config-2 physics")
    ap.add_argument("--profile-pairs", action="store_true",
                    help="profiling run only: the 1 GeV Au bunch (--particles electrons), then two pair transports")
    ap.add_argument("--profile-2d", action="store_true",
                    help="profiling run only: two launches of the 2D focus job (config 3 physics) on --particles "
                         "electrons, --job-steps steps each (the second is the one to capture)")
    ap.add_argument("--profile-bw", action="store_true",
                    help="profiling run only: the reflected-wave job (--particles electrons), then two Breit-Wheeler "
                         "transports of its photons")
    args = ap.parse_args()
    if args.profile_pic:
        profile_pic(args.particles or 200_000, args.job_steps or 500)
        return
    if args.profile_pairs:
        profile_pairs(args.particles or 100_000)
        return
    if args.profile_bw:
        profile_bw(args.particles or 100_000)
        return
    if args.profile_2d:
        profile_2d(args.particles or 4_000_000, args.job_steps or 200)
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    from paper_1612_07592_gb300 import workloads as W
    cfg = W.config2()
    if args.particles:
        cfg["n"] = args.particles
    if args.job_steps:
        cfg["steps"] = args.job_steps

    if args.impl == "reference":
        if rank != 0:
            return
        threads = os.cpu_count() or 1
        W_, K = args.warmup, args.steps
        n_sample = max(2000, 40_000 // max(1, 16 // threads))
        vals = []
        for k in range(W_ + K):
            v, ns, dt = cpu_baseline(cfg, n_sample // 8 if k < W_ else n_sample, cfg["steps"], threads)
            if k >= W_:
                vals.append((v, dt))
        value = statistics.median(v for v, _ in vals)
        ms = 1e3 * statistics.median(dt for _, dt in vals)          # one timed step = one sample, as timed
        sample = f"{n_sample} of {cfg['n']} electrons (strided ids) x {cfg['steps']} steps per timed step"
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": K, "warmup": W_,
                "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic", "impl": "reference",
                "config": {"workload": cfg["name"], "particles": cfg["n"], "job_steps": cfg["steps"],
                           "timed_step": sample},
                "ms_per_full_job_extrapolated": 1e3 * cfg["n"] * cfg["steps"] / value,
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    import paper_1612_07592_gb300 as pe

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    n, S = cfg["n"], cfg["steps"]
    if world * n > (1 << 32):
        raise SystemExit("electron ids would exceed 2^32")
    tables = pe.pe_create_tables(cfg["tables"], cfg["Z"])
    stream = torch.cuda.Stream()
    # one run of world x n electrons split by electron id: rank r steps ids [r n, (r + 1) n) (same seed
    # and run id; weak scaling, no exchange while stepping; the tallies are merged after timing)
    run = dict(cfg["run"], id0=rank * n)
    launch = dict(block=args.block, ctas_per_sm=args.ctas_per_sm, steps_per_launch=args.steps_per_launch)
    cap = 1 << 24
    with torch.cuda.stream(stream):
        r = pe.Run(tables, pe.run_params(precision=pe.PE_F32, **run), n, capacity=cap, stream=stream)
    torch.cuda.synchronize()
    init_state = [t.clone() for t in (r.x, r.y, r.ux, r.uy, r.uz, r.tau)]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def reset(run_obj, state):
        with torch.cuda.stream(stream):
            for dst, src in zip((run_obj.x, run_obj.y, run_obj.ux, run_obj.uy, run_obj.uz, run_obj.tau), state):
                dst.copy_(src)
            run_obj.hist.zero_()
            run_obj.tally.zero_()
            flush.fill_(1.0)       # evict L2 (256 MB > 129 MB) between timed jobs

    def one_job(run_obj):
        # rebind the run so its step counter restarts at 0 with the reset state
        pe.pe_step_ex([run_obj.handle], S, **launch)

    # fresh run handles per job restart the step index at 0 (the laser pulse timing)
    def fresh_handle(run_obj):
        b = pe.Buffers(run_obj.x.data_ptr(), run_obj.y.data_ptr(), run_obj.ux.data_ptr(), run_obj.uy.data_ptr(),
                       run_obj.uz.data_ptr(), run_obj.tau.data_ptr(), run_obj.photons.data_ptr(), cap,
                       run_obj.hist.data_ptr(), run_obj.tally.data_ptr(), None)
        p = pe.run_params(precision=pe.PE_F32, **dict(run, init_dist=pe.PE_CALLER))
        old = run_obj.handle
        run_obj.handle = pe.pe_init_particles(tables, p, n, b, stream.cuda_stream)
        pe.pe_destroy(old)

    times = []
    for k in range(args.warmup + args.steps):
        reset(r, init_state)
        fresh_handle(r)
        # PE_CALLER redraws tau from the same Philox stream: identical to the resident start
        stream.synchronize()
        if k == args.warmup:
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            launches = 0
            clocks = ClockSampler(local).__enter__()
            wall0 = time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = pe.pe_launch_count()
        e0.record(stream)
        one_job(r)
        e1.record(stream)
        e1.synchronize()
        if k >= args.warmup:
            times.append(e0.elapsed_time(e1))
            launches += pe.pe_launch_count() - l0
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall = time.perf_counter() - wall0
    clocks.__exit__()
    out = r.tally_out()
    ms = float(np.mean(times))
    merged = None
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        # the one exchange of the partitioned run: exact merge of tallies and histograms (after timing)
        from paper_1612_07592_gb300.shard import allgather_merge
        gloo = dist.new_group(backend="gloo")
        mt, mh = allgather_merge(np.frombuffer(bytes(out.tally), dtype=np.uint64),
                                 np.frombuffer(bytes(out.hist), dtype=np.uint64), group=gloo)
        merged = {"photons": int(mt[pe.T["N_PHOTONS"]]), "ncs_stored": int(mt[pe.T["N_NCS_STORED"]]),
                  "brems_stored": int(mt[pe.T["N_BR_STORED"]]), "hist_entries": int(mh.sum())}
    pst = out.live_particle_steps
    value = pst * world / (ms * 1e-3)

    pk, pk_kind = peaks()
    res = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": cfg["name"], "particles_per_gpu": n, "job_steps": S,
                      "precision": "fp32 push/emission, fp64 optical depth, 128-bit fixed-point tallies",
                      "kernel": "k_step_pair (FP32 persistent, two electrons per thread)",
                      "steps_per_launch": args.steps_per_launch or min(S, 4096),
                      "block": args.block or 256, "l2": "flushed between timed jobs (256 MB write)",
                      "parallelism": f"dp{world} (one run of {world} x {n} electrons split by electron id)"},
           "gpu_launches": int(launches),
           "clocks": clocks.summary(),
           "wall_s_timed_region": wall}
    # roofline of the dominant kernel (k_step_pair): FP32 pipe (state held in registers across steps),
    # against the FMA-loop peak measured here on this GPU
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    pipes = fma_peaks(pe, stream, sms)
    fp32_peak = max(pipes["fp32_ffma_tflops"], pipes["fp32_ffma2_tflops"])
    ach = FLOP_PER_PSTEP_1D * pst / (ms * 1e-3) / 1e12
    traffic = NCU_TRAFFIC_BYTES_PER_ELECTRON * n if NCU_TRAFFIC_BYTES_PER_ELECTRON else None
    derived = sms * FP32_LANES_PER_SM * 2 * (res["clocks"].get("sm_max_mhz") or 2070.0) * 1e6 / 1e12
    res["roofline"] = {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach / fp32_peak,
                       "traffic": traffic,
                       "peak_kind": "measured: FMA-loop kernel of the FP32 pipe (pe_fma_peak), this GPU, this run",
                       "flop_per_particle_step": FLOP_PER_PSTEP_1D, "flop_count": FLOP_COUNT_SOURCE,
                       "pipes_measured": pipes, "fp32_peak_derived_tflops": derived, "sm_count": sms}
    clk = (res["clocks"].get("sm_mhz") or res["clocks"].get("sm_max_mhz") or 2070.0) * 1e6
    issue_ceiling = sms * SCHEDULERS_PER_SM * clk
    issued = NCU_WARP_INST_PER_64_ESTEPS / 64.0 * pst / (ms * 1e-3)
    res["roofline"]["issue"] = {"achieved": issued, "peak": issue_ceiling, "unit": "warp instructions/s",
                                "frac": issued / issue_ceiling,
                                "warp_inst_per_64_electron_steps": NCU_WARP_INST_PER_64_ESTEPS,
                                "peak_kind": "one warp instruction per scheduler per clock at the median SM clock"}

    if rank == 0 and not args.skip_extras:
        res["roofline_hbm"] = hbm_form(pe, tables, cfg, stream, hbm_peak_gbs(pk), pk_kind)
        res["roofline"]["hbm_form"] = {k: res["roofline_hbm"][k] for k in
                                       ("bound", "achieved", "peak", "unit", "frac", "frac_at_48B", "traffic")}
        res["fp64_plain"] = fp64_plain(pe, tables, cfg, stream, flush)
        res["e2e"] = e2e(pe, tables, cfg, stream)
        res["workloads"] = {"batch64_graph": batch64(pe, stream, flush),
                            "gauss2d_cp_a855_3e7x2000": gauss2d(pe, stream, flush),
                            "serving_poisson50hz": serving(pe, stream, 50.0),
                            "serving_poisson25hz": serving(pe, stream, 25.0),
                            "bunch_1gev_au_5mm_1e6": bunch_methods(pe, stream, flush),
                            "bunch_1gev_au_5mm_1e6_dt_T10": bunch_methods(pe, stream, flush, dt_over_T=0.1),
                            "reflected_1d_a270_1e6x4000": reflected(pe, tables, cfg, stream, flush),
                            "pic_1d_au_a270_1e6x2000": pic_job(pe, tables, cfg, stream, flush),
                            "pairs_bh_bunch_1gev_au_5mm_1e6": bunch_pairs(pe, stream, flush)}
    if rank == 0 and not args.skip_cpu_baseline:
        threads = os.cpu_count() or 1
        v, ns, dt = cpu_baseline(cfg, 250_000 if not args.particles else max(1000, n // 4), S, threads)
        res["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                               "sample": f"{ns} of {n} electrons (strided ids) x {S} steps, {dt:.1f} s"}
        v1, ns1, dt1 = cpu_baseline(cfg, 10_000 if not args.particles else max(500, n // 100), S, 1)
        res["cpu_baseline_1core"] = {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle",
                                     "sample": f"{ns1} of {n} electrons (strided ids) x {S} steps, {dt1:.1f} s"}
    if merged is not None:
        res["merged_tally"] = merged
    if rank == 0:
        print(json.dumps(res))
    r.close()
    if dist:
        dist.destroy_process_group()


def hbm_form(pe, tables, cfg, stream, peak_gbs, peak_kind):
    """One step per launch (the state round-trips HBM every step, as when fields come from a
    grid) on 3e7 electrons of the same 1D physics (1.08 GB of state, > L2), over the whole
    4000-step job: mean per-launch time by CUDA events."""
    import torch
    n = 30_000_000
    run = dict(cfg["run"], run_id=7)
    with torch.cuda.stream(stream):
        r = pe.Run(tables, pe.run_params(precision=pe.PE_F32, **run), n, capacity=1 << 20, stream=stream)
    stream.synchronize()
    snap = r.snapshot()
    for _ in range(3):                                           # warm-up launches
        pe.pe_step_ex([r.handle], 1, steps_per_launch=1)
    with torch.cuda.stream(stream):
        r.restore(snap)
    r.rebind(tables)
    del snap
    stream.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    K = cfg["steps"]
    ev[0].record(stream)
    pe.pe_step_ex([r.handle], K, steps_per_launch=1)
    ev[1].record(stream)
    ev[1].synchronize()
    pst = r.tally_out().live_particle_steps
    ms = ev[0].elapsed_time(ev[1]) / K
    gbs = BYTES_PER_PSTEP_1D * pst / K / (ms * 1e-3) / 1e9
    gbs48 = BYTES_PER_PSTEP_1D_PLAIN_X * pst / K / (ms * 1e-3) / 1e9
    r.close()
    return {"bound": "hbm", "achieved": gbs, "peak": peak_gbs, "unit": "GB/s", "frac": gbs / peak_gbs,
            "frac_at_48B": gbs48 / peak_gbs,
            "traffic": NCU_STREAM_TRAFFIC_BYTES_PER_ELECTRON * n if NCU_STREAM_TRAFFIC_BYTES_PER_ELECTRON else None,
            "peak_kind": peak_kind, "particles": n, "bytes_per_particle_step": BYTES_PER_PSTEP_1D,
            "ms_per_launch": ms, "launches": K, "particle_steps_per_s": pst / K / (ms * 1e-3),
            "kernel": "k_step_pair (FP32, 1D plane wave), one step per launch"}


def fma_peaks(pe, stream, sms):
    """Peak of the FP32 (FFMA and paired FFMA2) and FP64 (DFMA) pipes: FMA-loop launches of 8
    CTAs of 256 threads per SM, timed by CUDA events on the launching stream after a warm-up;
    best of 5."""
    import torch
    out = {}
    buf = torch.empty(sms * 8 * 256, dtype=torch.float64, device="cuda")
    for name, kind, iters, per in (("fp32_ffma_tflops", pe.PE_FMA_F32, 20000, 1),
                                   ("fp32_ffma2_tflops", pe.PE_FMA_F32X2, 10000, 2),
                                   ("fp64_dfma_tflops", pe.PE_FMA_F64, 400, 1)):
        best = None
        for k in range(6):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            chains = pe.pe_fma_peak(kind, sms * 8, 256, iters, buf.data_ptr(), stream.cuda_stream)
            e1.record(stream)
            e1.synchronize()
            t = e0.elapsed_time(e1) * 1e-3
            if k:
                best = t if best is None else min(best, t)
        out[name] = 2.0 * chains * iters * sms * 8 * 256 * per / best / 1e12
    return out


def fp64_plain(pe, tables, cfg, stream, flush, reps=3):
    """The plain FP64 path (one launch per step, tables in global memory) on the same job: one
    warm-up job, then the mean of `reps` timed jobs from the same initial state, L2 flushed."""
    import torch
    run = dict(cfg["run"], run_id=0)
    n, S = cfg["n"], cfg["steps"]
    with torch.cuda.stream(stream):
        r = pe.Run(tables, pe.run_params(precision=pe.PE_F64, **run), n, capacity=1 << 24, stream=stream)
    stream.synchronize()
    ms = _timed_jobs(pe, r, tables, S, stream, flush, reps=reps + 1)
    out = r.tally_out()
    r.close()
    return {"value": out.live_particle_steps / (ms * 1e-3), "unit": UNIT, "ms_per_job": ms,
            "kernel": "k_step_plain (fp64, one launch per step)", "timed_jobs": reps, "warmup_jobs": 1}


def batch64(pe, stream, flush):
    """64 runs of uneven size (Al/Au, 1e21..1e24 W/cm^2, 1000 steps) advanced together by a CUDA
    graph of batched persistent launches, launch shape chosen by the autotuner."""
    import torch
    from paper_1612_07592_gb300 import autotune
    from paper_1612_07592_gb300 import workloads as W
    c = W.config4()
    tables = pe.pe_create_tables(c["tables"], c["Z"])
    runs = []
    with torch.cuda.stream(stream):
        for rk, n in zip(c["runs"], c["n"]):
            runs.append(pe.Run(tables, pe.run_params(precision=pe.PE_F32, **rk), int(n),
                               capacity=int(min(2 * n, 1 << 23)), stream=stream))
    stream.synchronize()
    cfg, trials = autotune.tune(tables, runs, 500, space=dict(block=(128, 256), ctas_per_sm=(7, 14, 21),
                                                                 steps_per_launch=(250, 500)), use_cache=False)
    snaps = [r.snapshot() for r in runs]
    times = []
    for k in range(4):                              # one warm-up, three timed
        with torch.cuda.stream(stream):
            for r, sn in zip(runs, snaps):
                r.restore(sn)
            flush.fill_(1.0)
        for r in runs:
            r.rebind(tables)
        g = pe.pe_graph_create([r.handle for r in runs], c["steps"], **cfg)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pe.pe_graph_launch(g)
        e1.record(stream)
        e1.synchronize()
        pe.pe_graph_destroy(g)
        if k:
            times.append(e0.elapsed_time(e1))
    pst = sum(r.tally_out().live_particle_steps for r in runs)
    for r in runs:
        r.close()
    pe.pe_destroy_tables(tables)
    ms = float(np.mean(times))
    return {"value": pst / (ms * 1e-3), "unit": UNIT, "ms_per_job": ms, "runs": 64, "electrons": int(c["n"].sum()),
            "steps": c["steps"], "launch": cfg, "autotune_trials": len(trials)}


def gauss2d(pe, stream, flush):
    """2D paraxial Gaussian focus, CP a0 = 855 per component, Au 2 um slab: 3e7 electrons at rest,
    2000 steps, photon buffer 2e8 records; FP32 path, state in registers per launch."""
    import torch
    from paper_1612_07592_gb300 import workloads as W
    c = W.config3()
    tables = pe.pe_create_tables(c["tables"], c["Z"])
    with torch.cuda.stream(stream):
        r = pe.Run(tables, pe.run_params(precision=pe.PE_F32, **c["run"]), c["n"], capacity=c["capacity"],
                   stream=stream)
    stream.synchronize()
    snap = r.snapshot()
    times = []
    for k in range(4):                              # one warm-up, three timed
        with torch.cuda.stream(stream):
            r.restore(snap)
            flush.fill_(1.0)
        r.rebind(tables)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pe.pe_step([r.handle], c["steps"])
        e1.record(stream)
        e1.synchronize()
        if k:
            times.append(e0.elapsed_time(e1))
    out = r.tally_out()
    ms = float(np.mean(times))
    res = {"value": out.live_particle_steps / (ms * 1e-3), "unit": UNIT, "ms_per_job": ms, "electrons": c["n"],
           "kernel": "k_step_pair (FP32, 2D focus, two electrons per thread)",
           "steps": c["steps"], "photons": int(out.tally[pe.T["N_PHOTONS"]]),
           "ncs_stored": int(out.tally[pe.T["N_NCS_STORED"]]), "brems_stored": int(out.tally[pe.T["N_BR_STORED"]])}
    r.close()
    pe.pe_destroy_tables(tables)
    return res


def _timed_jobs(pe, r, tables, steps, stream, flush, reps=4):
    """Mean CUDA-event time of reps - 1 jobs (the first is warm-up) from the same initial state."""
    import torch
    snap = r.snapshot()
    times = []
    for k in range(reps):
        with torch.cuda.stream(stream):
            r.restore(snap)
            flush.fill_(1.0)
        r.rebind(tables)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pe.pe_step([r.handle], steps)
        e1.record(stream)
        e1.synchronize()
        if k:
            times.append(e0.elapsed_time(e1))
    return float(np.mean(times))


def bunch_methods(pe, stream, flush, n=1_000_000, dt_over_T=1.0):
    """The Sec. 2.2 bunch benchmark: 1 GeV electrons into 5 mm of fully ionised Au, fields off,
    pusher + brems only, steps of dt_over_T laser periods (5000 steps at one period); the direct
    test of Eq. 4 in every step against null collisions, FP32, 1e6 electrons (ten of the paper's
    1e5-electron bunches)."""
    import torch
    from paper_1612_07592_gb300 import workloads as W
    c = W.bunch(1000.0, "Au", n=n, dt_over_T=dt_over_T)
    tables = pe.pe_create_tables(c["tables"], c["Z"])
    out = {}
    for name, method in (("direct", pe.PE_BREMS_DIRECT), ("null", pe.PE_BREMS_NULL)):
        with torch.cuda.stream(stream):
            r = pe.Run(tables, pe.run_params(precision=pe.PE_F32, **dict(c["run"], brems_method=method)), n,
                       capacity=1 << 24, stream=stream)
        stream.synchronize()
        ms = _timed_jobs(pe, r, tables, c["steps"], stream, flush)
        t = r.tally_out()
        st = r.state()
        g = np.sqrt(1 + (st[:, 2:5] ** 2).sum(1))
        g0 = 1000.0 / 0.51099895 + 1.0
        out[name] = {"value": t.live_particle_steps / (ms * 1e-3), "ms_per_job": ms,
                     "brems_stored": int(t.tally[pe.T["N_BR_STORED"]]),
                     "mean_energy_fraction_left": float((g - 1).mean() / (g0 - 1))}
        r.close()
    pe.pe_destroy_tables(tables)
    out.update({"unit": UNIT, "electrons": n, "steps": c["steps"], "speedup_null": out["null"]["value"] /
                out["direct"]["value"], "kernel": "k_step_pair (FP32, constant fields, two electrons per thread)"})
    return out


def bunch_pairs(pe, stream, flush, n=1_000_000, reps=3):
    """Bethe-Heitler pair production of the bunch's photons (Sec. 2.2): the 1 GeV Au bunch of
    1e6 electrons is run once (direct brems test, FP32), then its stored photons are stepped
    through the rest of the 5 mm target (pe_pair_transport, the Eq. 4 test per step with the
    pair cross section), timed by CUDA events on the run's stream with L2 flushed in between.
    The free-path method (one geometric draw per photon, the same law) is timed beside it."""
    import torch
    from paper_1612_07592_gb300 import workloads as W
    c = W.bunch(1000.0, "Au", n=n)
    tables = pe.pe_create_tables(c["tables"], c["Z"])
    with torch.cuda.stream(stream):
        r = pe.Run(tables, pe.run_params(precision=pe.PE_F32, **c["run"]), n, capacity=1 << 25, stream=stream)
    pe.pe_step([r.handle], c["steps"])
    stream.synchronize()
    n_ph = r.tally_out().photons_stored
    with torch.cuda.stream(stream):
        pairs = torch.zeros(n_ph * 10, dtype=torch.int32, device="cuda")
        tally = torch.zeros(pe.PAIR_TALLY_WORDS, dtype=torch.int64, device="cuda")

    def timed(method):
        ts = []
        for k in range(reps + 1):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pe.pe_pair_transport(r.handle, r.photons.data_ptr(), n_ph, -1, pairs.data_ptr(), n_ph, tally.data_ptr(),
                                 method)
            e1.record(stream)
            e1.synchronize()
            if k:
                ts.append(e0.elapsed_time(e1))
        return float(np.median(ts)), tally.cpu().numpy().view(np.uint64).copy()

    ms, t = timed(pe.PE_PAIR_DIRECT)
    ms_f, tf = timed(pe.PE_PAIR_FREE_PATH)
    r.close()
    pe.pe_destroy_tables(tables)
    tests = int(t[pe.PT["N_TESTS"]])
    return {"value": tests / (ms * 1e-3), "unit": "Eq. 4 pair tests/s", "ms_per_transport": ms, "photons": n_ph,
            "photons_per_s": n_ph / (ms * 1e-3), "tests": tests, "pairs": int(t[pe.PT["N_PAIRS"]]),
            "entered": int(t[pe.PT["N_ENTERED"]]), "electrons": n, "steps": c["steps"],
            "kernel": "k_pair_transport (warp-cooperative tests, integer Philox per step)",
            "free_path": {"ms_per_transport": ms_f, "photons_per_s": n_ph / (ms_f * 1e-3),
                          "pairs": int(tf[pe.PT["N_PAIRS"]]), "draws": int(tf[pe.PT["N_TESTS"]]),
                          "speedup_vs_direct": ms / ms_f,
                          "kernel": "k_pair_transport (free path: one geometric draw per photon)"}}


def profile_pairs(n):
    """Profiling run: the 1 GeV Au bunch with n electrons (untimed), then two pair transports of
    its photons by the per-step tests and two by the free path (the second of each is the one to
    capture)."""
    import torch
    import paper_1612_07592_gb300 as pe
    from paper_1612_07592_gb300 import workloads as W
    c = W.bunch(1000.0, "Au", n=n)
    tables = pe.pe_create_tables(c["tables"], c["Z"])
    r = pe.Run(tables, pe.run_params(precision=pe.PE_F32, **c["run"]), n, capacity=1 << 24)
    pe.pe_step([r.handle], c["steps"])
    out = None
    for _ in range(2):
        out = r.pair_transport()
    for _ in range(2):
        free = r.pair_transport(method=pe.PE_PAIR_FREE_PATH)
    torch.cuda.synchronize()
    print(json.dumps({"profile_pairs": True, "electrons": n, "photons": int(r.tally_out().photons_stored),
                      "pairs": out[1], "tests": int(out[2][pe.PT["N_TESTS"]]), "pairs_free_path": free[1]}))
    r.close()


def profile_2d(n, steps):
    """Profiling run: the 2D focus job (config 3 physics) with n electrons, two launches of `steps`
    steps (the second is the one to capture)."""
    import torch
    import paper_1612_07592_gb300 as pe
    from paper_1612_07592_gb300 import workloads as W
    c = W.config3()
    tables = pe.pe_create_tables(c["tables"], c["Z"])
    r = pe.Run(tables, pe.run_params(precision=pe.PE_F32, **c["run"]), n, capacity=1 << 24)
    for _ in range(2):
        pe.pe_step([r.handle], steps)
    torch.cuda.synchronize()
    out = r.tally_out()
    print(json.dumps({"profile_2d": True, "electrons": n, "steps": 2 * steps,
                      "photons": int(out.tally[pe.T["N_PHOTONS"]])}))
    r.close()
    pe.pe_destroy_tables(tables)


def profile_bw(n):
    """Profiling run: the reflected-wave job with n electrons (untimed), then two Breit-Wheeler
    transports of its photons (the second is the one to capture)."""
    import torch
    import paper_1612_07592_gb300 as pe
    from paper_1612_07592_gb300 import workloads as W
    c = W.config2()
    tables = pe.pe_create_tables(c["tables"], c["Z"])
    run = dict(c["run"], reflect_r=1.0, mirror_x_m=c["run"]["slab_x0_m"] + c["run"]["slab_thick_m"])
    r = pe.Run(tables, pe.run_params(precision=pe.PE_F32, **run), n, capacity=1 << 26)
    pe.pe_step([r.handle], c["steps"])
    bw = pe.pe_bw_tables_create(64, 1e-2, 1e3, 128)
    out = None
    for _ in range(2):
        out = r.bw_transport(bw, capacity=1 << 22)
    torch.cuda.synchronize()
    print(json.dumps({"profile_bw": True, "electrons": n, "photons": int(r.tally_out().photons_stored),
                      "pairs": out[1], "photon_steps": int(out[2][pe.PT["N_TESTS"]])}))
    pe.pe_bw_tables_destroy(bw)
    r.close()


def reflected(pe, tables, cfg, stream, flush):
    """The headline 1D Au a0 = 270 job with the pulse reflected by a mirror at the slab's rear face
    (r = 1): electrons meet the counter-propagating wave and emit at eta ~ 1."""
    import torch
    run = dict(cfg["run"], run_id=11, reflect_r=1.0, mirror_x_m=cfg["run"]["slab_x0_m"] + cfg["run"]["slab_thick_m"])
    with torch.cuda.stream(stream):
        r = pe.Run(tables, pe.run_params(precision=pe.PE_F32, **run), cfg["n"], capacity=1 << 28, stream=stream)
    stream.synchronize()
    ms = _timed_jobs(pe, r, tables, cfg["steps"], stream, flush)
    t = r.tally_out()
    res = {"value": t.live_particle_steps / (ms * 1e-3), "unit": UNIT, "ms_per_job": ms, "electrons": cfg["n"],
           "steps": cfg["steps"], "ncs_stored": int(t.tally[pe.T["N_NCS_STORED"]]),
           "ncs_below_cut": int(t.tally[pe.T["N_NCS_BELOW"]]), "photons": int(t.tally[pe.T["N_PHOTONS"]]),
           "kernel": "k_step_pair (FP32, reflected-wave field kind, two electrons per thread)",
           "breit_wheeler": bw_of_photons(pe, r, t.photons_stored, stream, flush)}
    r.close()
    return res


def bw_of_photons(pe, r, n_ph, stream, flush, reps=3):
    """Breit-Wheeler conversion (Sec. 1) of a run's stored photons in the run's fields up to its last
    step (FP32 transport), timed by CUDA events on the run's stream after one warm-up, L2 flushed."""
    import torch
    bw = pe.pe_bw_tables_create(64, 1e-2, 1e3, 128)
    cap = max(n_ph // 2, 1)
    with torch.cuda.stream(stream):
        pairs = torch.empty(cap * 10, dtype=torch.int32, device="cuda")
        tally = torch.zeros(pe.PAIR_TALLY_WORDS, dtype=torch.int64, device="cuda")
    ts = []
    for k in range(reps + 1):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pe.pe_bw_transport(r.handle, bw, r.photons.data_ptr(), n_ph, -1, pairs.data_ptr(), cap, tally.data_ptr())
        e1.record(stream)
        e1.synchronize()
        if k:
            ts.append(e0.elapsed_time(e1))
    t = tally.cpu().numpy().view(np.uint64)
    pe.pe_bw_tables_destroy(bw)
    ms = float(np.median(ts))
    steps = int(t[pe.PT["N_TESTS"]])
    return {"value": n_ph / (ms * 1e-3), "unit": "photons/s", "ms_per_transport": ms, "photons": int(n_ph),
            "followed": int(t[pe.PT["N_ENTERED"]]), "pairs": int(t[pe.PT["N_PAIRS"]]),
            "photon_steps": steps, "photon_steps_note": "includes the steps behind both pulses, counted not computed",
            "chi_above_table": int(t[pe.PT["N_K_ABOVE"]]),
            "kernel": "k_bw_transport (FP32, reflected-wave field kind, one thread per photon, flattened steps)"}


def pic_job(pe, tables, cfg, stream, flush, n=1_000_000, n_cells=1000, steps=2000):
    """The config-2 physics with self-consistent fields (1D PIC around the step): 1e6 electrons in
    a 1 um Au 51+ slab at 50 n_c, the a0 = 270 pulse injected at x = 0 of a 10 um grid (1000 cells),
    2000 steps; FP32.  One launch per step (particles with current deposit; the last CTA advances the fields)."""
    import torch
    run = dict(cfg["run"], run_id=13, geometry=pe.PE_PIC_1D, n_cells=n_cells)
    with torch.cuda.stream(stream):
        r = pe.Run(tables, pe.run_params(precision=pe.PE_F32, **run), n, capacity=1 << 26, stream=stream)
    stream.synchronize()
    ms = _timed_jobs(pe, r, tables, steps, stream, flush)
    t = r.tally_out()
    ex, ey, ez, by, bz, rho = r.pic_fields()
    r.close()
    return {"value": t.live_particle_steps / (ms * 1e-3), "unit": UNIT, "ms_per_job": ms, "electrons": n,
            "n_cells": n_cells, "steps": steps, "us_per_step": 1e3 * ms / steps,
            "ncs_stored": int(t.tally[pe.T["N_NCS_STORED"]]), "killed": int(t.tally[pe.T["N_KILLED"]]),
            "max_Ex": float(np.abs(ex).max()),
            "kernels": "k_pic_particles (FP32; deposit, then the field update by the last CTA), one launch per step"}


def profile_pic(n, steps):
    """One untimed PE_PIC_1D job for profilers: the config-2 physics with self-consistent fields
    (1000 cells), n electrons, `steps` steps in one pe_step call."""
    import torch
    import paper_1612_07592_gb300 as pe
    from paper_1612_07592_gb300 import workloads as W
    c = W.config2()
    tables = pe.pe_create_tables(c["tables"], c["Z"])
    r = pe.Run(tables, pe.run_params(precision=pe.PE_F32, **dict(c["run"], geometry=pe.PE_PIC_1D, n_cells=1000)), n,
               capacity=1 << 24)
    pe.pe_step([r.handle], steps)
    torch.cuda.synchronize()
    t = r.tally_out()
    print(json.dumps({"profile_pic": True, "electrons": n, "steps": steps,
                      "ncs_stored": int(t.tally[pe.T["N_NCS_STORED"]]), "killed": int(t.tally[pe.T["N_KILLED"]])}))
    r.close()


def serving(pe, stream, rate_hz=50.0, n_requests=600):
    """Continuous batching of a Poisson trace (geometry of the 2D case, intensity and target drawn
    per request, 1e4..1e7 electrons, 500..4000 steps), all n_requests arrivals served in real time:
    p50/p99 latency (arrival to results on the host, queueing included) and throughput."""
    from paper_1612_07592_gb300 import workloads as W
    from paper_1612_07592_gb300.serve import Server, requests_from_workload
    c = W.config5(rate_hz, n_requests)
    tables = pe.pe_create_tables(c["tables"], c["Z"])
    reqs = requests_from_workload(c)
    srv = Server(tables, steps_per_iteration=500, stream=stream)
    st = srv.run_trace(reqs, realtime=True).summary()
    pe.pe_destroy_tables(tables)
    offered = sum(q.n * q.steps for q in reqs) / max(reqs[-1].arrival_s, 1e-9)
    st.update({"unit": UNIT, "offered_rate_hz": rate_hz, "offered_particle_steps_per_s": offered,
               "trace": f"{n_requests} Poisson arrivals at {rate_hz:g}/s (config 5)"})
    return st


def e2e(pe, tables, cfg, stream):
    """Same job through the public API from pinned host buffers: H2D of the initial state,
    pe_init_particles (caller state) + pe_step + pe_tally, D2H of the final state and photons."""
    import torch
    n, S = cfg["n"], cfg["steps"]
    run = dict(cfg["run"], run_id=0)
    with torch.cuda.stream(stream):
        src = pe.Run(tables, pe.run_params(precision=pe.PE_F32, **run), n, capacity=16, stream=stream)
    stream.synchronize()
    host_in = [t[:n].cpu().pin_memory() for t in (src.x, src.ux, src.uy, src.uz)]   # x: float pairs
    src.close()
    cap = 1 << 22
    bufs = [torch.empty(n, dtype=torch.float64 if k < 2 else torch.float32, device="cuda") for k in range(5)]
    tau = torch.empty(n, dtype=torch.float64, device="cuda")
    photons = torch.empty(cap * 8, dtype=torch.int32, device="cuda")
    hist = torch.empty(pe.HIST_WORDS, dtype=torch.int64, device="cuda")
    tally = torch.empty(pe.TALLY_WORDS, dtype=torch.int64, device="cuda")
    host_out = [torch.empty(n, dtype=torch.float64 if k == 0 else torch.float32).pin_memory() for k in range(4)]
    host_tau = torch.empty(n, dtype=torch.float64).pin_memory()
    host_ph = torch.empty(cap * 8, dtype=torch.int32).pin_memory()
    times, h2d, d2h = [], 0, 0
    for k in range(11):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for d, h in zip((bufs[0], bufs[2], bufs[3], bufs[4]), host_in):
                d.copy_(h, non_blocking=True)
        b = pe.Buffers(bufs[0].data_ptr(), bufs[1].data_ptr(), bufs[2].data_ptr(), bufs[3].data_ptr(),
                       bufs[4].data_ptr(), tau.data_ptr(), photons.data_ptr(), cap, hist.data_ptr(),
                       tally.data_ptr(), None)
        h = pe.pe_init_particles(tables, pe.run_params(precision=pe.PE_F32, **dict(run, init_dist=pe.PE_CALLER)),
                                 n, b, stream.cuda_stream)
        pe.pe_step([h], S)
        out = pe.pe_tally(h)
        nst = int(out.photons_stored)
        with torch.cuda.stream(stream):
            for hh, d in zip(host_out, (bufs[0], bufs[2], bufs[3], bufs[4])):
                hh.copy_(d, non_blocking=True)
            host_tau.copy_(tau, non_blocking=True)
            host_ph[: nst * 8].copy_(photons[: nst * 8], non_blocking=True)
        stream.synchronize()
        dt = time.perf_counter() - t0
        pe.pe_destroy(h)
        times.append(dt)
        h2d = (8 + 3 * 4) * n
        d2h = (8 + 3 * 4 + 8) * n + 32 * nst + 8 * (pe.HIST_WORDS + pe.TALLY_WORDS)
        pst = out.live_particle_steps
    dt = statistics.median(times[1:])
    return {"value": pst / dt, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "s_per_job": dt, "jobs_timed": len(times) - 1, "warmup_jobs": 1,
            "path": "pinned host -> pe_init_particles(PE_CALLER) + pe_step + pe_tally -> pinned host"}


if __name__ == "__main__":
    main()
