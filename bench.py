"""Benchmark: micro-MD atom-steps/s on one GB300 (and weak scaling over ranks).

A bench step is one pass of the whole hot path over one batch: the 64-element
uneven batch (h ~ U[5, 20], lateral box 10-16, 500-5000 fluid atoms,
g ~ U[0.005, 0.05], 20 000 steps each) with FP32 pair forces and the atom
state in double-float (two FP32 words, ~44-bit significand):
element build, every MD step, on-device reduction of the time-averaged flow
rates.  Each rank runs its own batch (independent micro-elements: no
data-path collective), so scaling is weak.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

--impl reference times the FP64 CPU oracle (the paper has no code to run) on a
bounded sample of the same workload on this machine's host cores.
"""
import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "micro-MD atom-steps/s"
UNIT = "atom-steps/s"
STEPS_PER_ELEMENT = 20000
N_ELEMENTS = 64
FP32_PEAK_NOTE = "152 SMs x 128 FP32 lanes x 2 flop x SM clock"
ALG_FLOPS_PER_ATOM_STEP = 600.0      # 26.2 unique pairs x ~23 FP32 flops (Newton's third law);
                                     # the integration's few flops per atom are not counted
ALG_BYTES_PER_ATOM_STEP = 96.0       # FP64 x and v read and written once per step
CPU_SAMPLE_STEPS = 1000              # oracle steps per sampled element (~10-20 s of CPU work)
FP64_PEAK_TFLOPS = 0.99              # FP64 FMA chain measured on this GB300
# ncu counters of the persistent step kernel on this workload, written with
# the capture's command into the profile summary (a "counters:" JSON line);
# used only while the kernel source still has the hash recorded there
STEP_PROFILE = os.path.join(ROOT, "profiles", "k_steps_persist_uneven64.md")
STEP_SOURCE = os.path.join(ROOT, "paper_1603_04628_gb300", "csrc", "md_kernels.cuh")


def step_kernel_counters():
    """The profile's counters dict, or None when the file is missing or the
    kernel source changed since the capture."""
    import hashlib
    try:
        with open(STEP_PROFILE) as fh:
            line = next(l for l in fh if l.startswith("counters: "))
        c = json.loads(line[len("counters: "):])
        with open(STEP_SOURCE, "rb") as fh:
            if hashlib.sha256(fh.read()).hexdigest() != c.get("source_sha256"):
                return None
        return c
    except (OSError, StopIteration, ValueError):
        return None


def _oracle_element_steps(args):
    el, steps = args
    from oracle import md as omd
    el = dict(el, steps_eq=0, steps_sample=steps)
    p = omd.make_params(el)
    nf, nw = omd.counts(p)
    t0 = time.perf_counter()
    omd.element(p)
    return (nf + nw) * steps, time.perf_counter() - t0


def cpu_baseline(pool, els, steps):
    t0 = time.perf_counter()
    out = pool.map(_oracle_element_steps, [(e, steps) for e in els])
    wall = time.perf_counter() - t0
    units = sum(u for u, _ in out)
    return units / wall, units, wall


def sample_clocks_start(path):
    try:
        fh = open(path, "w")
        proc = subprocess.Popen(
            ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
             "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
            stdout=fh, stderr=subprocess.DEVNULL)
        return proc, fh
    except Exception:
        return None, None


def sample_clocks_stop(proc, fh, path, gpu_index):
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except Exception:
        proc.kill()
    fh.close()
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        f = [t.strip() for t in line.split(",")]
        if len(f) < 9 or f[0] != str(gpu_index):
            continue
        try:
            sm.append(float(f[1]))
            mx.append(float(f[2]))
        except ValueError:
            continue
        for nm, val in zip(names, f[5:9]):
            if val.lower() == "active":
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
            "reasons": sorted(reasons)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    els = synth.batch_uneven(N_ELEMENTS, steps=STEPS_PER_ELEMENT)
    cores = os.cpu_count() or 1
    sample_els = els[:min(len(els), cores)]
    sample_steps = args.sample_steps
    from oracle import md as omd
    omd.build()
    with mp.get_context("spawn").Pool(len(sample_els)) as pool:
        for _ in range(args.warmup):
            cpu_baseline(pool, sample_els, 20)
        rates, walls = [], []
        for _ in range(args.steps):
            r, units, wall = cpu_baseline(pool, sample_els, sample_steps)
            rates.append(r)
            walls.append(wall)
    value = statistics.mean(rates)
    sample = "%d of the %d uneven elements, %d steps each, FP64 oracle, one process per element" % (
        len(sample_els), N_ELEMENTS, sample_steps)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(walls),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "uneven batch: 64 elements, h 5-20, lateral 10-16, 500-5000 fluid atoms, "
                                   "20000 steps (sampled)", "elements": N_ELEMENTS,
                       "steps_per_element": STEPS_PER_ELEMENT},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": len(sample_els), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=1000,
                    help="steps of the FP64-forces pass reported beside the headline")
    ap.add_argument("--steps-per-element", type=int, default=STEPS_PER_ELEMENT,
                    help="MD steps per element (shorter runs for profiling only)")
    ap.add_argument("--case", default="micro",
                    choices=["micro", "channel", "channel-evidence", "gp", "learned-mean", "small-batch"],
                    help="micro: the uneven micro-element batch (default; its line also carries the channel "
                         "case); channel: the full hybrid (Algorithm 1) threshold sweep on the 200-section channel "
                         "judged against the full MD; channel-evidence: the same judged with evidence "
                         "hyperparameters, warm starts and long equilibration; gp: the GP and MLP timings alone; "
                         "learned-mean: the MLP prior mean against the plain GP hybrid at matched thresholds, "
                         "judged against the MD-everywhere run; small-batch: per-step time of the hybrid's MD "
                         "batches (1-30 channel elements), general and resident-atom step kernels")
    ap.add_argument("--elements", type=str, default="1,2,4,8,16,30",
                    help="small-batch case: batch sizes (comma separated)")
    ap.add_argument("--resident", type=str, default="0,1",
                    help="small-batch case: step kernels to time (0 general, 1 resident atoms)")
    ap.add_argument("--channel-steps", type=int, default=100)
    ap.add_argument("--form", default="paper", choices=["paper", "linear"],
                    help="channel case: the paper's p-GP and (h, n, F) q-GP inputs (default), or a linear "
                         "equation of state with (h, G) inputs")
    ap.add_argument("--paper-form", action="store_true", help="same as --form paper")
    ap.add_argument("--sample-steps", type=int, default=300,
                    help="oracle steps per sampled element in the reference arm")
    ap.add_argument("--no-gp-mlp", action="store_true", help="skip the GP and MLP timings")
    ap.add_argument("--no-hybrid", action="store_true", help="skip the hybrid-channel summary")
    ap.add_argument("--h-amp", type=float, default=0.5,
                    help="relative amplitude of the channel's height profile in the hybrid summary (0.5: the "
                         "benchmark channel; 0.25: the paper's Eq. heightEq)")
    ap.add_argument("--persistent", type=int, default=None, choices=[0, 1, 2],
                    help="step loop: 0 one launch per step, 1 persistent kernel in a graph WHILE loop, 2 the "
                         "persistent kernel launched by the host (profilers capture it)")
    ap.add_argument("--workload", default="uneven", choices=["uneven", "stress"],
                    help="uneven: 64 elements, 500-5000 fluid atoms, 20000 steps (default); stress: 4096 "
                         "elements, 2k-32k fluid atoms, 60 M atoms, 10000 steps")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.case == "channel":
        return run_channel_case(args)
    if args.case == "channel-evidence":
        return run_channel_evidence_case(args)
    if args.case == "learned-mean":
        return run_learned_mean_case(args)
    if args.case == "small-batch":
        return run_small_batch_case(args)
    if args.case == "gp":
        import torch
        torch.cuda.set_device(0)
        from paper_1603_04628_gb300 import native
        print(json.dumps({"case": "gp", "n_gpus": 1, "data": "synthetic", **gp_mlp_timings(native, 0)}), flush=True)
        return 0

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.workload == "stress":
        steps_el = args.steps_per_element if args.steps_per_element != STEPS_PER_ELEMENT else 10000
        els = synth.batch_stress(seed=synth.BASE_SEED + 5 + 1000 * rank, steps=steps_el)
    else:
        steps_el = args.steps_per_element
        els = synth.batch_uneven(N_ELEMENTS, seed=synth.BASE_SEED + 1000 * rank, steps=steps_el)

    # CPU pool first (spawned before any CUDA work)
    pool = None
    if rank == 0 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        pool = mp.get_context("spawn").Pool(min(cores, len(els)))

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1603_04628_gb300 import native

    stream = torch.cuda.Stream()
    path_kw = {}
    if args.persistent is not None:
        path_kw["persistent"] = args.persistent
    ctx = native.Context(local, native.PREC_FP32, stream=stream, **path_kw)
    n_atoms = ctx.micro_plan(els)
    units = n_atoms * steps_el
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    # neighbour lists that overflow (dense elements) are re-planned with more
    # room before anything is timed, as mdgp_micro_batch does
    cap = 128
    for _ in range(3):
        ctx.micro_launch()
        if not any(r["status"] == -8 for r in ctx.micro_results()):
            break
        cap = int(cap * 1.5) // 8 * 8
        ctx.set_md_params(list_capacity=cap, **path_kw)
        n_atoms = ctx.micro_plan(els)
    for _ in range(args.warmup):
        ctx.micro_launch()
        ctx.micro_results()
    launches_per_step = ctx.launch_count()
    rebuilds_per_step = ctx.rebuild_count()

    # clock samples during the timed region (nvidia-smi), kept beside the run
    clk_path = os.path.join(os.environ.get("MDGP_CLOCKS_DIR", "."), "bench_clocks_rank%d.csv" % rank)
    proc, fh = sample_clocks_start(clk_path)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    times = []
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            flush.zero_()                     # L2 flush between timed iterations (256 MB > 129 MB L2)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.micro_launch()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sample_clocks_stop(proc, fh, clk_path, local)
    res = ctx.micro_results()
    bad = [r["status"] for r in res if r["status"] != 0]
    ms = statistics.mean(times)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = units * world / (ms / 1e3)

    # per-kernel durations (CUDA events on the context's stream) for the
    # roofline: the persistent step kernel launched by the host once per
    # list-rebuild interval (the timed run's kernel, outside its graph), and
    # the one-launch-per-step kernel of the same step code
    path = ctx.path()
    shape = ctx.launch_shape() if path != "per-step" else None
    prof = ctx.micro_profile(min(200, steps_el))
    cdir = native.Context(local, native.PREC_FP32, stream=stream, persistent=2, list_capacity=cap)
    cdir.micro_plan(els)
    cdir.micro_launch()
    cdir.micro_results()
    cdir.micro_launch()
    cdir.micro_results()
    dt = cdir.direct_timing()
    cdir.close()
    persist_step_s = dt["kernel_ms"] / 1e3 / max(1, dt["steps"])
    sm_mhz = (clocks or {}).get("sm_max_mhz", 2070.0) or 2070.0
    fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    achieved = ALG_FLOPS_PER_ATOM_STEP * n_atoms / persist_step_s / 1e12
    counters = step_kernel_counters() if args.workload == "uneven" else None

    # end to end through the public API: host descriptors in, host results out
    e2e_times = []
    for _ in range(max(1, min(args.steps, 2))):
        t0 = time.perf_counter()
        ctx2_res = ctx.micro_batch(els)
        e2e_times.append(time.perf_counter() - t0)
    e2e_value = units * world / statistics.mean(e2e_times)
    # element descriptors + offsets up, results down
    h2d = len(els) * (256 + 16) + 16
    d2h = len(els) * 72

    # FP64-forces pass (same batch, shorter), reported beside the headline
    fp64 = None
    if args.fp64_steps > 0 and rank == 0:
        els64 = [dict(e, steps_eq=args.fp64_steps // 5, steps_sample=args.fp64_steps - args.fp64_steps // 5)
                 for e in els]
        c64 = native.Context(local, native.PREC_FP64, stream=stream)
        na = c64.micro_plan(els64)
        c64.micro_launch(); c64.micro_results()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream); c64.micro_launch(); e1.record(stream); e1.synchronize()
        fp64 = {"value": na * args.fp64_steps / (e0.elapsed_time(e1) / 1e3), "unit": UNIT,
                "steps_per_element": args.fp64_steps, "dtype": "f64"}
        c64.close()

    # GP fit + predict (FP64 Cholesky) and the MLP prior mean, reported beside
    # the MD headline (they are small against MD in every workload)
    gp_mlp = None
    if rank == 0 and args.workload == "uneven" and not args.no_gp_mlp:
        gp_mlp = gp_mlp_timings(native, local)
    hybrid = None
    if rank == 0 and world == 1 and args.workload == "uneven" and not args.no_hybrid:
        hybrid = channel_case(local, h_amp=args.h_amp, noise_run=False)
    small = None
    if rank == 0 and world == 1 and args.workload == "uneven" and not args.no_hybrid:
        # the hybrid's MD batch sizes with either step kernel (graph path);
        # a failure here is reported in the key, not in the headline
        try:
            small = [{k: r[k] for k in ("elements", "atoms", "us_per_step", "rebuilds", "clean")}
                     | {"threads_per_atom": r["launch_shape"]["threads_per_atom"],
                        "resident": r["launch_shape"]["resident"]}
                     for r in small_batch_rows(local, [1, 2, 8], [0, 1], [1])]
        except Exception as exc:   # noqa: BLE001
            small = {"error": repr(exc)}

    cpu = None
    if pool is not None:
        sample_els = els[:min(len(els), os.cpu_count() or 1)]
        csteps = CPU_SAMPLE_STEPS if args.workload == "uneven" else CPU_SAMPLE_STEPS // 10
        rate, cu, wall = cpu_baseline(pool, sample_els, csteps)
        pool.close()
        cpu = {"value": rate, "unit": UNIT, "cores": len(sample_els), "kind": "oracle",
               "sample": "%d of the %d elements x %d steps, FP64 oracle, one process per element "
                         "(%.1f s wall)" % (len(sample_els), len(els), csteps, wall)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 forces + double-f32 state", "data": "synthetic",
            "config": {"workload": ("uneven batch: 64 elements, h 5-20, lateral 10-16, 500-5000 fluid atoms, "
                                    "g 0.005-0.05, %d steps, FP32 forces + double-float state" % steps_el)
                       if args.workload == "uneven" else
                       ("stress batch: 4096 elements, h 5-40, n 0.7-0.9, 2k-32k fluid atoms, %d steps, FP32 forces "
                        "+ double-float state" % steps_el),
                       "elements": len(els), "atoms_per_rank": n_atoms, "steps_per_element": steps_el,
                       "l2": "flushed between timed iterations (256 MB write)",
                       "parallelism": "independent elements per rank" if world > 1 else "1 GPU"},
            "roofline": {"bound": "alu", "kernel": "k_steps_persist (pair forces + integration of every step "
                                                 "of a list-rebuild interval, a grid barrier between steps)",
                         "achieved": achieved, "peak": fp32_peak,
                         "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                         "traffic": counters["dram_bytes_per_step"] if counters else None,
                         "l1_frac": counters["l1tex_throughput_frac"] if counters else None,
                         "issue_frac": counters["issue_active_frac"] if counters else None,
                         "counters_from": os.path.relpath(STEP_PROFILE, ROOT) if counters else None,
                         "peak_note": FP32_PEAK_NOTE + " (derived, max SM clock)",
                         "alg_flops_per_atom_step": ALG_FLOPS_PER_ATOM_STEP,
                         "timing": "k_steps_persist launched by the host once per list-rebuild interval "
                                   "(persistent = 2), CUDA events around each launch on the context's "
                                   "stream, %d launches covering %d steps of the same batch"
                                   % (dt["launches"], dt["steps"]),
                         "persistent_step_us": persist_step_s * 1e6,
                         "per_step_launch_us": prof["force_ms"] * 1e3,
                         "persistent_minus_per_launch_us": persist_step_s * 1e6 - prof["force_ms"] * 1e3,
                         "rebuilds_per_run": rebuilds_per_step, "rebuild_ms": prof["rebuild_ms"],
                         "rebuild_share": rebuilds_per_step * prof["rebuild_ms"] / ms},
            "path": path,
            "launch_shape": shape,
            "hbm_roofline": {"alg_bytes_per_atom_step": ALG_BYTES_PER_ATOM_STEP,
                             "achieved_gbs": value / world * ALG_BYTES_PER_ATOM_STEP / 1e9,
                             "peak_gbs": _peak_hbm(), "frac": value / world * ALG_BYTES_PER_ATOM_STEP / 1e9 /
                             _peak_hbm()},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks,
            "fp64_forces": fp64,
            "gp_mlp": gp_mlp,
            "hybrid": hybrid,
            "small_batch": small,
            "element_status_errors": len(bad),
            "element_status_codes": sorted(set(bad)),
            "list_capacity": cap,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def evidence_warm_summary(device, n_sections=100, n_steps=50, long_eq=8000, thresholds=(1.0, 4.0), h_amp=0.5):
    """Algorithm 1 on the converging-diverging channel in the paper's form
    (p-GP over (h, n) from pre-simulations, q-GP on (h, n, F)), one forcing
    period (50 macro steps of 20), judged as the paper does (Sec. 3) against
    a full MD of the whole channel: one element of length L = 10^4 whose
    walls follow h(x), driven by the same external force, its flow-rate
    history filtered by the App. B periodic GP; the thermal noise is the
    same error between the raw and the filtered full MD.  Each threshold runs
    with warm starts (Sec. 2.4) and pseudoMD's start-up time (Algorithm 1,
    viscosity and slip fitted to the library's own MD), the q-GP's
    hyperparameters by maximum evidence (Sec. 2.3) on the database of an
    MD-at-every-section run (each run equilibrated long_eq steps), which is
    also reported as a second reference.  Reports MD runs, Eq. error, Eq.
    speedup with the full MD's own atom count, and measured wall times."""
    import numpy as np
    from paper_1603_04628_gb300 import cases, native
    t_all = time.perf_counter()
    ctx = native.Context(device, native.PREC_FP32)
    sn = 0.5
    # elements 6 x 6 wall-lattice cells across (9.52 sigma): the full MD's
    # walls have the unstretched FCC lattice, and a 10 sigma element would
    # stretch its walls by 5 % along x and z, which changes the wall friction
    # and the flow rate by about 10 % (measured at h = 12 and 18)
    box = 6.0 * 4.0 ** (1.0 / 3.0)
    fit = cases.fit_pseudo_md(ctx, Lx=box, Lz=box)
    params = dict(n_sections=n_sections, dx=10000.0 / n_sections, h0=12.0, Lx=box, Lz=box, eos_K=10.0,
                  eos_n0=0.8, dP_amp=400.0, period=1000.0, dt=20.0, T=1.1, md_steps_eq=long_eq,
                  md_steps_sample=3000, seed=synth.BASE_SEED, sf2=(20 * sn) ** 2, l2=1.0, sn2=sn ** 2,
                  sn2_from_data=0, inputs=1, h_amp=h_amp)
    X, p, p_se = cases.pressure_sweep(ctx, np.linspace(12.0 * (1 - h_amp), 12.0 * (1 + h_amp), 5),
                                      np.linspace(0.6, 1.0, 9), T=params["T"], seed=synth.BASE_SEED + 7, Lx=box, Lz=box)
    pdb = (X, p, float(np.var(p)), 1.0, float(np.mean(p_se)) ** 2)
    # the full MD of the channel and its App. B filtered history
    full = cases.full_channel_md(ctx, n_steps, **dict(params, seed=synth.BASE_SEED + 55))
    t = np.arange(1, n_steps + 1) * params["dt"]
    filt, _, _, _ = cases.periodic_filter(ctx, t, full["Q"], params["period"], sf2=float(np.var(full["Q"])),
                                          sn2=1e-4, fit_until=None)
    ref = cases.run_channel(ctx, 0.0, n_steps, pressure_db=pdb, **params)
    # q-GP hyperparameters by maximum evidence (Sec. 2.3) on 400 entries of
    # the MD-everywhere run's database, sigma_n^2 held at its mean squared SE
    Xr, yr, ser = ref["db"]
    sub = np.random.default_rng(synth.BASE_SEED).choice(len(yr), size=min(400, len(yr)), replace=False)
    sn2_ev = float(np.mean(ser)) ** 2
    sf2_ev, l2_ev = cases.evidence_hyperparameters(ctx, Xr[sub], yr[sub], sn2_ev)
    rows = []
    t_end_steps = full["md_steps"]
    for s in thresholds:
        hy = native.Hybrid(ctx, **dict(params, warm_start=1, md_steps_eq_warm=250, pseudo_nu=fit["nu"],
                                       pseudo_slip=fit["slip"], sf2=sf2_ev, l2=l2_ev, sn2=sn2_ev))
        hy.set_pressure(*pdb)
        qbar, runs, warm, steps, atoms, md_s, gp_s = [], 0, 0, 0, 0, 0.0, 0.0
        t0 = time.perf_counter()
        for _ in range(n_steps):
            st = hy.step(s)
            qbar.append(st["q_mean"])
            runs += st["md_runs"]
            warm += st["md_warm"]
            steps += st["md_warm"] * (st["md_steps_eq_warm"] + params["md_steps_sample"]) + \
                (st["md_runs"] - st["md_warm"]) * (long_eq + params["md_steps_sample"])
            atoms += st["md_atoms"]
            md_s += st["md_seconds"]
            gp_s += st["gp_seconds"]
        wall = time.perf_counter() - t0
        hy.close()
        rows.append(dict(sigma_t=s, md_runs=runs, md_warm=warm, mean_md_steps=steps / runs if runs else 0.0,
                         error=cases.error(qbar, filt), error_vs_raw_full_md=cases.error(qbar, full["Q"]),
                         error_vs_md_everywhere=cases.error(qbar, ref["qbar"]),
                         speedup_eq=(t_end_steps * full["n_atoms"] / steps / (atoms / runs)) if runs else None,
                         wall_s=wall, wall_vs_full_md=full["wall_s"] / wall,
                         wall_vs_md_everywhere=ref["wall_s"] / wall, md_s=md_s, gp_s=gp_s))
    ctx.close()
    return {"metric": "hybrid flow error against a full MD of the channel and speed-up over it (Eqs. error, "
                      "speedup)",
            "config": {"workload": "%d-section converging-diverging channel (h0 = 12, a = %g, L = 10^4), one forcing "
                                   "period (%d macro steps of 20), %.3f x h x %.3f elements (6 x 6 wall cells, FP32 "
                                   "forces), paper form: p-GP on (h, n) from 45 pre-simulations, q-GP on (h, n, F)"
                                   % (n_sections, h_amp, n_steps, box, box),
                       "sigma_n": sn, "md_steps_sample": params["md_steps_sample"],
                       "md_everywhere_eq_steps": long_eq, "warm_eq_floor": 250},
            "full_md": {"atoms": full["n_atoms"], "md_steps": full["md_steps"], "wall_s": full["wall_s"],
                        "atom_steps_per_s": full["n_atoms"] * full["md_steps"] / full["wall_s"],
                        "f_ext_amplitude": full["f_amp"], "windows": len(full["q_windows"]),
                        "Q_mean_abs": float(np.mean(np.abs(full["Q"])))},
            "thermal_noise_error": cases.error(full["Q"], filt),
            "pseudo_md_fit": {"nu": fit["nu"], "slip": fit["slip"]},
            "evidence_hyperparameters": {"sf2": sf2_ev, "l2": l2_ev, "sn2": sn2_ev, "entries": int(len(sub))},
            "md_everywhere": {"md_runs": ref["md_runs"], "wall_s": ref["wall_s"],
                              "error_vs_full_md": cases.error(ref["qbar"], filt)},
            "rows": rows, "wall_s": time.perf_counter() - t_all}


def gp_mlp_timings(native, device):
    """Wall times of the GP (fit on M = 2000 entries in D = 2, predict 200
    queries) and of the MLP prior mean (1000 epochs on 10^4 rows); the fit's
    FP64 Cholesky rate against the measured FP64 peak."""
    import numpy as np
    ctx = native.Context(device, native.PREC_FP64)
    M, m = 2000, 200
    X, y = synth.gp_dataset(M, seed=synth.BASE_SEED + 21)
    Xs = synth.gp_queries(m, seed=synth.BASE_SEED + 22)
    g = native.GP(ctx, X, y, 1.0, 1.0, 0.0025)          # warm-up (allocations, module load)
    g.predict(Xs); g.close()
    reps = 5
    t0 = time.perf_counter()
    for _ in range(reps):
        g = native.GP(ctx, X, y, 1.0, 1.0, 0.0025)
        g.close()
    fit_s = (time.perf_counter() - t0) / reps
    g = native.GP(ctx, X, y, 1.0, 1.0, 0.0025)
    t0 = time.perf_counter()
    for _ in range(reps):
        g.predict(Xs)
    pred_s = (time.perf_counter() - t0) / reps
    g.close()
    chol_flops = M ** 3 / 3.0
    Xm = np.random.default_rng(synth.BASE_SEED + 23).uniform([6.0, -0.05], [18.0, 0.05], (10000, 2))
    ym = np.sin(Xm[:, 0]) + 10.0 * Xm[:, 1]
    net = native.MLP(ctx, seed=3)
    t0 = time.perf_counter()
    net.train(Xm, ym, epochs=1000, eval_every=100)
    mlp_s = time.perf_counter() - t0
    ctx.close()
    return {"gp_fit_s": fit_s, "gp_predict_s": pred_s, "gp_M": M, "gp_queries": m,
            "gp_fit_fp64_tflops": chol_flops / fit_s / 1e12, "fp64_peak_tflops": FP64_PEAK_TFLOPS,
            "fp64_peak_note": "measured FP64 FMA chain on this GB300 (0.99 TFLOP/s)",
            "gp_fit_frac": chol_flops / fit_s / 1e12 / FP64_PEAK_TFLOPS,
            "mlp_train_s": mlp_s, "mlp_rows": len(ym), "mlp_epochs": 1000,
            "timing": "wall clock of the C-ABI calls (host in/out), mean of 5 for the GP"}


def channel_case(device, n_steps=100, h_amp=0.5, paper_form=True, noise_run=True):
    """Configured channel case (cfg 3): Algorithm 1 on the 200-section
    converging-diverging channel, 100 macro steps, the cfg 1 elements
    (2000 + 3000 steps) in 6 x 6 wall cells, sigma_f = 20 sigma_n and l^2 = 1
    (the paper's ratios, Sec. 2.3), thresholds 0.5-8 sigma_n from an empty
    database; judged against the full MD of the channel (App. B filtered,
    Sec. 3) and against MD at every section.  Returns the result dict."""
    from paper_1603_04628_gb300 import cases, native
    import numpy as np
    ctx = native.Context(device, native.PREC_FP32)
    t_all = time.perf_counter()
    sn = 0.5
    box = 6.0 * 4.0 ** (1.0 / 3.0)   # 6 x 6 wall-lattice cells, like the full MD's walls
    params = dict(n_sections=200, dx=50.0, h0=12.0, Lx=box, Lz=box, eos_K=10.0, eos_n0=0.8, dP_amp=400.0,
                  period=1000.0, dt=20.0, T=1.1, md_steps_eq=2000, md_steps_sample=3000, seed=synth.BASE_SEED,
                  sf2=(20 * sn) ** 2, l2=1.0, sn2=sn ** 2, sn2_from_data=0, h_amp=h_amp)
    thresholds = [f * sn for f in (0.5, 1.0, 2.0, 4.0, 8.0)]
    pressure_db, form = None, "q-GP on (h, G), linear equation of state"
    if paper_form:
        # the paper's form (Sec. 2.4): p-GP over (h, n) from pre-simulations,
        # q-GP on (h, n, F)
        X, p, p_se = cases.pressure_sweep(ctx, np.linspace(12.0 * (1 - h_amp), 12.0 * (1 + h_amp), 5),
                                          np.linspace(0.6, 1.0, 9), T=params["T"], seed=synth.BASE_SEED + 7,
                                          Lx=box, Lz=box)
        psn = float(np.mean(p_se))
        pressure_db = (X, p, float(np.var(p)), 1.0, psn ** 2)
        params["inputs"] = 1
        form = "q-GP on (h, n, F), p-GP on (h, n) from %d pre-simulations (mean p SE %.3f)" % (len(p), psn)
    # the full MD of the channel (Sec. 3's judge), its App. B filtered history
    full = cases.full_channel_md(ctx, n_steps, **dict(params, seed=synth.BASE_SEED + 55))
    t = np.arange(1, n_steps + 1) * params["dt"]
    full["Q_filtered"] = cases.periodic_filter(ctx, t, full["Q"], params["period"], sf2=float(np.var(full["Q"])),
                                               sn2=1e-4, fit_until=None)[0]
    out = cases.channel_sweep(ctx, thresholds, n_steps=n_steps,
                              seed_noise=synth.BASE_SEED + 99 if noise_run else None,
                              pressure_db=pressure_db, full_md=full, **params)
    ctx.close()
    ref = out["reference"]
    keys = ("sigma_t", "md_runs", "error_vs_full_md", "speedup_eq_full_md", "wall_s", "wall_vs_full_md",
            "error", "speedup_eq", "wall_vs_reference", "gp_s", "md_s")
    rows = []
    for r in out["rows"]:
        row = {k: r[k] for k in keys if k in r}
        row["error_vs_md_everywhere"] = row.pop("error")
        row["speedup_eq_estimated_atoms"] = row.pop("speedup_eq")
        row["wall_vs_md_everywhere"] = row.pop("wall_vs_reference")
        rows.append(row)
    return {"metric": "hybrid flow error against a full MD of the channel and speed-up over it (Eqs. error, "
                      "speedup)",
            "config": {"workload": "200-section converging-diverging channel, h0 = 12, a = %g, L = 10^4, %d macro "
                                   "steps of 20 (two forcing periods), %.3f x h x %.3f elements (2000 + 3000 "
                                   "steps, FP32 forces), thresholds 0.5-8 sigma_n from an empty database"
                                   % (h_amp, n_steps, box, box),
                       "sigma_n": sn, "sigma_f": 20 * sn, "l2": 1.0, "form": form},
            "full_md": {"atoms": full["n_atoms"], "md_steps": full["md_steps"], "wall_s": full["wall_s"],
                        "atom_steps_per_s": full["n_atoms"] * full["md_steps"] / full["wall_s"],
                        "windows": len(full["q_windows"]), "f_ext_amplitude": full["f_amp"]},
            "thermal_noise_error": out["full_md_noise"],
            "md_everywhere": {"md_runs": ref["md_runs"], "wall_s": ref["wall_s"],
                              "error_vs_full_md": out["reference_error_vs_full_md"],
                              "noise_error_two_runs": out.get("noise_error")},
            "rows": rows, "wall_s": time.perf_counter() - t_all}


def small_batch_rows(device, elements, residents, paths):
    """Per-step time of batches of the hybrid's MD elements (9.524 x h x 9.524,
    h ~ U[6, 18], n = 0.8, 2000 + 3000 steps, FP32 forces): one row per batch
    size, step kernel (resident 0: the general one, 1: resident atoms where
    it applies) and step-loop path (persistent 1 or 2)."""
    import numpy as np
    import torch
    from paper_1603_04628_gb300 import native
    stream = torch.cuda.Stream(device)
    box = 6.0 * 4.0 ** (1.0 / 3.0)
    rng = np.random.default_rng(synth.BASE_SEED + 17)
    rows = []
    for nel in elements:
        hs = rng.uniform(6.0, 18.0, nel)
        els = [dict(h=float(h), Lx=box, Lz=box, density=0.8, T=1.1, g_ext=0.03, dpdx=0.0, steps_eq=2000,
                    steps_sample=3000, seed=synth.BASE_SEED + 11 + k, id=k) for k, h in enumerate(hs)]
        steps = 5000
        for resident in residents:
            for p in paths:
                ctx = native.Context(device, native.PREC_FP32, stream=stream, persistent=p, resident=resident)
                n = ctx.micro_plan(els)
                ctx.micro_launch()
                ctx.micro_results()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                ctx.micro_launch()
                e1.record(stream)
                e1.synchronize()
                res = ctx.micro_results()
                row = {"elements": nel, "atoms": n, "persistent": p, "launch_shape": ctx.launch_shape(),
                       "us_per_step": 1e3 * e0.elapsed_time(e1) / steps, "rebuilds": ctx.rebuild_count(),
                       "clean": all(r["status"] == 0 for r in res), "q": [r["q"] for r in res]}
                if p == 2:
                    dt = ctx.direct_timing()
                    row["kernel_us_per_step"] = 1e3 * dt["kernel_ms"] / max(1, dt["steps"])
                    row["rebuild_us"] = 1e3 * dt["rebuild_ms"] / max(1, dt["rebuilds"])
                rows.append(row)
                ctx.close()
    return rows


def run_small_batch_case(args):
    """bench.py --case small-batch: small_batch_rows as JSON lines."""
    import torch
    torch.cuda.set_device(0)
    pers = [args.persistent] if args.persistent is not None else [1, 2]
    for row in small_batch_rows(0, [int(v) for v in args.elements.split(",")],
                                [int(v) for v in args.resident.split(",")], pers):
        print(json.dumps({"case": "small-batch", **row}), flush=True)
    return 0


def run_channel_case(args):
    """cfg 3's sweep as a JSON line (bench.py --case channel)."""
    import torch
    torch.cuda.set_device(0)
    line = channel_case(0, n_steps=args.channel_steps, h_amp=args.h_amp,
                        paper_form=args.paper_form or args.form == "paper", noise_run=True)
    line.update({"case": "channel", "n_gpus": 1, "data": "synthetic"})
    print(json.dumps(line), flush=True)
    return 0


def run_channel_evidence_case(args):
    """The channel judged against the full MD with the q-GP's hyperparameters
    by maximum evidence, warm starts and pseudoMD, elements equilibrated
    8000 steps (bench.py --case channel-evidence)."""
    import torch
    torch.cuda.set_device(0)
    line = evidence_warm_summary(0, h_amp=args.h_amp)
    line.update({"case": "channel-evidence", "n_gpus": 1, "data": "synthetic"})
    print(json.dumps(line), flush=True)
    return 0


def run_learned_mean_case(args):
    """The learned prior mean (MLP 2 -> 64 -> 64 -> 1 on (h, G)) against the
    plain GP in the linear-form channel: MD runs and Eq. error against the
    MD-everywhere run at five thresholds, both arms' hyperparameters by
    maximum evidence on the same MD database."""
    import torch
    from paper_1603_04628_gb300 import cases, native
    torch.cuda.set_device(0)
    ctx = native.Context(0, native.PREC_FP32)
    # 50 sections: the plain arm with evidence hyperparameters runs MD at
    # most sections, and every appended entry refits the GP (O(M^3))
    import numpy as np
    box = 6.0 * 4.0 ** (1.0 / 3.0)   # 6 x 6 wall-lattice cells, like the full MD's walls
    params = dict(n_sections=50, dx=200.0, h0=12.0, Lx=box, Lz=box, eos_K=10.0, eos_n0=0.8, dP_amp=400.0,
                  period=1000.0, dt=20.0, T=1.1, md_steps_eq=2000, md_steps_sample=3000, seed=synth.BASE_SEED,
                  sn2_from_data=0, inputs=0)
    t0 = time.perf_counter()
    full = cases.full_channel_md(ctx, args.channel_steps, **dict(params, seed=synth.BASE_SEED + 55))
    t = np.arange(1, args.channel_steps + 1) * params["dt"]
    full["Q_filtered"] = cases.periodic_filter(ctx, t, full["Q"], params["period"], sf2=float(np.var(full["Q"])),
                                               sn2=1e-4, fit_until=None)[0]
    thresholds = [0.5, 1.0, 2.0, 4.0]
    rows, info, net = cases.learned_mean_comparison(
        ctx, thresholds, args.channel_steps, db_elements=256, db_seed=synth.BASE_SEED + 31,
        log=lambda d: print(json.dumps(d), file=sys.stderr, flush=True), full_md=full, **params)
    line = {"case": "learned-mean", "n_gpus": 1, "data": "synthetic",
            "config": {"workload": "50-section channel (L = 10^4), linear equation of state, q-GP on (h, G), %d "
                                   "macro steps, %.3f x h x %.3f elements (2000 + 3000 steps, FP32 forces); MLP "
                                   "trained on 256 MD runs over h 6-18, G -0.06..0.06; judged against MD at every "
                                   "section and against the full MD of the channel" % (args.channel_steps, box, box)},
            "info": info, "rows": rows, "wall_s": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)
    net.close()
    ctx.close()
    return 0


def _peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except Exception:
        return 6800.0


if __name__ == "__main__":
    sys.exit(main())
