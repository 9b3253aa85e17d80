"""Throughput benchmark: spin-site updates per second of the fused field + Heun step.

Workload (default, `sc_j123_dmi_1024`): simple cubic 1024^3 = 1,073,741,824
spins, exchange on three distance shells (J1..J3 = 1, -0.164, -0.082 meV) plus
interfacial DMI D = 0.1 meV, mu = 2.2 mu_B, stochastic Heun LLG at T = 50 K,
alpha = 0.1, dt = 0.1 fs, periodic; FP32 field with FP64 spin state.  One
"step" is one full Heun time step of every spin.  `--workload bcc_4shell_128`
selects the bcc two-sublattice four-shell model (4.19M spins, T = 300 K).

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events
on the launching stream.  A state larger than L2 (the 1e9-spin state is
25.8 GB) needs no flush; a smaller one is preceded by an L2 flush (256 MB
written, then read) before every timed step.  Barrier + synchronize on both
sides of the timed region, max over ranks.  Under torchrun every rank runs its
own independent replica (different seed); no data crosses ranks ("weak"
scaling).

Also reported: the roofline of the step (48 algorithmic bytes per spin-step:
read S^n, write S^{n+1}, FP64) and the FP64 arithmetic bound of the state
update, an end-to-end figure through the host-memory C-ABI entry (pinned host
buffers, copies inside the timed region), SM clocks sampled during the timed
region, and the CPU oracle timed on a bounded sample of the same workload.
`--impl reference` times the CPU oracle alone (the reference arm).
"""
import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "spin-site updates/s (field+Heun) and %HBM roofline on 1 GB300, vs FP64 plain path"
UNIT = "spin-steps/s"
BYTES_PER_SPIN_STEP = 48  # FP64 state: read S^n (24 B) + write S^{n+1} (24 B)
# two-pass stencil step: predictor reads S^n (24) and writes S~, f0 (12 + 12); corrector reads S~, S^n, f0
# (12 + 24 + 12) and writes S^{n+1} (24); a thermal step also writes and reads the normals (12 + 12)
EXECUTED_BYTES_TWO_PASS = 120
EXECUTED_BYTES_TWO_PASS_THERMAL = 144
# FP64 operations per spin-step of the state update (x = S + d: 3 additions; S' = x + x t: 3 fused
# multiply-adds; |x|^2 - 1 and t run in 64-bit fixed point on the integer pipe), and GB300's FP64 rate
# measured by the pipe-rate GPU test (tests/test_gpu_pipe_rates.py: 503 G FP64 FMA/s at 2070 MHz)
FP64_OPS_PER_SPIN_STEP = 6
FP64_OPS_PER_S = 503e9
# spin fields larger than this are generated on the device (numpy would take minutes at 1e9 spins)
HOST_GEN_MAX_SITES = 1 << 26

WORKLOADS = {
    "bcc_4shell_128": dict(name="bcc_4shell", n=(128, 128, 128),
                           desc="bcc 2-sublattice 128^3 cells (4,194,304 spins), J1..J4 = 20,10,-1,0.5 meV, "
                                "mu = 2.2, K = 0.005 meV || z, T = 300 K, alpha = 0.05, dt = 0.1 fs, periodic"),
    "sc_nn_32": dict(name="sc_nn", n=(32, 32, 32),
                     desc="simple cubic 32^3 (32,768 spins), NN J = 1 meV, B = 1 T || z, alpha = 0.1, dt = 0.1 fs"),
    "sc_4shell_256": dict(name="sc_4shell", n=(256, 256, 256),
                          desc="simple cubic 256^3 (16.8M spins), four-shell frustrated exchange J1..J4 = 1, 0.188, "
                               "-0.274, -0.161 meV (the hopfion Hamiltonian), open boundaries, T = 10 K, "
                               "alpha = 0.1, dt = 0.1 fs"),
    "sc_j123_dmi_1024": dict(name="sc_j123_dmi", n=(1024, 1024, 1024),
                             desc="simple cubic 1024^3 (1.07e9 spins), J1..J3 = 1,-0.164,-0.082 meV + interfacial "
                                  "DMI 0.1 meV, mu = 2.2, T = 50 K, alpha = 0.1, dt = 0.1 fs, periodic"),
    "sc_j123_dmi_256": dict(name="sc_j123_dmi", n=(256, 256, 256),
                            desc="simple cubic 256^3 (16.8M spins), J1..J3 = 1,-0.164,-0.082 meV + interfacial "
                                 "DMI 0.1 meV, mu = 2.2, T = 50 K, alpha = 0.1, dt = 0.1 fs, periodic"),
}
DEFAULT_WORKLOAD = "sc_j123_dmi_1024"


def initial_spins(nsub, n, seed, device):
    """Seeded uniform random unit spins: numpy's generator for small lattices, torch's device
    generator (the same recipe, z = 2u - 1, phi = 2 pi v) beyond HOST_GEN_MAX_SITES."""
    import torch
    from workloads import random_spins, random_spins_torch
    if nsub * n[0] * n[1] * n[2] > HOST_GEN_MAX_SITES:
        return random_spins_torch(nsub, n, seed, device=device), "device (torch Philox)"
    return torch.from_numpy(random_spins(nsub, n, seed)).to(device), "host (numpy PCG64)"


def replica_of(rank, base_seed):
    """Every rank runs an independent replica: its own seed and Philox replica index."""
    return {"seed": base_seed + 1000 * rank, "replica": rank}


def max_over_ranks(value, dist, device):
    """The timed region's duration, max over ranks (the slowest rank sets the whole-job time)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def whole_job_rate(world, units_per_rank, steps, total_ms):
    """Units processed by all ranks divided by the (max-over-ranks) timed duration."""
    return world * units_per_rank * steps / (total_ms * 1e-3)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p["hbm_gbs"], "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw samples: BENCH_CLOCKS_DIR if set (kept for inspection), else the system temporary directory
        self.path = os.path.join(os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir(),
                                 f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_oracle_rate(wl, budget_s=15.0, cells=None, steps=None, seed=7):
    """The CPU oracle on a bounded sample of the workload: a smaller lattice of the same
    Hamiltonian, timed over a few stochastic Heun steps."""
    import oracle
    from workloads import WORKLOADS as W, random_spins
    from oracle.models import oracle_model
    w = W[wl["name"]]
    ncell = cells or min(64, wl["n"][0])
    n = (ncell, ncell, ncell)
    m, _ = oracle_model(wl["name"], n)
    S = random_spins(len(w["pos"]), n, seed)
    T = w["T"]
    t0 = time.perf_counter()
    S = m.heun(S, w["dt"], w["alpha"], T=T, seed=seed, step0=0, nsteps=1)
    one = time.perf_counter() - t0
    k = steps or max(1, min(10000, int(budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    m.heun(S, w["dt"], w["alpha"], T=T, seed=seed, step0=1, nsteps=k)
    dt = time.perf_counter() - t0
    nsite = len(w["pos"]) * ncell ** 3
    return {"value": nsite * k / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{wl['name'] if 'name' in wl else ''}: {ncell}^3 cells ({nsite} spins) x {k} stochastic "
                      f"Heun steps, FP64 pair-list oracle, OpenMP", "seconds": dt}


def run_reference(args):
    wl = WORKLOADS[args.workload]
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from workloads import WORKLOADS as W, random_spins
    from oracle.models import oracle_model
    w = W[wl["name"]]
    # one reference step = one oracle Heun step on a bounded sample lattice of the same Hamiltonian,
    # sized so that K + W steps finish in about two minutes
    ncell = min(32, wl["n"][0])
    while True:
        n = (ncell, ncell, ncell)
        m, _ = oracle_model(wl["name"], n)
        S = random_spins(len(w["pos"]), n, 11)
        t0 = time.perf_counter()
        S = m.heun(S, w["dt"], w["alpha"], T=w["T"], seed=11, step0=0, nsteps=1)
        one = time.perf_counter() - t0
        if one * (args.steps + args.warmup) < 120 or ncell <= 8:
            break
        ncell = max(8, int(ncell * 0.75))
    if args.warmup > 1:
        S = m.heun(S, w["dt"], w["alpha"], T=w["T"], seed=11, step0=1, nsteps=args.warmup - 1)
    t0 = time.perf_counter()
    m.heun(S, w["dt"], w["alpha"], T=w["T"], seed=11, step0=args.warmup, nsteps=args.steps)
    dt = time.perf_counter() - t0
    nsite = len(w["pos"]) * ncell ** 3
    val = nsite * args.steps / dt
    sample = f"{ncell}^3 cells ({nsite} spins) of the same Hamiltonian, one oracle Heun step per step"
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic: seeded random unit spins",
           "config": {"workload": args.workload, "lattice": wl["desc"], "reference": "CPU FP64 pair-list oracle",
                      "sample": sample},
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# DRAM bytes per spin-step of the Heun step measured by ncu (dram__bytes_read.sum + dram__bytes_write.sum of both
# two-pass launches of one step, from the one-pass ncu launch list of the bench command), keyed by (workload, scheme, launch
# shape, plane staging, z chunk); reported as roofline.traffic when the bench runs that shape
MEASURED_TRAFFIC = {
    ("sc_j123_dmi_1024", "two_pass", 0, 0, 171): (147.6, "ncu of the 1024^3 bench step, z chunk 171, site-by-site "
                                                         "plane copies, one-pass launch list of this bench"),
    ("sc_j123_dmi_1024", "two_pass", 0, 0, 512): (152.7, "ncu of the 1024^3 bench step, z chunk 512, site-by-site "
                                                         "plane copies, one-pass launch list of this bench"),
}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    import paper_2605_26016_gb300 as sx

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    wl = WORKLOADS[args.workload]
    s, w = sx.system_from_workload(wl["name"], wl["n"])
    if args.dipolar:
        s.set_dipolar(True)
    if args.scheme != "autotune":
        sx.sx_set_stencil_scheme(s.ctx, args.scheme)
    info = s.plan(args.backend, args.precision)
    nsite = s.nsite
    rep = replica_of(rank, w["seed"])
    S, gen = initial_spins(s.nsub, wl["n"], rep["seed"], dev)
    S2 = torch.empty_like(S)
    stream = torch.cuda.current_stream()
    p = sx.llg_params(w["dt"], w["alpha"], w["T"], seed=rep["seed"], replica=rep["replica"])
    tune = None
    if args.tiles and args.backend == "stencil":
        sx.sx_set_tiles(s.ctx, "two_pass", *[int(v) for v in args.tiles.split(",")])
        info = s.info()
    elif args.scheme == "autotune" and args.backend == "stencil":
        # setup, untimed: time both stencil schemes on this replica's spins and keep the faster
        chosen, tune = sx.sx_autotune(s.ctx, S, S2, p, nsite, steps=3, stream=stream)
        info = s.info()
    tiles = sx.sx_plan_tiles(s.ctx)
    scheme = {1: "fused", 2: "two_pass"}.get(info["launches_per_step"], "fused") if args.backend == "stencil" \
        else "single"

    # the state (24 B per spin) is read and written every step; beyond the 126 MB L2 nothing stays resident
    state_bytes = 24 * nsite
    need_flush = state_bytes < 4 * 2 ** 30
    if need_flush:
        flush_w = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
        flush_r = torch.ones(256 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
        sink = torch.zeros((), dtype=torch.float32, device=dev)

    def flush(k):
        if need_flush:
            flush_w.fill_(float(k))
            sink.add_(flush_r.sum())

    bufs = [S, S2]
    step = 0
    for _ in range(args.warmup):
        sx.sx_llg_heun_step_out(s.ctx, bufs[step & 1], bufs[(step + 1) & 1], p, step, nsite, stream)
        step += 1
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(dev.index)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush(k)
        ev[k][0].record(stream)
        sx.sx_llg_heun_step_out(s.ctx, bufs[step & 1], bufs[(step + 1) & 1], p, step, nsite, stream)
        ev[k][1].record(stream)
        step += 1
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    times = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(times)
    if world > 1:
        total_ms = max_over_ranks(total_ms, dist, dev)
    # sanity: the state stays on the unit sphere
    Sf = bufs[step & 1]
    norm_err = (Sf.view(3, -1).pow(2).sum(0).sqrt() - 1).abs().max().item()

    # end to end: host buffers through the C ABI, copies inside the timed region
    e2e_steps = max(3, min(20 if nsite <= HOST_GEN_MAX_SITES else 3, args.steps))
    Sh = Sf.cpu().pin_memory()
    sx.sx_llg_heun_host(s.ctx, Sh, p, step, 1, nsite, stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        sx.sx_llg_heun_host(s.ctx, Sh, p, step + 1 + k, 1, nsite, stream)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if world > 1:
        e2e_s = max_over_ranks(e2e_s, dist, dev)

    if rank != 0:
        dist.destroy_process_group()
        return
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(world, nsite, args.steps, total_ms)
    hbm, peak_kind = peaks()
    launches = info["launches_per_step"]
    achieved = BYTES_PER_SPIN_STEP * nsite / (ms_per_step * 1e-3) / 1e9
    traffic, traffic_src = args.traffic, "--traffic" if args.traffic is not None else None
    meas = MEASURED_TRAFFIC.get((args.workload, scheme, tiles.get("ring_or_schedule", 0), tiles.get("tma_staging", 0),
                                 tiles.get("tile_z", 0)))
    if traffic is None and meas is not None and args.backend == "stencil":
        traffic, traffic_src = meas[0] * nsite, meas[1]
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": traffic, "traffic_source": traffic_src, "peak_kind": peak_kind,
            "kernel": "heun step, %s scheme (%d launch%s per step)" % (scheme, launches,
                                                                       "" if launches == 1 else "es"),
            "bytes_per_unit": BYTES_PER_SPIN_STEP, "units_per_launch": nsite}
    if scheme == "two_pass":
        # the two-pass scheme moves S~ and f0 through HBM: 120 executed bytes per spin-step
        eb = EXECUTED_BYTES_TWO_PASS_THERMAL if w["T"] > 0 else EXECUTED_BYTES_TWO_PASS
        own = eb * nsite / (ms_per_step * 1e-3) / 1e9
        roof.update({"executed_bytes_per_unit": eb, "achieved_executed": own,
                     "frac_executed": own / hbm})
    if args.backend == "stencil" and args.precision == "fp32":
        # the FP64 state update bounds the step too: FP64_OPS_PER_SPIN_STEP at the measured FP64 rate
        rate = value / world
        cap = FP64_OPS_PER_S / FP64_OPS_PER_SPIN_STEP
        hbm_cap = hbm * 1e9 / BYTES_PER_SPIN_STEP
        roof["alu"] = {"bound": "fp64", "ops_per_unit": FP64_OPS_PER_SPIN_STEP, "peak_ops_per_s": FP64_OPS_PER_S,
                       "peak_kind": "measured (pipe-rate GPU test: independent FP64 FMA chains on every SM)",
                       "achieved_ops_per_s": rate * FP64_OPS_PER_SPIN_STEP, "frac": rate / cap,
                       "cap_units_per_s": cap}
        roof["binds"] = "fp64" if cap < hbm_cap else "hbm"
        roof["cap_frac_of_hbm_roofline"] = min(cap, hbm_cap) / hbm_cap
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32-field/f64-state" if args.precision == "fp32" else args.precision,
           "data": "synthetic: seeded random unit spins; every rank an independent replica",
           "config": {"workload": args.workload, "lattice": wl["desc"], "backend": args.backend, "dipolar": args.dipolar,
                      "precision": args.precision, "nsite_per_gpu": nsite, "parallelism": f"replicas x{world}",
                      "stencil_scheme": scheme, "autotune_ms": tune, "tiles": tiles, "initial_spins": gen,
                      "l2": ("flushed before every timed step (256 MB write + 256 MB read)" if need_flush else
                             "no flush: the %.1f GB state is far larger than the 126 MB L2" % (state_bytes / 1e9)),
                      "median_step_ms": statistics.median(times), "wall_s": t_wall, "max_norm_error": norm_err},
           "roofline": roof,
           "e2e": {"value": world * nsite / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 24 * nsite,
                   "d2h_bytes_per_step": 24 * nsite, "steps": e2e_steps,
                   "path": "sx_llg_heun_host, pinned host buffers, one Heun step per call"},
           "gpu_launches": launches * args.steps, "clocks": clk}
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_oracle_rate(wl)
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------------------------------------ profiling drivers
# `python bench.py --profile KIND ARGS...` runs one of the workloads below a few times and prints a JSON line;
# the ncu summaries run these drivers (alone for CUDA-event timings, under ncu for captures).


def _profile_step(argv):
    """step WORKLOAD NX,NY,NZ [STEPS=3] [BACKEND=stencil] [PRECISION=fp32] [SCHEME=auto|fused|two_pass|field]
    [STAGING=default|tma|copy|MASK] [SHAPE=TZ,LAUNCH] out-of-place Heun steps (or field evaluations with
    SCHEME=field) of a workload; STAGING sets the plane staging of the stencil pass kernels (tensor copies for
    every pass, site-by-site copies, or the mask of sx_set_tiles in[4]), SHAPE the two-pass z chunk and launch
    shape (sx_set_tiles in[1], in[2])."""
    import torch
    import paper_2605_26016_gb300 as sx
    name = argv[0]
    n = tuple(int(v) for v in argv[1].split(","))
    steps = int(argv[2]) if len(argv) > 2 else 3
    backend = argv[3] if len(argv) > 3 else "stencil"
    prec = argv[4] if len(argv) > 4 else "fp32"
    scheme = argv[5] if len(argv) > 5 else "auto"
    s, w = sx.system_from_workload(name, n)
    if backend == "stencil" and scheme in ("auto", "fused", "two_pass"):
        sx.sx_set_stencil_scheme(s.ctx, scheme)
    info = s.plan(backend, prec)
    staging = argv[6] if len(argv) > 6 else "default"
    staging = int(staging) if staging.isdigit() else staging
    shape = [int(v) for v in argv[7].split(",")] if len(argv) > 7 else None
    if backend == "stencil" and (staging != "default" or shape):
        t = sx.sx_plan_tiles(s.ctx)
        tz, launch = shape if shape else (t["tile_z"] or n[2], t["ring_or_schedule"])
        sx.sx_set_tiles(s.ctx, t["scheme"], tz, launch, t["regen_noise"],
                        t["tma_staging"] if staging == "default" else {"copy": 0, "tma": 3}.get(staging, staging))
    tiles = sx.sx_plan_tiles(s.ctx)
    S, gen = initial_spins(s.nsub, n, 1, "cuda")
    bufs = [S, torch.empty_like(S)]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    p = sx.llg_params(w["dt"], w["alpha"], w["T"], seed=3)
    ev[0].record()
    for k in range(steps):
        if scheme == "field":
            s.field(S, bufs[1])
        else:
            sx.sx_llg_heun_step_out(s.ctx, bufs[k & 1], bufs[(k + 1) & 1], p, k, s.nsite)
        ev[k + 1].record()
    torch.cuda.synchronize()
    ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
    print(json.dumps({"profile": "step", "workload": f"{name} {n}", "plan": info, "tiles": tiles, "ms": ms,
                      "input": gen}))


def _profile_min(argv):
    """min [BACKEND=stencil] [PRECISION=fp32] [METHOD=vp] [TOL=1e-6] [MAX_ITER=20000] [L=100]
    energy minimisation of the hopfion workload (SC L^3, J1..J3 distance shells, open z, Hopf ansatz R = 12)."""
    import torch
    import paper_2605_26016_gb300 as sx
    from workloads import hopf_ansatz
    backend = argv[0] if len(argv) > 0 else "stencil"
    prec = argv[1] if len(argv) > 1 else "fp32"
    method = argv[2] if len(argv) > 2 else "vp"
    tol = float(argv[3]) if len(argv) > 3 else 1e-6
    max_iter = int(argv[4]) if len(argv) > 4 else 20000
    L = int(argv[5]) if len(argv) > 5 else 100
    n = (L, L, L)
    s, w = sx.system_from_workload("sc_j123", n)
    s.plan(backend, prec)
    S = torch.from_numpy(hopf_ansatz(n, 12.0)).cuda()
    e0 = s.energy(S)["total"]
    kw = dict(method=method, tol=tol, max_iter=max_iter, check_every=200)
    kw.update(dict(dt=0.1) if method == "vp" else dict(dt=1.0, alpha=1.0))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    it, tq = s.minimise(S, **kw)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    e1 = s.energy(S)["total"]
    print(json.dumps({"profile": "min", "workload": f"sc_j123 {L}^3 open z, Hopf ansatz R=12", "backend": backend,
                      "precision": prec, "method": method, "tol_meV": tol, "iterations": it, "ms": ms,
                      "ms_per_iteration": ms / max(it, 1), "final_torque_meV": tq, "energy_before": e0,
                      "energy_after": e1, "min_Sz": S[2].min().item()}))


def _profile_path(argv):
    """path [WORKLOAD=bcc_4shell] [NX,NY,NZ=64,64,64] [IMAGES=32] [ITERATIONS=50] [BACKEND=stencil]
    [PRECISION=fp32] [METHOD=ci_gneb] [OPTIMIZER=steepest]: path-method iterations on a chain from the
    uniform +z state to a seeded random state (site-wise normalised blend, 2% seeded jitter)."""
    import torch
    import paper_2605_26016_gb300 as sx
    from workloads import nlerp_chain, random_spins, uniform_spins
    name = argv[0] if len(argv) > 0 else "bcc_4shell"
    n = tuple(int(v) for v in argv[1].split(",")) if len(argv) > 1 else (64, 64, 64)
    nimg = int(argv[2]) if len(argv) > 2 else 32
    iters = int(argv[3]) if len(argv) > 3 else 50
    backend = argv[4] if len(argv) > 4 else "stencil"
    prec = argv[5] if len(argv) > 5 else "fp32"
    method = argv[6] if len(argv) > 6 else "ci_gneb"
    optimizer = argv[7] if len(argv) > 7 else "steepest"
    s, w = sx.system_from_workload(name, n)
    s.plan(backend, prec)
    A = uniform_spins(s.nsub, n, [0.0, 0.0, 1.0])
    B = random_spins(s.nsub, n, 41)
    chain = torch.from_numpy(nlerp_chain(A, B, nimg, jitter=0.02, seed=4)).cuda()
    dt = 2e-4 if name == "bcc_4shell" else 0.02
    kw = dict(method=method, dt=dt, k_spring=1.0, tol=0.0, optimizer=optimizer)
    s.path(chain, max_iter=3, check_every=3, **kw)  # warm-up (allocates the workspace)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    it, E, fm = s.path(chain, max_iter=iters, check_every=iters, **kw)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    rate = (nimg - 2) * s.nsite * iters / (ms * 1e-3)
    hbm, _ = peaks()
    gbs = 48.0 * rate / 1e9
    print(json.dumps({"profile": "path", "workload": f"{name} {n[0]}x{n[1]}x{n[2]} x{s.nsub} sublattices, {nimg} images",
                      "method": method, "optimizer": optimizer, "backend": backend, "precision": prec,
                      "iterations": it, "ms_per_iteration": ms / iters, "image_site_iterations_per_s": rate,
                      "hbm_gbs_at_48B": gbs, "frac_of_measured_hbm": gbs / hbm, "fmax": fm,
                      "energy_span": max(E) - min(E)}))


def _profile_batch(argv):
    """batch [WORKLOAD=bcc_4shell] [NREP=64] [LMIN=24] [LMAX=96] [STEPS=20] [SEED=4]: an ensemble of replicas
    (cubes of L^3 cells, L ~ U{LMIN..LMAX}) advanced by the batched step against one launch pair per replica."""
    import numpy as np
    import torch
    import paper_2605_26016_gb300 as sx
    from workloads import random_spins
    name = argv[0] if len(argv) > 0 else "bcc_4shell"
    nrep = int(argv[1]) if len(argv) > 1 else 64
    lmin = int(argv[2]) if len(argv) > 2 else 24
    lmax = int(argv[3]) if len(argv) > 3 else 96
    steps = int(argv[4]) if len(argv) > 4 else 20
    seed = int(argv[5]) if len(argv) > 5 else 4
    rng = np.random.default_rng(seed)
    edges = rng.integers(lmin, lmax + 1, size=nrep)
    systems = []
    for L in edges:
        s, w = sx.system_from_workload(name, (int(L), int(L), int(L)))
        sx.sx_set_stencil_scheme(s.ctx, "two_pass")
        s.plan("stencil", "fp32")
        systems.append(s)
    nsite = sum(s.nsite for s in systems)
    batch = sx.Batch(systems)
    p = sx.llg_params(w["dt"], w["alpha"], w["T"], seed=seed)
    A = [torch.from_numpy(random_spins(s.nsub, s.n, 100 + r)).cuda() for r, s in enumerate(systems)]
    B = [torch.empty_like(x) for x in A]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    state = {"A": A, "B": B}

    def run_batch(k0):
        for k in range(steps):
            batch.heun_step(state["A"], state["B"], p, k0 + k)
            state["A"], state["B"] = state["B"], state["A"]

    def run_single(k0):
        for k in range(steps):
            for r, s in enumerate(systems):
                pr = sx.llg_params(w["dt"], w["alpha"], w["T"], seed=seed, replica=r)
                sx.sx_llg_heun_step_out(s.ctx, state["A"][r], state["B"][r], pr, k0 + k, s.nsite)
            state["A"], state["B"] = state["B"], state["A"]

    out = {"profile": "batch", "workload": f"{name}: {nrep} replicas, L ~ U{{{lmin}..{lmax}}} cells, {nsite} spins",
           "steps": steps}
    for label, fn in (("batched", run_batch), ("one_launch_pair_per_replica", run_single)):
        fn(0)
        torch.cuda.synchronize()
        e0.record()
        fn(1000)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[label] = {"ms_per_step": ms, "spin_steps_per_s": nsite / (ms * 1e-3)}
    print(json.dumps(out))


def _profile_field(argv):
    """field [WORKLOAD=dense7] [N=100] [BACKENDS=igemm_tc/tf32,igemm_tc/bf16,stencil/fp32,gather/fp32,fft/fp32]
    [REPS=20]: time the field (FP64 output, on-site terms) of one backend after another on seeded random spins of an
    N^3 lattice.  dense7 is a 3x3 tensor coupling on every offset of the 7x7x7 window (workloads.dense_window_bonds);
    other names are the workloads of this file."""
    import torch
    import paper_2605_26016_gb300 as sx
    from workloads import cubic_cell, dense_window_bonds, random_spins_torch
    name = argv[0] if len(argv) > 0 else "dense7"
    n = (int(argv[1]),) * 3 if len(argv) > 1 else (100, 100, 100)
    backends = (argv[2] if len(argv) > 2 else "igemm_tc/tf32,igemm_tc/bf16,stencil/fp32,gather/fp32,fft/fp32").split(",")
    reps = int(argv[3]) if len(argv) > 3 else 20

    def system():
        if name == "dense7":
            s = sx.SpinSystem(n, (1, 1, 1), cubic_cell(), [[0, 0, 0]], [1.0])
            s.add_bonds(dense_window_bonds())
            return s
        return sx.system_from_workload(name, n)[0]

    s0 = system()
    S = random_spins_torch(s0.nsub, n, 1)
    out = torch.empty_like(S)
    res = {"profile": "field", "workload": f"{name} {n[0]}x{n[1]}x{n[2]}", "nsite": s0.nsite}
    s0.close()
    for bp in backends:
        backend, prec = bp.split("/")
        s = system()
        try:
            s.plan(backend, prec)
        except sx.SxError as e:
            res[bp] = f"unsupported: {e}"
            continue
        for _ in range(3):
            s.field(S, out=out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            s.field(S, out=out)
        e1.record()
        torch.cuda.synchronize()
        res[bp] = {"us": 1e3 * e0.elapsed_time(e1) / reps}
        s.close()
    print(json.dumps(res))


def _profile_ensemble(argv):
    """ensemble [WORKLOAD=bcc_4shell] [NREP=64] [LMIN=24] [LMAX=96] [STEPS=20] [NIMG=32] [IMG_L=64] [SEED=4]: uneven
    replicas (cubes of L^3 cells, L ~ U{LMIN..LMAX}) advanced STEPS Heun steps plus the field of NIMG chain images
    (IMG_L^3 cells): one persistent sx_batch_run against per-step batched launches plus one field launch per image,
    and against one launch pair per replica and step."""
    import numpy as np
    import torch
    import paper_2605_26016_gb300 as sx
    from workloads import random_spins
    name = argv[0] if len(argv) > 0 else "bcc_4shell"
    nrep = int(argv[1]) if len(argv) > 1 else 64
    lmin = int(argv[2]) if len(argv) > 2 else 24
    lmax = int(argv[3]) if len(argv) > 3 else 96
    steps = int(argv[4]) if len(argv) > 4 else 20
    nimg = int(argv[5]) if len(argv) > 5 else 32
    limg = int(argv[6]) if len(argv) > 6 else 64
    seed = int(argv[7]) if len(argv) > 7 else 4
    rng = np.random.default_rng(seed)
    edges = rng.integers(lmin, lmax + 1, size=nrep)
    systems = []
    for L in edges:
        s, w = sx.system_from_workload(name, (int(L), int(L), int(L)))
        sx.sx_set_stencil_scheme(s.ctx, "two_pass")
        s.plan("stencil", "fp32")
        systems.append(s)
    img_s, _ = sx.system_from_workload(name, (limg, limg, limg))
    img_s.plan("stencil", "fp32")
    nsite = sum(s.nsite for s in systems)
    batch = sx.Batch(systems, image_system=img_s, nimg=nimg)
    p = sx.llg_params(w["dt"], w["alpha"], w["T"], seed=seed)
    A = [torch.from_numpy(random_spins(s.nsub, s.n, 100 + r)).cuda() for r, s in enumerate(systems)]
    B = [torch.empty_like(x) for x in A]
    images = torch.from_numpy(np.stack([random_spins(img_s.nsub, img_s.n, 500 + k) for k in range(nimg)])).cuda()
    fields = torch.empty_like(images)
    batch.bind(A, B, images, fields)
    state = {"A": A, "B": B}

    def run_combined(k0):
        batch.run(p, k0, steps)

    def run_batched(k0):
        for k in range(steps):
            batch.heun_step(state["A"], state["B"], p, k0 + k)
            state["A"], state["B"] = state["B"], state["A"]
        for k in range(nimg):
            img_s.field(images[k], out=fields[k])

    def run_single(k0):
        for k in range(steps):
            for r, s in enumerate(systems):
                pr = sx.llg_params(w["dt"], w["alpha"], w["T"], seed=seed, replica=r)
                sx.sx_llg_heun_step_out(s.ctx, state["A"][r], state["B"][r], pr, k0 + k, s.nsite)
            state["A"], state["B"] = state["B"], state["A"]
        for k in range(nimg):
            img_s.field(images[k], out=fields[k])

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"profile": "ensemble", "workload": f"{name}: {nrep} replicas, L ~ U{{{lmin}..{lmax}}} cells, {nsite} spins, "
           f"{steps} steps; {nimg} images of {limg}^3 cells", "persistent": batch.info()["persistent"]}
    for label, fn in (("one_persistent_launch", run_combined), ("batched_launch_pairs_plus_field_per_image",
                                                                 run_batched),
                      ("launch_pair_per_replica_plus_field_per_image", run_single)):
        fn(0)
        torch.cuda.synchronize()
        e0.record()
        fn(1000)
        e1.record()
        torch.cuda.synchronize()
        batch.status()
        ms = e0.elapsed_time(e1)
        out[label] = {"ms": ms, "replica_spin_steps_per_s": nsite * steps / (ms * 1e-3)}
    print(json.dumps(out))


def _profile_cnn(argv):
    """cnn [NX,NY,NZ=64,64,64] [BATCH=30] [REPEATS=20] [MODE=both|forward|train]: the chain proposer's
    inference and one training step on seeded random unit fields."""
    import torch
    import paper_2605_26016_gb300 as sx
    from workloads import cnn_init_flat, random_spins_torch
    n = tuple(int(v) for v in argv[0].split(",")) if len(argv) > 0 else (64, 64, 64)
    nb = int(argv[1]) if len(argv) > 1 else 30
    reps = int(argv[2]) if len(argv) > 2 else 20
    mode = argv[3] if len(argv) > 3 else "both"
    ncell = n[0] * n[1] * n[2]
    P = sx.Proposer(n, nb)
    P.set_params(cnn_init_flat(7))
    A = random_spins_torch(1, n, 1).reshape(3, ncell)
    B = random_spins_torch(1, n, 2).reshape(3, ncell)
    I = torch.stack([random_spins_torch(1, n, 10 + b).reshape(3, ncell) for b in range(nb)])
    T = torch.stack([random_spins_torch(1, n, 100 + b).reshape(3, ncell) for b in range(nb)])
    s = torch.linspace(0.05, 0.95, nb, dtype=torch.float64, device="cuda")
    X = P.new_packed(nb)
    P.pack(I, A, B, s, X, shared_endpoints=True)
    out = torch.empty_like(I)
    st = torch.cuda.current_stream()
    res = {"profile": "cnn", "workload": f"proposer {n[0]}x{n[1]}x{n[2]}, {nb} samples", "sites": nb * ncell}

    def timed(fn):
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    if mode in ("both", "forward"):
        ms = timed(lambda: P.forward(X, I, out))
        flops = 2 * 27 * (10 * 16 + 16 * 16 + 16 * 16 + 16 * 3) * nb * ncell
        res.update(forward_ms=ms, forward_sites_per_s=nb * ncell / (ms * 1e-3),
                   forward_useful_tflops=flops / (ms * 1e-3) / 1e12,
                   forward_algorithmic_gbs=4 * 64 * nb * ncell / (ms * 1e-3) / 1e9)
    if mode in ("both", "train"):
        def step():
            P.loss_grad(X, I, T)
            P.adam_step(1e-4)
        ms = timed(step)
        res.update(train_step_ms=ms, train_sites_per_s=nb * ncell / (ms * 1e-3))
    print(json.dumps(res))
    P.close()


PROFILES = {"step": _profile_step, "min": _profile_min, "path": _profile_path, "batch": _profile_batch,
            "ensemble": _profile_ensemble, "field": _profile_field, "cnn": _profile_cnn}


def main():
    if len(sys.argv) > 2 and sys.argv[1] == "--profile":
        if sys.argv[2] not in PROFILES:
            raise SystemExit("--profile KIND: one of " + ", ".join(sorted(PROFILES)))
        PROFILES[sys.argv[2]](sys.argv[3:])
        return
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0],
                                 epilog="python bench.py --profile {%s} ARGS...: the profiling drivers" %
                                        ",".join(sorted(PROFILES)))
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--backend", default="stencil")
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--traffic", type=float, default=None,
                    help="dram bytes per launch of the step kernel from an ncu capture (GB/s roofline context)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--dipolar", action="store_true", help="add the point-dipole field (FFT backend)")
    ap.add_argument("--tiles", default=None,
                    help="TZ,LAUNCH,REGEN,MASK: run the two-pass scheme with this tile shape (sx_set_tiles in[1..4]) "
                         "instead of autotuning")
    ap.add_argument("--scheme", choices=["autotune", "auto", "fused", "two_pass"], default="autotune",
                    help="stencil Heun scheme (default: time both on the bench's spins, keep the faster)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
