"""Throughput benchmark: spin-site updates per second of the fused field + Heun step.

Workload (default): bcc iron-like lattice as two sublattices, 128^3 conventional
cells = 4,194,304 spins, isotropic exchange on four distance shells
(J = 20, 10, -1, 0.5 meV), mu = 2.2 mu_B, uniaxial K = 0.005 meV along z,
stochastic Heun LLG at T = 300 K, alpha = 0.05, dt = 0.1 fs, FP32 field with
FP64 spin state.  One "step" is one full Heun time step of every spin.

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events
on the launching stream; before every timed step L2 is flushed by writing and
then reading 256 MB buffers (the spin state, 100 MB, would otherwise partly
stay in the 126 MB L2).  Barrier + synchronize on both sides of the timed
region, max over ranks.  Under torchrun every rank runs its own independent
replica (different seed); no data crosses ranks ("weak" scaling).

Also reported: the roofline of the step kernel (48 algorithmic bytes per
spin-step: read S^n, write S^{n+1}, FP64), an end-to-end figure through the
host-memory C-ABI entry (pinned host buffers, copies inside the timed region),
SM clocks sampled during the timed region, and the CPU oracle timed on a
bounded sample of the same workload.  `--impl reference` times the CPU oracle
alone (the reference arm).
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
}


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


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    import paper_2605_26016_gb300 as sx
    from workloads import random_spins

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
    S = torch.from_numpy(random_spins(s.nsub, wl["n"], rep["seed"])).to(dev)
    S2 = torch.empty_like(S)
    stream = torch.cuda.current_stream()
    p = sx.llg_params(w["dt"], w["alpha"], w["T"], seed=rep["seed"], replica=rep["replica"])
    tune = None
    if args.scheme == "autotune" and args.backend == "stencil":
        # setup, untimed: time both stencil schemes on this replica's spins and keep the faster
        chosen, tune = sx.sx_autotune(s.ctx, S, S2, p, nsite, steps=5, stream=stream)
        info = s.info()
    scheme = {1: "fused", 2: "two_pass"}.get(info["launches_per_step"], "fused") if args.backend == "stencil" \
        else "single"

    flush_w = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    flush_r = torch.ones(256 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    sink = torch.zeros((), dtype=torch.float32, device=dev)

    def flush(k):
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
    e2e_steps = max(3, min(20, args.steps))
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
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": args.traffic, "peak_kind": peak_kind,
            "kernel": "heun step, %s scheme (%d launch%s per step)" % (scheme, launches,
                                                                       "" if launches == 1 else "es"),
            "bytes_per_unit": BYTES_PER_SPIN_STEP, "units_per_launch": nsite}
    if scheme == "two_pass":
        # the two-pass scheme moves S~ and f0 through HBM: 120 executed bytes per spin-step
        eb = EXECUTED_BYTES_TWO_PASS_THERMAL if w["T"] > 0 else EXECUTED_BYTES_TWO_PASS
        own = eb * nsite / (ms_per_step * 1e-3) / 1e9
        roof.update({"executed_bytes_per_unit": eb, "achieved_executed": own,
                     "frac_executed": own / hbm})
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32-field/f64-state" if args.precision == "fp32" else args.precision,
           "data": "synthetic: seeded random unit spins; every rank an independent replica",
           "config": {"workload": args.workload, "lattice": wl["desc"], "backend": args.backend, "dipolar": args.dipolar,
                      "precision": args.precision, "nsite_per_gpu": nsite, "parallelism": f"replicas x{world}",
                      "stencil_scheme": scheme, "autotune_ms": tune,
                      "l2": "flushed before every timed step (256 MB write + 256 MB read)",
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


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="bcc_4shell_128")
    ap.add_argument("--backend", default="stencil")
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--traffic", type=float, default=None,
                    help="dram bytes per launch of the step kernel from an ncu capture (GB/s roofline context)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--dipolar", action="store_true", help="add the point-dipole field (FFT backend)")
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
