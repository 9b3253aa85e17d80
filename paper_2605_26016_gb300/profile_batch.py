"""Time an ensemble of replicas of one Hamiltonian advanced by the batched step against stepping each
replica on its own (the replica-ensemble workload: cubes of L^3 cells with L drawn uniformly).

    python -m paper_2605_26016_gb300.profile_batch [workload] [nrep] [Lmin] [Lmax] [steps] [seed]

Defaults: bcc_4shell, 64 replicas, L ~ U{24..96}, 20 timed steps, seed 4.  Prints one JSON line with
spin-steps per second for both ways.
"""
import json
import os
import sys


def main(argv):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
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

    def run_batch(k0):
        nonlocal A, B
        for k in range(steps):
            batch.heun_step(A, B, p, k0 + k)
            A, B = B, A

    def run_single(k0):
        nonlocal A, B
        for k in range(steps):
            for r, s in enumerate(systems):
                pr = sx.llg_params(w["dt"], w["alpha"], w["T"], seed=seed, replica=r)
                sx.sx_llg_heun_step_out(s.ctx, A[r], B[r], pr, k0 + k, s.nsite)
            A, B = B, A

    out = {"workload": f"{name}: {nrep} replicas, L ~ U{{{lmin}..{lmax}}} cells, {nsite} spins", "steps": steps}
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


if __name__ == "__main__":
    main(sys.argv[1:])
