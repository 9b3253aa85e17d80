"""Time the energy minimisation of the hopfion workload on one backend (the static-optimisation
workload: SC 100^3, J1..J3 distance shells, open z, Hopf-map ansatz of radius 12).

    python -m paper_2605_26016_gb300.profile_min [backend] [precision] [method] [tol] [max_iter] [n]

Defaults: stencil, fp32, vp, 1e-6 meV, 20000 iterations, 100.  Prints one JSON line: iterations,
wall time (CUDA events around the call), final max |S x b|, energy before and after, and the
minimum of S_z (the hopfion core survives while it stays near -1).
"""
import json
import os
import sys


def main(argv):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
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
    print(json.dumps({"workload": f"sc_j123 {L}^3 open z, Hopf ansatz R=12", "backend": backend, "precision": prec,
                      "method": method, "tol_meV": tol, "iterations": it, "ms": ms, "ms_per_iteration": ms / max(it, 1),
                      "final_torque_meV": tq, "energy_before": e0, "energy_after": e1,
                      "min_Sz": S[2].min().item()}))


if __name__ == "__main__":
    main(sys.argv[1:])
