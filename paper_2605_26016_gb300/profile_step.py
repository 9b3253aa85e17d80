"""Run a few out-of-place Heun steps of a workload (the launch bench.py times); used for ncu captures.

    python -m paper_2605_26016_gb300.profile_step bcc_4shell 128,128,128 3 [backend] [precision] [field]

With the last argument `field` it runs that many field evaluations (sx_field) instead of Heun steps.
"""
import os
import sys


def main(argv):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch
    import paper_2605_26016_gb300 as sx
    from workloads import random_spins
    name = argv[0]
    n = tuple(int(v) for v in argv[1].split(","))
    steps = int(argv[2]) if len(argv) > 2 else 3
    backend = argv[3] if len(argv) > 3 else "stencil"
    prec = argv[4] if len(argv) > 4 else "fp32"
    field_only = len(argv) > 5 and argv[5] == "field"
    s, w = sx.system_from_workload(name, n)
    print(s.plan(backend, prec))
    S = torch.from_numpy(random_spins(s.nsub, n, 1)).cuda()
    bufs = [S, torch.empty_like(S)]
    if field_only:
        for _ in range(steps):
            s.field(S, bufs[1])
        torch.cuda.synchronize()
        print("ok")
        return
    p = sx.llg_params(w["dt"], w["alpha"], w["T"], seed=3)
    for k in range(steps):
        sx.sx_llg_heun_step_out(s.ctx, bufs[k & 1], bufs[(k + 1) & 1], p, k, s.nsite)
    torch.cuda.synchronize()
    print("ok")


if __name__ == "__main__":
    main(sys.argv[1:])
