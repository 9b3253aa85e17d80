"""Time iterations of a path method on a chain of images (the batched string / GNEB workload).

    python -m paper_2605_26016_gb300.profile_path [workload] [nx,ny,nz] [images] [iterations] \
        [backend] [precision] [method] [optimizer]

Defaults: bcc_4shell, 64,64,64 (524,288 spins per image), 32 images, 50 iterations, stencil, fp32,
ci_gneb, steepest (or vp: velocity projection, GNEB and CI-GNEB only).  The chain runs from the
uniform state along +z to a seeded random state, interior images the site-wise normalised blend
with 2% seeded jitter.  Prints one JSON line: image-site
iterations per second (interior images x sites x iterations / time), the time per iteration
from CUDA events around one call of all timed iterations, and the HBM roofline of the
iteration at 48 algorithmic bytes per image-site (read S, write S').
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
    info = s.plan(backend, prec)
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
    # the call also evaluates the endpoint energies and the final energies (one field pass)
    units = (nimg - 2) * s.nsite * iters
    rate = units / (ms * 1e-3)
    peak = None
    try:
        with open(os.path.join(root, "MEASURED_PEAKS.json")) as f:
            peak = json.load(f).get("hbm_gbs")
    except (OSError, ValueError):
        pass
    gbs = 48.0 * rate / 1e9
    field = "one batched field launch" if backend == "stencil" else "one field launch per image"
    launches = f"{field} ({nimg - 2} images) + {6 if optimizer == 'vp' else 4} path kernels"
    print(json.dumps({"workload": f"{name} {n[0]}x{n[1]}x{n[2]} x{s.nsub} sublattices, {nimg} images",
                      "method": method, "optimizer": optimizer, "backend": backend, "precision": prec, "iterations": it,
                      "ms_per_iteration": ms / iters, "image_site_iterations_per_s": rate,
                      "hbm_gbs_at_48B": gbs, "frac_of_measured_hbm": (gbs / peak) if peak else None,
                      "launches_per_iteration": launches,
                      "fmax": fm, "energy_span": max(E) - min(E)}))


if __name__ == "__main__":
    main(sys.argv[1:])
