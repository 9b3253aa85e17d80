"""Learned chain proposals for minimum-energy paths: generate converged paths, train the proposer, compare.

    python -m paper_2605_26016_gb300.proposer_workflow [L] [ntrain] [ntest] [train_seconds] [max_iters] \
        [params_out.npy] [params_in.npy]

Defaults: L = 32 (simple cubic L^3, open boundaries), 200 training paths, 12 test paths, 200 s of training,
at most 20000 path iterations per run.

Hamiltonian family: the four-shell frustrated exchange of the hopfion calculation (J1 = 1 meV, J2/J1 = 0.188,
J3/J1 = -0.274, J4/J1 = -0.161), with J2..J4 scaled by seeded factors in [0.97, 1.03] and a Zeeman field
B_z in [0, 0.04] T per path (stronger fields or larger changes shrink the barrier to nothing).  Endpoint
A is a hopfion (Hopf ansatz of seeded radius 8..10 and centre offset +-2 sites, relaxed by velocity
projection); endpoint B is the ferromagnet along +z.

Fields come from the stencil backend's four-shell family (FP32 field, FP64 state).  A path is a chain of
16 images relaxed with velocity projection (dt = 0.05, k = 1 meV/rad, calls of 1000
iterations that carry the velocity) in two stages, as GNEB refinement is followed by climbing-image
refinement in the paper: GNEB until the largest site force is below 1e-2 meV, then CI-GNEB from rest until
it is below 1e-3 meV (J1 = 1 meV; the paper keeps the path force below about 1e-3 J1), at most max_iters
iterations in all.  A run whose barrier exceeds the hopfion energy scale E(A) - E(B) has left the basin of
the path and is stopped as diverged.  Training paths start from the
geodesic interpolation; only converged paths with a barrier between 1% of E(A) - E(B) and E(A) - E(B) are
kept (near-zero barriers are paths along which the hopfion hardly resists and teach the proposer nothing about
the saddle).  Paths are generated on 8 CUDA streams from 8 host threads (distinct contexts are independent).

The proposer (include/sx.h, sx_cnn_*) is trained with Adam on (interpolated image, A, B, s) -> converged
image over all interior images of the training paths, batches of 28 samples, cosine learning-rate decay.

Evaluation on held-out Hamiltonians: each test path is relaxed twice on one stream, from the geodesic
interpolation (plain) and from the proposer's chain (learned, falling back to the geodesic interpolation
when its run diverges, the fallback's time included), recording wall-clock seconds (proposal included),
iterations, the converged barrier (climbing-image energy minus E(A)) and the force.  With params_in the
training paths and the training are skipped and the proposer's parameters are read from that file.  Two
converged barriers are the same when they differ by at most 1e-3 of the hopfion energy scale E(A) - E(B);
otherwise the runs found different annihilation channels.  Where the learned run finds the lower barrier, a
third arm checks that channel: a plain run from the piecewise geodesic chain through the learned run's
climbing image (A -> saddle -> B) must reach the same barrier.  Prints one JSON line per stage and a summary.
"""
import json
import os
import sys
import threading
import time


def main(argv):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import numpy as np
    import torch
    import paper_2605_26016_gb300 as sx
    from workloads import cnn_init_flat, cubic_cell, hopf_ansatz, uniform_spins

    L = int(argv[0]) if len(argv) > 0 else 32
    ntrain = int(argv[1]) if len(argv) > 1 else 200
    ntest = int(argv[2]) if len(argv) > 2 else 12
    train_s = float(argv[3]) if len(argv) > 3 else 200.0
    max_iters = int(argv[4]) if len(argv) > 4 else 20000
    ftol, chunk = 1e-3, 1000
    min_barrier_frac = 0.01
    nimg, dt = 16, 0.05
    n = (L, L, L)
    ncell = L ** 3
    shells = (1.0, 0.188, -0.274, -0.161)

    def system(h):
        s = sx.SpinSystem(n, (0, 0, 0), cubic_cell(), [[0, 0, 0]], [1.0])
        for k, J in enumerate(shells):
            s.add_shell_exchange(k + 1, J * (h["f"][k - 1] if k > 0 else 1.0))
        s.set_zeeman([0.0, 0.0, h["B"]])
        s.plan("stencil", "fp32")
        return s

    rng = np.random.default_rng(2605)
    hams = [dict(f=rng.uniform(0.97, 1.03, 3).tolist(), B=float(rng.uniform(0.0, 0.04)), R=float(rng.uniform(8, 10)),
                 c=(rng.uniform(-2, 2, 3) + (L - 1) / 2).tolist()) for _ in range(ntrain + ntest)]
    FM = torch.from_numpy(uniform_spins(1, n, [0.0, 0.0, 1.0])).cuda()
    helper = sx.Proposer(n, nimg - 2)

    def geodesic_chain(A, stream=None):
        chain = torch.empty((nimg, 3, ncell), dtype=torch.float64, device="cuda")
        chain[0].copy_(A.view(3, ncell))
        chain[-1].copy_(FM.view(3, ncell))
        helper.interpolate(chain, stream=stream)
        return chain

    # ------------------------------------------------------------ converged paths
    def relax(s, chain, t0, stream=None):
        """Two-stage VP relaxation (GNEB to 1e-2 meV, then CI-GNEB from rest to ftol); returns (history,
        converged, diverged)."""
        hist, done = [], 0
        for method, tol, cap in (("gneb", 1e-2, max_iters // 2), ("ci_gneb", ftol, max_iters)):
            start = done
            while done < cap:
                it, E, fm = s.path(chain, method=method, dt=dt, k_spring=1.0, tol=tol, max_iter=chunk,
                                   check_every=50, optimizer="vp", keep_velocity=done > start, stream=stream)
                done += it
                hist.append((done, time.perf_counter() - t0, max(E) - E[0], fm, E[0] - E[-1]))
                if max(E) - E[0] > E[0] - E[-1]:
                    return hist, False, True
                if fm < tol:
                    break
        return hist, hist[-1][3] < ftol, False

    def make_path(h, stream, prop):
        with torch.cuda.stream(stream):
            s = system(h)
            A = torch.from_numpy(hopf_ansatz(n, h["R"], h["c"])).cuda()
            s.minimise(A, method="vp", dt=0.1, tol=1e-4, max_iter=6000, check_every=1000, stream=stream)
            zmin = A[2].min().item()
            if zmin > -0.5:
                s.close()
                return None
            chain = torch.empty((nimg, 3, ncell), dtype=torch.float64, device="cuda")
            chain[0].copy_(A.view(3, ncell))
            chain[-1].copy_(FM.view(3, ncell))
            prop.interpolate(chain, stream=stream)
            hist, conv, _ = relax(s, chain, time.perf_counter(), stream)
            stream.synchronize()
            s.close()
            done, _, barrier, fm, scale = hist[-1]
            ok = conv and min_barrier_frac * scale <= barrier < scale
            return dict(A=A, chain=chain, barrier=barrier, scale=scale, fmax=fm, iters=done, ok=ok)

    params_in = argv[6] if len(argv) > 6 else None
    t0 = time.time()
    paths = [None] * len(hams)
    nthreads = 8
    lock = threading.Lock()
    todo = list(range(ntrain if params_in else 0, len(hams)))

    def worker():
        st = torch.cuda.Stream()
        prop = sx.Proposer(n, nimg - 2)
        while True:
            with lock:
                if not todo:
                    prop.close()
                    return
                i = todo.pop(0)
            paths[i] = make_path(hams[i], st, prop)

    th = [threading.Thread(target=worker) for _ in range(nthreads)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    torch.cuda.synchronize()
    gen_s = time.time() - t0
    train_ids = [i for i in range(ntrain) if paths[i] is not None and paths[i]["ok"]]
    train_ids = train_ids if not params_in else []
    test_ids = [i for i in range(ntrain, ntrain + ntest) if paths[i] is not None and paths[i]["ok"]]
    print(json.dumps({"stage": "paths", "lattice": list(n), "images": nimg, "method": "ci_gneb+vp",
                      "force_tol": ftol, "train_paths": len(train_ids), "test_paths": len(test_ids),
                      "collapsed": sum(paths[i] is None for i in range(ntrain if params_in else 0, len(hams))),
                      "unconverged": sum(p is not None and not p["ok"] for p in paths), "seconds": gen_s,
                      "median_iterations": float(np.median([paths[i]["iters"] for i in train_ids + test_ids])),
                      "barrier_range": [min(paths[i]["barrier"] for i in train_ids + test_ids),
                                        max(paths[i]["barrier"] for i in train_ids + test_ids)]}), flush=True)

    # ------------------------------------------------------------ training set
    batch = 2 * (nimg - 2)
    model = sx.Proposer(n, batch)
    ns, steps, losses, train_time = 0, 0, [float("nan")], 0.0
    if params_in:
        model.set_params(np.load(params_in))
    else:
        nint = nimg - 2
        ns = len(train_ids) * nint
        X = torch.empty((ns, ncell, 16), dtype=torch.int16, device="cuda")
        I = torch.empty((ns, 3, ncell), dtype=torch.float64, device="cuda")
        T = torch.empty((ns, 3, ncell), dtype=torch.float64, device="cuda")
        svals = torch.tensor([k / (nimg - 1) for k in range(1, nimg - 1)], dtype=torch.float64, device="cuda")
        for j, i in enumerate(train_ids):
            g = geodesic_chain(paths[i]["A"])
            sl = slice(j * nint, (j + 1) * nint)
            I[sl].copy_(g[1:-1])
            T[sl].copy_(paths[i]["chain"][1:-1])
            helper.pack(I[sl], paths[i]["A"], FM, svals, X[sl], shared_endpoints=True)
        model.set_params(cnn_init_flat(7))
        gen = torch.Generator(device="cpu").manual_seed(11)
        lr0, lr1 = 2e-3, 5e-5
        steps, losses = 0, []
        t0 = time.time()
        est_steps = None
        while True:
            perm = torch.randperm(ns, generator=gen).cuda()
            for b0 in range(0, ns - batch + 1, batch):
                idx = perm[b0:b0 + batch]
                Xb, Ib, Tb = X.index_select(0, idx), I.index_select(0, idx), T.index_select(0, idx)
                loss = model.loss_grad(Xb, Ib, Tb)
                el = time.time() - t0
                if est_steps is None and steps == 20:
                    est_steps = int(20 * train_s / max(el, 1e-6))
                frac = min(1.0, steps / est_steps) if est_steps else 0.0
                lr = lr1 + 0.5 * (lr0 - lr1) * (1 + np.cos(np.pi * frac))
                model.adam_step(lr)
                losses.append(loss)
                steps += 1
                if el > train_s:
                    break
            if time.time() - t0 > train_s:
                break
        torch.cuda.synchronize()
        train_time = time.time() - t0
        if len(argv) > 5:
            np.save(argv[5], model.get_params())

    def angles(P, Tt):
        d = (P * Tt).sum(1).clamp(-1, 1)
        return torch.rad2deg(torch.acos(d)).mean().item()

    # held-out error of the proposals against the converged images
    err = {"interp_deg": [], "proposal_deg": []}
    for i in test_ids:
        g = geodesic_chain(paths[i]["A"])
        c = g.clone()
        model.propose(c)
        err["interp_deg"].append(angles(g[1:-1], paths[i]["chain"][1:-1]))
        err["proposal_deg"].append(angles(c[1:-1], paths[i]["chain"][1:-1]))
    print(json.dumps({"stage": "train", "samples": ns, "batch": batch, "steps": steps, "seconds": train_time,
                      "loss_first": float(np.mean(losses[:20])), "loss_last": float(np.mean(losses[-20:])),
                      "test_mean_angle_interp_deg": float(np.mean(err["interp_deg"])),
                      "test_mean_angle_proposal_deg": float(np.mean(err["proposal_deg"]))}), flush=True)

    def seeded_chain(A, learned_chain, E_learned):
        """Piecewise geodesic chain A -> the learned run's highest interior image -> B, on the same image count."""
        k = 1 + int(np.argmax(E_learned[1:-1]))
        chain = torch.empty((nimg, 3, ncell), dtype=torch.float64, device="cuda")
        chain[0].copy_(A.view(3, ncell))
        chain[-1].copy_(FM.view(3, ncell))
        chain[k].copy_(learned_chain[k])
        if k > 1:
            helper.interpolate(chain[0:k + 1])
        if k < nimg - 2:
            helper.interpolate(chain[k:])
        return chain

    def max_jump_deg(chain):
        """Largest angle (degrees) any site turns between adjacent images: a converged chain whose images
        are this far apart does not resolve the energy between them."""
        d = (chain[1:] * chain[:-1]).sum(1).clamp(-1.0, 1.0)
        return float(torch.rad2deg(torch.acos(d)).max().item())

    # ------------------------------------------------------------ evaluation
    results = []
    for i in test_ids:
        h = hams[i]
        s = system(h)
        row = dict(path=i, B=h["B"], f=h["f"])
        chains = {}
        for arm in ("plain", "learned"):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            c = geodesic_chain(paths[i]["A"])
            if arm == "learned":
                model.propose(c)
            torch.cuda.synchronize()
            t_init = time.perf_counter() - t0
            hist, conv, div = relax(s, c, t0)
            fallback = False
            if arm == "learned" and div:
                # the geodesic interpolation as fallback, after the diverged run
                spent = hist[-1][0]
                c = geodesic_chain(paths[i]["A"])
                hist, conv, div = relax(s, c, t0)
                hist = [(h_[0] + spent,) + tuple(h_[1:]) for h_ in hist]
                fallback = True
            done, sec, barrier, fm, scale = hist[-1]
            row[arm] = dict(converged=conv, diverged=div, fallback=fallback, iterations=done, seconds=sec,
                            t_init=t_init, barrier=barrier, fmax=fm, first_barrier=hist[0][2],
                            max_jump_deg=max_jump_deg(c))
            row["scale"] = scale
            chains[arm] = c
        tol_b = 1e-3 * abs(row["scale"])
        row["same_barrier"] = abs(row["plain"]["barrier"] - row["learned"]["barrier"]) <= tol_b
        if (row["plain"]["converged"] and row["learned"]["converged"] and
                row["learned"]["barrier"] < row["plain"]["barrier"] - tol_b):
            E_l = [s.energy(chains["learned"][k])["total"] for k in range(nimg)]
            c = seeded_chain(paths[i]["A"], chains["learned"], E_l)
            t0 = time.perf_counter()
            hist, conv, div = relax(s, c, t0)
            done, sec, barrier, fm, _ = hist[-1]
            row["plain_seeded"] = dict(converged=conv, diverged=div, iterations=done, seconds=sec, barrier=barrier,
                                       fmax=fm, same_as_learned=abs(barrier - row["learned"]["barrier"]) <= tol_b,
                                       max_jump_deg=max_jump_deg(c))
        results.append(row)
        print(json.dumps({"stage": "eval", **row}), flush=True)
        s.close()
    conv = [r for r in results if r["plain"]["converged"] and r["learned"]["converged"]]
    same = [r for r in conv if r["same_barrier"]]
    sp_all = [r["plain"]["seconds"] / r["learned"]["seconds"] for r in conv]
    sp_same = [r["plain"]["seconds"] / r["learned"]["seconds"] for r in same]
    seeded = [r for r in conv if "plain_seeded" in r]
    same_direct = [r for r in same if not r["learned"]["fallback"]]
    sp_same_direct = [r["plain"]["seconds"] / r["learned"]["seconds"] for r in same_direct]
    direct = [r for r in conv if not r["learned"]["fallback"]]
    sp_direct = [r["plain"]["seconds"] / r["learned"]["seconds"] for r in direct]
    print(json.dumps({"stage": "summary", "test_paths": len(results), "both_converged": len(conv),
                      "learned_fallbacks": sum(r["learned"]["fallback"] for r in results),
                      "same_barrier": len(same),
                      "lower_barrier": {"learned": sum(r["learned"]["barrier"] < r["plain"]["barrier"] -
                                                       1e-3 * abs(r["scale"]) for r in conv),
                                        "plain": sum(r["plain"]["barrier"] < r["learned"]["barrier"] -
                                                     1e-3 * abs(r["scale"]) for r in conv)},
                      "learned_faster": sum(r["learned"]["seconds"] < r["plain"]["seconds"] for r in conv),
                      "lower_channel_confirmed_by_seeded_plain": sum(r["plain_seeded"]["converged"] and
                                                                    r["plain_seeded"]["same_as_learned"]
                                                                    for r in seeded),
                      "lower_channel_checked": len(seeded),
                      "median_speedup_all": float(np.median(sp_all)) if sp_all else None,
                      "median_speedup_same_barrier": float(np.median(sp_same)) if sp_same else None,
                      "same_barrier_without_fallback": len(same_direct),
                      "median_speedup_same_barrier_without_fallback":
                          float(np.median(sp_same_direct)) if sp_same_direct else None,
                      "median_max_jump_deg": {arm: float(np.median([r[arm]["max_jump_deg"] for r in conv]))
                                              for arm in ("plain", "learned")} if conv else None,
                      "lower_learned_with_jump_over_90deg": sum(r["learned"]["max_jump_deg"] > 90.0 for r in seeded),
                      "median_speedup_without_fallback": float(np.median(sp_direct)) if sp_direct else None,
                      "median_plain_s": float(np.median([r["plain"]["seconds"] for r in conv])) if conv else None,
                      "median_learned_s": float(np.median([r["learned"]["seconds"] for r in conv])) if conv else None,
                      "generation_s": gen_s, "training_s": train_time}), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
