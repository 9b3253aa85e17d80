"""Time the chain proposer's kernels: inference (sx_cnn_forward) and one training step (sx_cnn_loss_grad +
sx_cnn_adam_step) on a batch of samples; used for ncu captures as well.

    python -m paper_2605_26016_gb300.profile_cnn [nx,ny,nz] [batch] [repeats] [mode]

Defaults: 64,64,64, 30 samples (the interior images of a 32-image chain on 64^3), 20 repeats, mode "both"
("forward" or "train" run only that part).  Inputs are seeded random unit fields.  Prints one JSON line:
milliseconds per forward pass and per training step (CUDA events on the launching stream, after 3 warm-up
calls; every call reads inputs far larger than L2), sites per second, and the algorithmic traffic and flops of
the forward convolutions: 64 B per site per layer (a 32-byte BF16 site read, a 32-byte site written) and
2 x 27 x c_in x c_out useful flops per site per layer.
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
    res = {"workload": f"proposer {n[0]}x{n[1]}x{n[2]}, {nb} samples", "sites": nb * ncell}

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


if __name__ == "__main__":
    main(sys.argv[1:])
