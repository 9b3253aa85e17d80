"""Batched replicas (sx_batch): one launch pair advances several independent lattices of one Hamiltonian,
bit-identical to stepping each context on its own."""
import numpy as np
import pytest

import paper_2605_26016_gb300 as sx
from workloads import random_spins

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_26016_gb300.build import build
    build()


def systems(name, shapes, **override):
    out = []
    for n, pbc in shapes:
        s, w = sx.system_from_workload(name, n, pbc=pbc, **override)
        s.plan("stencil", "fp32")
        out.append((s, w))
    return out


@pytest.mark.parametrize("thermal", [False, True])
@pytest.mark.parametrize("name,shapes", [
    ("bcc_4shell", [((24, 24, 24), (1, 1, 1)), ((17, 13, 11), (1, 1, 0)), ((40, 30, 20), (0, 1, 1)), ((9, 9, 9), (1, 1, 1))]),
    ("sc_j123_dmi", [((33, 20, 7), (1, 1, 1)), ((64, 48, 40), (1, 1, 0)), ((5, 5, 5), (0, 0, 0))]),
])
def test_batch_step_equals_single_steps(name, shapes, thermal):
    sw = systems(name, shapes)
    w = sw[0][1]
    batch = sx.Batch([s for s, _ in sw])
    T = 120.0 if thermal else 0.0
    p = sx.llg_params(w["dt"], w["alpha"], T, seed=6, replica=3)
    S_in = [torch.from_numpy(random_spins(s.nsub, s.n, 50 + r)).cuda() for r, (s, _) in enumerate(sw)]
    S_out = [torch.empty_like(x) for x in S_in]
    for step in (0, 7):
        batch.heun_step(S_in, S_out, p, step)
        torch.cuda.synchronize()
        for r, (s, _) in enumerate(sw):
            pr = sx.llg_params(w["dt"], w["alpha"], T, seed=6, replica=3 + r)
            ref = torch.empty_like(S_in[r])
            sx.sx_llg_heun_step_out(s.ctx, S_in[r], ref, pr, step, s.nsite)
            torch.cuda.synchronize()
            assert torch.equal(S_out[r], ref), (r, step)
        S_in, S_out = S_out, S_in


def test_batch_rejects_mixed_hamiltonians_and_replanned_contexts():
    a, _ = sx.system_from_workload("bcc_4shell", (12, 12, 12))
    b, _ = sx.system_from_workload("bcc_4shell", (14, 12, 10), shells=[20.0, 10.0, -1.0, 0.6])
    a.plan("stencil", "fp32")
    b.plan("stencil", "fp32")
    with pytest.raises(sx.SxError) as e:
        sx.Batch([a, b])
    assert e.value.code == sx.SX_ERR_ARG
    with pytest.raises(sx.SxError):
        sx.Batch([a, a])
    c, w = sx.system_from_workload("bcc_4shell", (10, 10, 10))
    c.plan("stencil", "fp32")
    batch = sx.Batch([a, c])
    c.plan("stencil", "fp32")
    S = [torch.from_numpy(random_spins(2, x.n, 1)).cuda() for x in (a, c)]
    with pytest.raises(sx.SxError) as e:
        batch.heun_step(S, [torch.empty_like(x) for x in S], sx.llg_params(0.1, 0.1), 0)
    assert e.value.code == sx.SX_ERR_STATE


def reference_steps(sw, S0, w, T, replica0, step0, nsteps, seed=6):
    """Each replica stepped on its own context, nsteps times."""
    out = []
    for r, (s, _) in enumerate(sw):
        cur, nxt = S0[r].clone(), torch.empty_like(S0[r])
        for k in range(nsteps):
            pr = sx.llg_params(w["dt"], w["alpha"], T, seed=seed, replica=replica0 + r)
            sx.sx_llg_heun_step_out(s.ctx, cur, nxt, pr, step0 + k, s.nsite)
            cur, nxt = nxt, cur
        out.append(cur)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("nsteps", [1, 3])
@pytest.mark.parametrize("name,shapes,img_shape", [
    ("bcc_4shell", [((24, 24, 24), (1, 1, 1)), ((17, 13, 11), (1, 1, 0)), ((9, 9, 9), (1, 1, 1))], ((20, 16, 12), (1, 1, 1))),
    ("sc_j123_dmi", [((33, 20, 7), (1, 1, 1)), ((64, 48, 40), (1, 1, 0))], ((32, 32, 16), (1, 1, 0))),
])
def test_batch_run_replicas_and_images_in_one_launch(name, shapes, img_shape, nsteps):
    # sx_batch_run: uneven replicas stepped nsteps times and a chain's images evaluated in one persistent
    # launch, bit-identical to separate per-context calls
    sw = systems(name, shapes)
    w = sw[0][1]
    img_s, _ = sx.system_from_workload(name, img_shape[0], pbc=img_shape[1])
    img_s.plan("stencil", "fp32")
    nimg = 4
    batch = sx.Batch([s for s, _ in sw], image_system=img_s, nimg=nimg)
    info = batch.info()
    assert info["replicas"] == len(sw) and info["images"] == nimg
    T = 80.0
    S0 = [torch.from_numpy(random_spins(s.nsub, s.n, 70 + r)).cuda() for r, (s, _) in enumerate(sw)]
    S_a = [x.clone() for x in S0]
    S_b = [torch.empty_like(x) for x in S0]
    images = torch.from_numpy(np.stack([random_spins(img_s.nsub, img_s.n, 90 + k) for k in range(nimg)])).cuda()
    fields = torch.full_like(images, float("nan"))
    batch.bind(S_a, S_b, images, fields, replica0=2)
    p = sx.llg_params(w["dt"], w["alpha"], T, seed=6)
    batch.run(p, 5, nsteps)
    batch.status()
    got = S_b if nsteps % 2 else S_a
    ref = reference_steps(sw, S0, w, T, 2, 5, nsteps)
    for r in range(len(sw)):
        assert torch.equal(got[r], ref[r]), r
    for k in range(nimg):
        assert torch.equal(fields[k], img_s.field(images[k])), k


def test_batch_run_is_graph_capturable():
    sw = systems("sc_j123_dmi", [((33, 20, 7), (1, 1, 1)), ((24, 24, 24), (1, 1, 0))])
    w = sw[0][1]
    img_s, _ = sx.system_from_workload("sc_j123_dmi", (16, 16, 16))
    img_s.plan("stencil", "fp32")
    batch = sx.Batch([s for s, _ in sw], image_system=img_s, nimg=2)
    S0 = [torch.from_numpy(random_spins(1, s.n, 5 + r)).cuda() for r, (s, _) in enumerate(sw)]
    S_a = [x.clone() for x in S0]
    S_b = [torch.empty_like(x) for x in S0]
    images = torch.from_numpy(np.stack([random_spins(1, img_s.n, 30 + k) for k in range(2)])).cuda()
    fields = torch.zeros_like(images)
    batch.bind(S_a, S_b, images, fields)
    p = sx.llg_params(w["dt"], w["alpha"], 40.0, seed=1)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            batch.run(p, 11, 2)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    for r in range(len(sw)):       # capture did not execute
        assert torch.equal(S_a[r], S0[r])
    g.replay()
    torch.cuda.synchronize()
    batch.status()
    ref = reference_steps(sw, S0, w, 40.0, 0, 11, 2, seed=1)
    for r in range(len(sw)):
        assert torch.equal(S_a[r], ref[r]), r
    for k in range(2):
        assert torch.equal(fields[k], img_s.field(images[k])), k
