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
