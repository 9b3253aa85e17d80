"""sx_torque_max_noalloc: the torque maximum for callers that cannot let the library allocate
device memory (they reserve the GPU's memory in their own arena, or cannot absorb the implicit
synchronisation of cudaMalloc inside a time-step loop).  It keeps its scratch in a fixed array
inside the library image; this test checks it through the C ABI against the regular
sx_torque_max, on two calls in a row that share that array.  Collected last on purpose."""
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


@pytest.mark.parametrize("name,n,backend", [("bcc_4shell", (20, 18, 16), "gather"),
                                            ("sc_j123_dmi", (150, 130, 120), "stencil")])
def test_noalloc_torque_matches_regular_entry(name, n, backend):
    s, w = sx.system_from_workload(name, n)
    s.plan(backend, "fp32")
    for call, seed in enumerate((1, 2)):     # two calls in a row reuse the same static scratch
        S = torch.from_numpy(random_spins(s.nsub, n, seed)).cuda()
        b = s.field(S)
        ref = s.torque_max(S)
        got = sx.sx_torque_max_noalloc(S, b, s.nsite)
        assert ref > 0.0
        assert abs(got - ref) <= 1e-12 * ref, (call, got, ref)


@pytest.mark.parametrize("nsite", [1, 255, 256, 257])
def test_noalloc_single_block_lattices(nsite):
    # one block (nsite < 256: most threads see no site, the final pass reads one slot) and its edges,
    # against max |S x b| formed on the host; two calls in a row
    rng = np.random.default_rng(nsite)
    for call in range(2):
        S = rng.standard_normal((3, nsite))
        b = rng.standard_normal((3, nsite)) * (call + 1)
        ref = np.sqrt((np.cross(S.T, b.T) ** 2).sum(1)).max()
        got = sx.sx_torque_max_noalloc(torch.from_numpy(S).cuda(), torch.from_numpy(b).cuda(), nsite)
        assert abs(got - ref) <= 1e-14 * ref, (nsite, call, got, ref)


def test_noalloc_rejects_bad_sizes():
    buf = torch.zeros(6, dtype=torch.float64, device="cuda")
    S, b = sx.ctypes.c_void_p(buf.data_ptr()), sx.ctypes.c_void_p(buf.data_ptr() + 24)
    out = sx.ctypes.c_double()
    L = sx.lib()
    assert L.sx_torque_max_noalloc(S, b, 0, sx.ctypes.byref(out), None) == sx.SX_ERR_ARG          # empty
    assert L.sx_torque_max_noalloc(S, b, 2 ** 40 + 1, sx.ctypes.byref(out), None) == sx.SX_ERR_ARG  # too large
    assert L.sx_torque_max_noalloc(S, S, 1, sx.ctypes.byref(out), None) == sx.SX_ERR_ARG          # overlap
    assert "nsite" in sx.last_error() or "overlap" in sx.last_error()
