"""GPU parity of the tensor-core (tcgen05 implicit GEMM) field backend against the CPU oracle.

Tolerances (normwise field): TF32 inputs are rounded to 10-bit mantissas (2^-11 relative per
input), BF16 uses the split hi+lo representation with three MMAs (about 2^-16 per input).  The
bound for both is 2e-3 (the BF16 class for fields); the split BF16 path is also held to 1e-4.
"""
import numpy as np
import pytest

import oracle
import paper_2605_26016_gb300 as sx
from oracle.models import oracle_model
from workloads import cubic_cell, random_spins

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {"tf32": 2e-3, "bf16": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_26016_gb300.build import build
    build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def normwise(got, ref):
    got = np.asarray(got).reshape(3, -1)
    ref = np.asarray(ref).reshape(3, -1)
    return np.sqrt(((got - ref) ** 2).sum(0)).max() / np.sqrt((ref ** 2).sum(0)).max()


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("n,pbc", [((33, 17, 11), (1, 1, 0)), ((130, 20, 24), (1, 1, 1)), ((9, 8, 8), (0, 0, 0))])
def test_tc_field_and_energy(prec, n, pbc):
    s, w = sx.system_from_workload("sc_j123", n, pbc=pbc, B=[0.2, 0.0, 1.5])
    info = s.plan("igemm_tc", prec)
    assert info["launches_per_step"] == 4
    m, _ = oracle_model("sc_j123", n, pbc=pbc, B=[0.2, 0.0, 1.5])
    S = random_spins(1, n, 11)
    Sd = dev(S)
    ref = m.field(S)
    assert normwise(s.field(Sd).cpu().numpy(), ref) <= TOL[prec]
    e = s.energy(Sd)
    e_ref = m.energy(S)
    assert abs(e["total"] - e_ref) <= TOL[prec] * 0.5 * np.sqrt((ref.reshape(3, -1) ** 2).sum(0)).sum()


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_tc_dense_7x7x7_window(prec):
    # isotropic couplings scattered over the full 7x7x7 window (R = 3)
    rng = np.random.default_rng(1)
    bonds = []
    for _ in range(30):
        d = tuple(int(v) for v in rng.integers(-3, 4, 3))
        if d != (0, 0, 0):
            bonds.append((0, 0, d, np.eye(3) * rng.normal()))
    n = (40, 16, 16)
    s = sx.SpinSystem(n, (1, 0, 1), cubic_cell(), [[0, 0, 0]], [1.0])
    s.add_bonds(bonds)
    assert s.plan("igemm_tc", prec)["rx"] == 3
    m = oracle.Model(n, (1, 0, 1), cubic_cell(), [[0, 0, 0]], [1.0])
    for a, b, d, J in bonds:
        m.add_bond(a, b, d, J)
    m.build()
    S = random_spins(1, n, 6)
    assert normwise(s.field(dev(S)).cpu().numpy(), m.field(S)) <= TOL[prec]


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_tc_heun_step(prec):
    n = (36, 16, 12)
    s, w = sx.system_from_workload("sc_j123", n, pbc=(1, 1, 0), B=[0.0, 0.0, 2.0])
    s.plan("igemm_tc", prec)
    m, _ = oracle_model("sc_j123", n, pbc=(1, 1, 0), B=[0.0, 0.0, 2.0])
    S = random_spins(1, n, 21)
    Sd = dev(S)
    s.heun(Sd, torch.empty_like(Sd), dt=0.5, alpha=0.1, T=20.0, seed=3, step0=7, nsteps=2)
    got = Sd.cpu().numpy()
    ref = m.heun(S, 0.5, 0.1, T=20.0, seed=3, step0=7, nsteps=2)
    assert normwise(got - S, ref - S) <= 2 * TOL[prec] + 1e-5
    assert np.abs(np.sqrt((got.reshape(3, -1) ** 2).sum(0)) - 1).max() < 1e-13


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_tc_full_size_hopfion_lattice_sampled(prec):
    # 100^3 simple cubic, three distance shells, open in z (the dense-path workload)
    n = (100, 100, 100)
    s, w = sx.system_from_workload("sc_j123", n)
    s.plan("igemm_tc", prec)
    S = random_spins(1, n, w["seed"])
    b = s.field(dev(S)).cpu().numpy().reshape(3, -1)
    m, _ = oracle_model("sc_j123", n, build=False)
    sites = np.concatenate([np.random.default_rng(2).choice(s.nsite, 2000, replace=False), [0, s.nsite - 1]])
    assert normwise(b[:, sites], m.field_sites(S, sites).T) <= TOL[prec]


def test_tc_rejects_unsupported_hamiltonians():
    s, _ = sx.system_from_workload("sc_j123_dmi", (16, 16, 16))       # DMI: tensor taps
    with pytest.raises(sx.SxError) as e:
        s.plan("igemm_tc", "bf16")
    assert e.value.code == sx.SX_ERR_UNSUPPORTED
    s2, _ = sx.system_from_workload("bcc_4shell", (8, 8, 8))            # two sublattices
    with pytest.raises(sx.SxError) as e:
        s2.plan("igemm_tc", "tf32")
    assert e.value.code == sx.SX_ERR_UNSUPPORTED
    s3, _ = sx.system_from_workload("sc_j123", (8, 8, 8))
    with pytest.raises(sx.SxError) as e:
        s3.plan("igemm_tc", "fp32")
    assert e.value.code == sx.SX_ERR_UNSUPPORTED
