"""GPU parity of the tensor-core (tcgen05 implicit GEMM) field backend against the CPU oracle.

The backend contracts the sublattice spin channels (C = 3 nsub) with the channel matrix of every
kernel plane, so sublattices, 3x3 tensor taps (DMI) and dense 7x7x7 windows all run through it.

Tolerances (normwise field): TF32 inputs are rounded to 10-bit mantissas (2^-11 relative per
input), BF16 uses the split hi+lo representation with three MMAs (about 2^-16 per input).  The
bound for both is 2e-3 (the BF16 class for fields); the split BF16 path is also held to 1e-4.
"""
import numpy as np
import pytest

import oracle
import paper_2605_26016_gb300 as sx
from oracle.models import oracle_model
from workloads import cubic_cell, dense_window_bonds, random_spins

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


def pair_systems(n, pbc, pos, mu, bonds, B=None):
    """The same bond list in the library and in the oracle."""
    s = sx.SpinSystem(n, pbc, cubic_cell(), pos, mu)
    s.add_bonds(bonds)
    m = oracle.Model(n, pbc, cubic_cell(), pos, mu)
    for a, b, d, J in bonds:
        m.add_bond(a, b, d, J)
    if B is not None:
        s.set_zeeman(B)
        m.set_zeeman(B)
    m.build()
    return s, m


def random_bonds(rng, nsub, radius, count, tensor=True):
    """count unordered bonds between random sublattices at random cell offsets within |d| <= radius,
    with random 3x3 couplings (isotropic + antisymmetric + symmetric anisotropic parts)."""
    bonds, seen = [], set()
    while len(bonds) < count:
        a, b = (int(v) for v in rng.integers(0, nsub, 2))
        d = tuple(int(v) for v in rng.integers(-radius, radius + 1, 3))
        if a == b and d == (0, 0, 0):
            continue
        key = (a, b, d)
        if key in seen or (b, a, tuple(-v for v in d)) in seen:
            continue
        seen.add(key)
        J = np.eye(3) * rng.normal()
        if tensor:
            J = J + 0.3 * rng.normal(size=(3, 3))
        bonds.append((a, b, d, J))
    return bonds


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("n,pbc", [((33, 17, 11), (1, 1, 0)), ((130, 20, 24), (1, 1, 1)), ((9, 8, 8), (0, 0, 0))])
def test_tc_field_and_energy(prec, n, pbc):
    s, w = sx.system_from_workload("sc_j123", n, pbc=pbc, B=[0.2, 0.0, 1.5])
    info = s.plan("igemm_tc", prec)
    assert info["launches_per_step"] == 6
    m, _ = oracle_model("sc_j123", n, pbc=pbc, B=[0.2, 0.0, 1.5])
    S = random_spins(1, n, 11)
    Sd = dev(S)
    ref = m.field(S)
    assert normwise(s.field(Sd).cpu().numpy(), ref) <= TOL[prec]
    assert normwise(s.field(Sd, dtype=torch.float32).double().cpu().numpy(), ref) <= TOL[prec]
    e = s.energy(Sd)
    e_ref = m.energy(S)
    assert abs(e["total"] - e_ref) <= TOL[prec] * 0.5 * np.sqrt((ref.reshape(3, -1) ** 2).sum(0)).sum()


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("name,n,pbc", [
    ("bcc_4shell", (24, 20, 18), (1, 1, 1)),     # two sublattices, four shells, anisotropy
    ("bcc_4shell", (13, 9, 21), (1, 0, 1)),      # ragged tiles, one open face
    ("sc_j123_dmi", (33, 17, 19), (1, 1, 1)),    # interfacial DMI: antisymmetric tensor taps
    ("sc_j123_dmi", (22, 8, 16), (0, 1, 0)),
    ("sc_4shell", (25, 11, 7), (0, 0, 0)),       # fourth shell (2,0,0): rx = 2
])
def test_tc_multichannel_workloads(prec, name, n, pbc):
    s, w = sx.system_from_workload(name, n, pbc=pbc, B=[0.3, -0.2, 1.1])
    s.plan("igemm_tc", prec)
    m, _ = oracle_model(name, n, pbc=pbc, B=[0.3, -0.2, 1.1])
    S = random_spins(s.nsub, n, 17)
    ref = m.field(S)
    Sd = dev(S)
    assert normwise(s.field(Sd).cpu().numpy(), ref) <= TOL[prec]
    assert normwise(s.field(Sd, dtype=torch.float32).double().cpu().numpy(), ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_tc_dense_7x7x7_tensor_window(prec):
    # a 3x3 tensor coupling on every cell offset of the 7x7x7 window (342 directed taps per site)
    rng = np.random.default_rng(1)
    bonds = []
    for d in np.ndindex(7, 7, 7):
        d = tuple(int(v) - 3 for v in d)
        if d > (0, 0, 0):
            J = np.eye(3) * rng.normal() / (1.0 + sum(v * v for v in d)) + 0.05 * rng.normal(size=(3, 3))
            bonds.append((0, 0, d, J))
    n = (47, 19, 18)
    s, m = pair_systems(n, (1, 0, 1), [[0, 0, 0]], [1.0], bonds, B=[0.0, 0.5, 1.0])
    assert s.plan("igemm_tc", prec)["rx"] == 3
    S = random_spins(1, n, 6)
    assert normwise(s.field(dev(S)).cpu().numpy(), m.field(S)) <= TOL[prec]


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("nsub,radius,n,pbc", [
    (2, 3, (23, 12, 17), (1, 1, 0)),
    (3, 2, (15, 9, 20), (0, 1, 1)),
    (4, 1, (11, 10, 9), (1, 1, 1)),
    (4, 2, (7, 5, 3), (1, 0, 1)),
])
def test_tc_random_sublattice_couplings(prec, nsub, radius, n, pbc):
    rng = np.random.default_rng(100 + nsub)
    pos = [[0.0, 0.0, 0.0], [0.5, 0.5, 0.5], [0.5, 0.0, 0.0], [0.0, 0.5, 0.0]][:nsub]
    bonds = random_bonds(rng, nsub, radius, 40)
    s, m = pair_systems(n, pbc, pos, [1.0 + 0.1 * k for k in range(nsub)], bonds, B=[0.1, 0.2, 0.3])
    s.plan("igemm_tc", prec)
    S = random_spins(nsub, n, 5)
    assert normwise(s.field(dev(S)).cpu().numpy(), m.field(S)) <= TOL[prec]


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("name,n,pbc", [("sc_j123", (36, 16, 12), (1, 1, 0)), ("bcc_4shell", (20, 10, 17), (1, 1, 1)),
                                        ("sc_j123_dmi", (24, 9, 16), (1, 1, 1))])
def test_tc_heun_step(prec, name, n, pbc):
    s, w = sx.system_from_workload(name, n, pbc=pbc, B=[0.0, 0.0, 2.0])
    s.plan("igemm_tc", prec)
    m, _ = oracle_model(name, n, pbc=pbc, B=[0.0, 0.0, 2.0])
    S = random_spins(s.nsub, n, 21)
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


def test_tc_full_size_dense_window_sampled():
    # 100^3 with a tensor coupling on every offset of the 7x7x7 window, TF32, at sampled sites
    bonds = dense_window_bonds(9)
    n = (100, 100, 100)
    s = sx.SpinSystem(n, (1, 1, 1), cubic_cell(), [[0, 0, 0]], [1.0])
    s.add_bonds(bonds)
    s.plan("igemm_tc", "tf32")
    S = random_spins(1, n, 4)
    b = s.field(dev(S)).cpu().numpy().reshape(3, -1)
    m = oracle.Model(n, (1, 1, 1), cubic_cell(), [[0, 0, 0]], [1.0])
    for a, bb, d, J in bonds:
        m.add_bond(a, bb, d, J)
    sites = np.concatenate([np.random.default_rng(3).choice(s.nsite, 600, replace=False), [0, s.nsite - 1]])
    assert normwise(b[:, sites], m.field_sites(S, sites).T) <= TOL["tf32"]


def test_tc_rejects_unsupported_hamiltonians():
    s, _ = sx.system_from_workload("sc_j123", (8, 8, 8))
    with pytest.raises(sx.SxError) as e:
        s.plan("igemm_tc", "fp32")
    assert e.value.code == sx.SX_ERR_UNSUPPORTED
    far = sx.SpinSystem((12, 8, 8), (1, 1, 1), cubic_cell(), [[0, 0, 0]], [1.0])
    far.add_bonds([(0, 0, (4, 0, 0), np.eye(3))])                    # beyond the 7x7x7 window
    with pytest.raises(sx.SxError) as e:
        far.plan("igemm_tc", "tf32")
    assert e.value.code == sx.SX_ERR_UNSUPPORTED
    pos5 = [[0.1 * k, 0.0, 0.0] for k in range(5)]
    five = sx.SpinSystem((4, 4, 4), (1, 1, 1), cubic_cell(), pos5, [1.0] * 5)  # five sublattices
    five.add_bonds([(0, 1, (0, 0, 0), np.eye(3))])
    with pytest.raises(sx.SxError) as e:
        five.plan("igemm_tc", "bf16")
    assert e.value.code == sx.SX_ERR_UNSUPPORTED


def test_tc_autotune_layouts_keep_the_field():
    # ring depth and CTAs per SM change the schedule of tiles, not the arithmetic of one
    n = (40, 24, 32)
    s, w = sx.system_from_workload("sc_j123_dmi", n)
    s.plan("igemm_tc", "tf32")
    Sd = dev(random_spins(1, n, 8))
    b0 = s.field(Sd)
    p = sx.llg_params(w["dt"], w["alpha"], w["T"], seed=1)
    name, t = sx.sx_autotune(s.ctx, Sd, torch.empty_like(Sd), p, s.nsite, steps=2)
    assert name == "fused" and t["fused"] > 0
    tiles = sx.sx_plan_tiles(s.ctx)
    assert 2 <= tiles["ring_or_schedule"] <= 4 and tiles["ctas"] > 0 and tiles["tile_z"] == 16
    assert torch.equal(s.field(Sd), b0)


def test_tc_every_layout_gives_the_same_field():
    n = (44, 24, 33)
    s, w = sx.system_from_workload("bcc_4shell", n)
    s.plan("igemm_tc", "bf16")
    Sd = dev(random_spins(2, n, 4))
    b0 = s.field(Sd)
    tried = 0
    for ring in (2, 3, 4):
        for ctas in (1, 2):
            try:
                sx.sx_set_tiles(s.ctx, 0, ring, ctas)
            except sx.SxError as e:
                assert e.code == sx.SX_ERR_ARG  # the layout does not fit
                continue
            tried += 1
            assert sx.sx_plan_tiles(s.ctx)["ring_or_schedule"] == ring
            assert torch.equal(s.field(Sd), b0), (ring, ctas)
    assert tried >= 2
