"""GPU parity of the FFT (reciprocal-space kernel) backend against the CPU oracle.

The oracle evaluates the dipolar term by direct summation over every pair
(periodic minimum image, half-period images split evenly) and the exchange/DMI
terms from its pair list; the FFT backend multiplies spectra.  Tolerances:
FP64 transforms 1e-12 normwise on the field, 1e-11 on a Heun increment; FP32
transforms 2e-6 on the field (FP32 round-off of log2(N) butterfly stages of a
field whose spectrum is dominated by the exchange kernel), 2e-5 on a Heun
increment.
"""
import numpy as np
import pytest

import paper_2605_26016_gb300 as sx
from oracle.models import oracle_model
from workloads import random_spins, uniform_spins

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_FIELD = {"fp64": 1e-12, "fp32": 2e-6}
TOL_STEP = {"fp64": 1e-11, "fp32": 2e-5}


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
    return np.sqrt(((got - ref) ** 2).sum(0)).max() / max(np.sqrt((ref ** 2).sum(0)).max(), 1e-300)


def pair(name, n, dipolar, **override):
    s, w = sx.system_from_workload(name, n, pbc=(1, 1, 1), **override)
    s.set_dipolar(dipolar)
    m, _ = oracle_model(name, n, pbc=(1, 1, 1), dipolar=dipolar, **override)
    return s, m, w


# the last case has z lines of 1024 points: its z pass holds four lines of three channels (111 KB) and runs
# with 512 threads per CTA
CASES = [("sc_j123_dmi", (16, 8, 4), False), ("sc_j123_dmi", (8, 8, 8), True), ("bcc_4shell", (8, 4, 8), False),
         ("bcc_4shell", (4, 8, 4), True), ("sc_nn", (32, 1, 2), True), ("sc_j123_dmi", (8, 4, 1024), False)]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_fft_field_and_energy(prec, case):
    name, n, dip = CASES[case]
    s, m, w = pair(name, n, dip)
    s.plan("fft", prec)
    S = random_spins(s.nsub, n, 300 + case)
    Sd = dev(S)
    b = s.field(Sd).cpu().numpy()
    ref = m.field(S)
    assert normwise(b, ref) <= TOL_FIELD[prec]
    e = s.energy(Sd)
    e_ref, t = m.energy(S, terms=True)
    bound = 0.5 * np.sqrt((ref.reshape(3, -1) ** 2).sum(0)).sum()
    assert abs(e["total"] - e_ref) <= TOL_FIELD[prec] * bound
    assert abs(e["bilinear"] + e["dipolar"] - (t[0] + t[3])) <= TOL_FIELD[prec] * bound


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", [0, 1, 3, 5])
def test_fft_heun(prec, case):
    name, n, dip = CASES[case]
    s, m, w = pair(name, n, dip)
    s.plan("fft", prec)
    S = random_spins(s.nsub, n, 400 + case)
    T = w["T"] or 40.0
    Sd = dev(S)
    s.heun(Sd, torch.empty_like(Sd), dt=w["dt"], alpha=w["alpha"], T=T, seed=6, replica=1, step0=3, nsteps=2)
    got = Sd.cpu().numpy()
    ref = m.heun(S, w["dt"], w["alpha"], T=T, seed=6, replica=1, step0=3, nsteps=2)
    assert normwise(got - S, ref - S) <= 2 * TOL_STEP[prec]
    assert np.abs(np.sqrt((got.reshape(3, -1) ** 2).sum(0)) - 1).max() < 1e-13


def test_fft_uniform_state_has_no_dipolar_field_at_256():
    # property that holds at any size: a uniform state in a periodic cube feels no dipolar field
    n = (256, 256, 256)
    s = sx.SpinSystem(n, (1, 1, 1), [[0.287, 0, 0], [0, 0.287, 0], [0, 0, 0.287]], [[0, 0, 0]], [2.2])
    s.set_dipolar(True)
    s.plan("fft", "fp32")
    S = dev(uniform_spins(1, n, [0.3, -0.5, 0.8]))
    b = s.field(S)
    scale = 5.368e-5 * 2.2 ** 2 / 0.287 ** 3
    assert b.abs().max().item() < 1e-5 * scale


def test_fft_sampled_sites_with_dipolar_at_64():
    n = (64, 64, 64)
    s, w = sx.system_from_workload("sc_j123_dmi", n)
    s.set_dipolar(True)
    s.plan("fft", "fp32")
    S = random_spins(1, n, 77)
    b = s.field(dev(S)).cpu().numpy().reshape(3, -1)
    m, _ = oracle_model("sc_j123_dmi", n, dipolar=True, build=False)
    sites = np.random.default_rng(3).choice(s.nsite, 64, replace=False)
    ref = m.field_sites(S, sites)
    assert normwise(b[:, sites], ref.T) <= TOL_FIELD["fp32"]


def test_fft_rejects_unsupported_geometry():
    s, _ = sx.system_from_workload("sc_j123", (16, 16, 16), pbc=(1, 1, 0))
    with pytest.raises(sx.SxError) as e:
        s.plan("fft", "fp32")
    assert e.value.code == sx.SX_ERR_UNSUPPORTED
    s2, _ = sx.system_from_workload("sc_j123", (12, 16, 16), pbc=(1, 1, 1))
    with pytest.raises(sx.SxError) as e:
        s2.plan("fft", "fp32")
    assert e.value.code == sx.SX_ERR_UNSUPPORTED
    with pytest.raises(sx.SxError) as e:
        s2.plan("fft", "bf16")
    assert e.value.code == sx.SX_ERR_UNSUPPORTED
