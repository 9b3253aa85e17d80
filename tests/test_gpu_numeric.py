"""Numeric-error reporting (SX_ERR_NUMERIC) through the C ABI.

A host-made spin field with one non-finite or zero-length site is an ordinary
input, not a device fault: the state update flags it in the context's status
word, the torque and energy reductions propagate NaN instead of skipping it,
and no call reports convergence on such a state."""
import math

import numpy as np
import pytest

import paper_2605_26016_gb300 as sx
from workloads import nlerp_chain, random_spins, uniform_spins

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_26016_gb300.build import build
    build()


N = (12, 10, 9)


def _bad_spins(nsub, kind, site=37):
    S = random_spins(nsub, N, 5).reshape(3, -1)
    if kind == "nan":
        S[1, site] = math.nan
    elif kind == "inf":
        S[0, site] = math.inf
    else:
        S[:, site] = 0.0
    return torch.from_numpy(S.reshape(3, nsub, N[2], N[1], N[0]).copy()).cuda()


def _expect_numeric(fn, *a, **kw):
    with pytest.raises(sx.SxError) as e:
        fn(*a, **kw)
    assert e.value.code == sx.SX_ERR_NUMERIC, str(e.value)


CASES = [("sc_j123_dmi", "stencil", "fp32", "two_pass"), ("sc_j123_dmi", "stencil", "fp32", "fused"),
         ("bcc_4shell", "stencil", "fp32", "two_pass"), ("bcc_4shell", "gather", "fp32", None),
         ("bcc_4shell", "gather", "fp64", None)]


@pytest.mark.parametrize("name,backend,prec,scheme", CASES)
@pytest.mark.parametrize("kind", ["nan", "inf", "zero"])
def test_heun_step_flags_bad_site(name, backend, prec, scheme, kind):
    s, w = sx.system_from_workload(name, N)
    if scheme:
        sx.sx_set_stencil_scheme(s.ctx, scheme)
    s.plan(backend, prec)
    S = _bad_spins(s.nsub, kind)
    s.heun(S, torch.empty_like(S), dt=w["dt"], alpha=w["alpha"], T=w["T"], seed=3, nsteps=2)  # asynchronous: no error
    _expect_numeric(sx.sx_device_status, s.ctx)
    sx.sx_device_status(s.ctx)  # reading the status clears it
    good = torch.from_numpy(random_spins(s.nsub, N, 6)).cuda()
    s.heun(good, torch.empty_like(good), dt=w["dt"], alpha=w["alpha"], T=w["T"], seed=3, nsteps=2)
    sx.sx_device_status(s.ctx)
    n = good.view(3, -1).pow(2).sum(0).sqrt()
    assert (n - 1).abs().max().item() < 1e-13


def test_host_entry_reports_bad_site():
    s, w = sx.system_from_workload("sc_j123_dmi", N)
    s.plan("stencil", "fp32")
    Sh = _bad_spins(1, "nan").cpu()
    _expect_numeric(s.heun_host, Sh, dt=w["dt"], alpha=w["alpha"], T=w["T"], seed=3, nsteps=1)


@pytest.mark.parametrize("backend,prec", [("stencil", "fp32"), ("gather", "fp64")])
def test_torque_and_energy_propagate_nan(backend, prec):
    s, w = sx.system_from_workload("sc_j123_dmi", N)
    s.plan(backend, prec)
    S = _bad_spins(1, "nan")
    _expect_numeric(s.torque_max, S)
    _expect_numeric(s.energy, S)
    good = torch.from_numpy(random_spins(1, N, 7)).cuda()
    b = s.field(good)
    b.view(3, -1)[2, 101] = math.nan
    _expect_numeric(sx.sx_torque_max_noalloc, good, b, s.nsite)
    assert s.torque_max(good) > 0.0


@pytest.mark.parametrize("method", ["vp", "damped_llg"])
def test_minimise_does_not_converge_on_nan(method):
    s, w = sx.system_from_workload("sc_j123_dmi", N)
    s.plan("stencil", "fp32")
    S = _bad_spins(1, "nan")
    # a huge tolerance would be met at once if the NaN site read as zero torque
    _expect_numeric(s.minimise, S, method=method, dt=0.05, tol=1e30, max_iter=20, check_every=5)


@pytest.mark.parametrize("method,optimizer", [("gneb", "steepest"), ("ci_gneb", "vp"), ("string", "steepest")])
def test_path_step_does_not_converge_on_nan(method, optimizer):
    n = (10, 9, 8)
    s, w = sx.system_from_workload("sc_4shell", n)
    s.plan("stencil", "fp32")
    A = uniform_spins(1, n, [0, 0, 1.0])
    B = random_spins(1, n, 3)
    chain = nlerp_chain(A, B, 6, jitter=0.02, seed=1)
    chain[3].reshape(3, -1)[0, 17] = math.nan
    X = torch.from_numpy(np.ascontiguousarray(chain)).cuda()
    _expect_numeric(s.path, X, method=method, optimizer=optimizer, dt=0.01, tol=1e30, max_iter=10, check_every=1)


# The FP32 field path rounds the FP64 spins to the nearest FP32 value, a value exactly halfway between two
# FP32 values to the one of larger magnitude: nearest-neighbour exchange J = 1 around one non-zero spin
# whose components are such halfway values (and one whose are not), open faces, so each neighbour's FP32
# field is that spin rounded.
@pytest.mark.parametrize("fam", ["stencil", "fft"])
def test_fp32_field_rounds_spins_to_nearest_even(fam):
    from workloads import SC_POS, cubic_cell
    n = (32, 8, 8)
    pbc = (1, 1, 1) if fam == "fft" else (0, 0, 0)
    s = sx.SpinSystem(n, pbc, cubic_cell(), SC_POS, [1.0])
    s.add_shell_exchange(1, 1.0)
    s.plan(fam, "fp32")
    ties = [1 + 2.0 ** -24, -(0.5 + 2.0 ** -25), 0.75 + 2.0 ** -25]   # halfway between FP32 neighbours
    away = [1 + 2.0 ** -23, -(0.5 + 2.0 ** -24), 0.75 + 2.0 ** -24]   # their larger-magnitude neighbours
    plain = [0.3, -0.6, 0.7]
    for comps, rounded in ((ties, away), (plain, plain)):
        S = torch.zeros(3, 1, n[2], n[1], n[0], dtype=torch.float64, device="cuda")
        S[:, 0, 4, 4, 10] = torch.tensor(comps, dtype=torch.float64)
        b = s.field(S, dtype=torch.float32)
        want = torch.tensor(rounded, dtype=torch.float64).float().cuda()
        if fam == "stencil":  # sums of exact FP32 products with zeros: the rounded spin itself
            for z, y, x in [(4, 4, 9), (4, 4, 11), (4, 3, 10), (4, 5, 10), (3, 4, 10), (5, 4, 10)]:
                assert torch.equal(b[:, 0, z, y, x], want), (comps, (z, y, x))
        else:  # transforms in FP32 round further: within a few FP32 ulps of the rounded spin
            for z, y, x in [(4, 4, 9), (4, 4, 11)]:
                assert torch.allclose(b[:, 0, z, y, x], want, atol=2e-6, rtol=0)


def test_fp32_field_may_sit_right_before_the_spins():
    # an FP32 field is half as long as the FP64 spins: a field array that ends where S begins does not
    # overlap it (one allocation, the field in its first 12 nsite bytes, S in the next 24 nsite bytes)
    n = (16, 12, 10)
    s, w = sx.system_from_workload("sc_j123_dmi", n)
    s.plan("stencil", "fp32")
    n3 = 3 * s.nsite
    raw = torch.empty(n3 * 12, dtype=torch.uint8, device="cuda")
    b = raw[: n3 * 4].view(torch.float32)
    S = raw[n3 * 4:].view(torch.float64)
    S.copy_(torch.from_numpy(random_spins(1, n, 4)).reshape(-1))
    sx.sx_field(s.ctx, S, b, s.nsite)
    ref = s.field(S.clone(), dtype=torch.float32).reshape(-1)
    assert torch.equal(b, ref)
    with pytest.raises(sx.SxError):  # one float of real overlap is still refused
        sx.sx_field(s.ctx, S, raw[4: n3 * 4 + 4].view(torch.float32), s.nsite)
