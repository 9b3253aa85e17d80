"""GPU minimum-energy-path methods (string, GNEB, CI-GNEB, geodesic distance) against the CPU oracle,
and the closed-form saddle of a single spin in a transverse field."""
import numpy as np
import pytest

import oracle
import paper_2605_26016_gb300 as sx
from oracle.models import oracle_model
from workloads import cubic_cell, nlerp_chain, polar_chain, random_spins, uniform_spins

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_26016_gb300.build import build
    build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


K, H = 1.0, 0.6
THETA0 = np.arcsin(H / (2 * K))


def macrospin_pair():
    mu_B = oracle.constants()["mu_B"]
    s = sx.SpinSystem((1, 1, 1), (0, 0, 0), cubic_cell(), [[0, 0, 0]], [1.0])
    s.set_zeeman([H / mu_B, 0.0, 0.0])
    s.set_anisotropy(0, K, [0.0, 0.0, 1.0])
    m = oracle.Model((1, 1, 1), (0, 0, 0), cubic_cell(), [[0, 0, 0]], [1.0])
    m.set_zeeman([H / mu_B, 0.0, 0.0])
    m.set_anisotropy(0, K, [0.0, 0.0, 1.0])
    m.build()
    return s, m


@pytest.mark.parametrize("method", ["gneb", "ci_gneb", "string"])
def test_macrospin_path_matches_oracle_and_converges(method):
    s, m = macrospin_pair()
    s.plan("gather", "fp64")
    chain = polar_chain(THETA0, np.pi - THETA0, 9, phi_bulge=0.8)
    d = dev(chain)
    it, E, fm = s.path(d, method=method, dt=0.1, k_spring=1.0, tol=0.0, max_iter=25, check_every=25)
    assert it == 25
    if method == "string":
        ref, Er, fr = m.string(chain, dt=0.1, niter=25)
    else:
        ref, Er, fr = m.gneb(chain, dt=0.1, k=1.0, niter=25, climbing=method == "ci_gneb")
    assert np.abs(d.cpu().numpy() - ref).max() < 1e-12
    assert np.abs(np.array(E) - Er).max() < 1e-12
    assert fm == pytest.approx(fr, rel=1e-10, abs=1e-14)
    # run on to convergence: the x-z meridian through +x, saddle E = -h for CI-GNEB
    it, E, fm = s.path(d, method=method, dt=0.1, k_spring=1.0, tol=1e-10 if method != "string" else 0.0,
                       max_iter=6000, check_every=100)
    S = d.cpu().numpy().reshape(9, 3)
    assert np.abs(S[:, 1]).max() < 1e-8 and np.all(S[:, 0] > 0)
    theta = np.arctan2(S[:, 0], S[:, 2])
    if method == "ci_gneb":
        assert fm < 1e-10
        top = int(np.argmax(E[1:-1])) + 1
        assert E[top] == pytest.approx(-H, abs=1e-12)
        assert E[top] - E[0] == pytest.approx(K * (1 - H / (2 * K)) ** 2, abs=1e-12)
    else:
        expect = THETA0 + (np.pi - 2 * THETA0) * np.arange(9) / 8
        assert np.abs(theta - expect).max() < 1e-8


def chain_case(name, n, pbc, nimg, seed, **override):
    s, w = sx.system_from_workload(name, n, pbc=pbc, **override)
    m, _ = oracle_model(name, n, pbc=pbc, **override)
    nsub = len(w["pos"])
    A = random_spins(nsub, n, seed)
    B = random_spins(nsub, n, seed + 1)
    chain = nlerp_chain(A, B, nimg, jitter=0.1, seed=seed)
    return s, m, chain


CASES = [
    # name, n, pbc, backend, precision, tolerance on spins, dt
    ("sc_j123_dmi", (12, 10, 8), (1, 1, 0), "gather", "fp64", 1e-11, 0.02),
    ("sc_j123_dmi", (12, 10, 8), (1, 1, 0), "stencil", "fp32", 2e-5, 0.02),
    ("bcc_4shell", (8, 6, 5), (1, 1, 1), "stencil", "fp32", 2e-5, 5e-4),
    ("sc_j123_dmi", (16, 8, 8), (1, 1, 1), "fft", "fp32", 2e-5, 0.02),
    ("sc_j123", (12, 12, 9), (1, 1, 0), "igemm_tc", "bf16", 2e-4, 0.05),
]


@pytest.mark.parametrize("method", ["gneb", "ci_gneb", "string"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_chain_iterations_match_oracle(case, method):
    name, n, pbc, backend, prec, tol, dt = CASES[case]
    s, m, chain = chain_case(name, n, pbc, 7, 20 + case, B=[0.0, 0.4, 0.8])
    s.plan(backend, prec)
    d = dev(chain)
    it, E, fm = s.path(d, method=method, dt=dt, k_spring=0.5, max_iter=4, check_every=4)
    assert it == 4
    if method == "string":
        ref, Er, fr = m.string(chain, dt=dt, niter=4)
    else:
        ref, Er, fr = m.gneb(chain, dt=dt, k=0.5, niter=4, climbing=method == "ci_gneb")
    got = d.cpu().numpy()
    assert np.array_equal(got[0], chain[0]) and np.array_equal(got[-1], chain[-1])
    assert np.abs(got - ref).max() < tol
    scale = max(1.0, np.abs(Er).max())
    assert np.abs(np.array(E) - Er).max() < (1e-11 if prec == "fp64" else 1e-5) * scale
    assert fm == pytest.approx(fr, rel=1e-9 if prec == "fp64" else 1e-4)
    norms = np.sqrt((got * got).sum(1))
    assert np.abs(norms - 1).max() < 1e-13


def test_geodesic_matches_oracle_and_rigid_rotation():
    n = (10, 9, 8)
    s = sx.SpinSystem(n, (1, 1, 1), cubic_cell(), [[0, 0, 0], [0.5, 0.5, 0.5]], [1.0, 1.0])
    s.add_shell_exchange(1, 1.0)
    s.plan("gather", "fp64")
    A, B = random_spins(2, n, 1), random_spins(2, n, 2)
    assert s.geodesic(dev(A), dev(B)) == pytest.approx(oracle.geodesic(A, B), rel=1e-13)
    U = uniform_spins(2, n, [0, 0, 1])
    V = uniform_spins(2, n, [np.sin(1e-5), 0, np.cos(1e-5)])
    assert s.geodesic(dev(U), dev(V)) == pytest.approx(np.sqrt(2 * 720) * 1e-5, rel=1e-9)


def test_stiff_cluster_ci_gneb_barrier_on_gpu():
    n = (2, 2, 2)
    s = sx.SpinSystem(n, (0, 0, 0), cubic_cell(), [[0, 0, 0]], [1.0])
    s.add_shell_exchange(1, 10.0)
    s.set_anisotropy(0, 0.1, [0.0, 0.0, 1.0])
    s.plan("gather", "fp64")
    chain = nlerp_chain(uniform_spins(1, n, [0, 0, 1]), uniform_spins(1, n, [0, 0, -1]), 7, jitter=0.05, seed=3)
    d = dev(chain)
    it, E, fm = s.path(d, method="ci_gneb", dt=0.02, k_spring=1.0, tol=1e-8, max_iter=20000, check_every=200)
    assert fm < 1e-8
    assert max(E) - E[0] == pytest.approx(8 * 0.1, abs=1e-9)


def test_path_rejects_bad_arguments():
    s, _ = macrospin_pair()
    s.plan("gather", "fp64")
    d = dev(polar_chain(0.1, 3.0, 3))
    for kw in (dict(dt=0.0), dict(k_spring=-1.0), dict(tol=-1.0), dict(check_every=0), dict(method=7)):
        args = dict(method="gneb", dt=0.1, max_iter=1)
        args.update(kw)
        with pytest.raises(sx.SxError):
            sx.sx_path_step(s.ctx, d, 3, 1, **args)
    with pytest.raises(sx.SxError):
        sx.sx_path_step(s.ctx, d[:2].contiguous(), 2, 1, method="gneb", dt=0.1, max_iter=1)


def test_zero_iterations_report_energies_only():
    s, m = macrospin_pair()
    s.plan("gather", "fp64")
    chain = polar_chain(THETA0, np.pi - THETA0, 5, phi_bulge=0.3)
    d = dev(chain)
    it, E, fm = s.path(d, method="gneb", dt=0.1, max_iter=0)
    assert it == 0 and fm == -1.0
    assert np.array_equal(d.cpu().numpy(), chain)
    Er = [m.energy(c) for c in chain]
    assert np.abs(np.array(E) - Er).max() < 1e-13


def test_full_size_ci_gneb_iteration_bcc_64_32_images():
    # 32 images of the bcc four-shell model at 64^3 conventional cells (524,288 spins per image):
    # one climbing-image iteration on the stencil backend against the oracle's, every site
    n = (64, 64, 64)
    s, w = sx.system_from_workload("bcc_4shell", n)
    s.plan("stencil", "fp32")
    m, _ = oracle_model("bcc_4shell", n)
    A = uniform_spins(2, n, [0.0, 0.0, 1.0])
    B = random_spins(2, n, 41)
    chain = nlerp_chain(A, B, 32, jitter=0.02, seed=4)
    d = dev(chain)
    it, E, fm = s.path(d, method="ci_gneb", dt=2e-4, k_spring=1.0, max_iter=1)
    ref, Er, fr = m.gneb(chain, dt=2e-4, k=1.0, niter=1, climbing=True)
    assert np.abs(d.cpu().numpy() - ref).max() < 2e-5
    assert np.abs(np.array(E) - Er).max() < 1e-5 * np.abs(Er).max()
    assert fm == pytest.approx(fr, rel=1e-4)


@pytest.mark.parametrize("method", ["gneb", "ci_gneb"])
@pytest.mark.parametrize("case", [0, 1, 2])
def test_vp_chain_iterations_match_oracle_and_carry_velocity(case, method):
    name, n, pbc, backend, prec, tol, dt = CASES[case]
    s, m, chain = chain_case(name, n, pbc, 7, 40 + case, B=[0.0, 0.4, 0.8])
    s.plan(backend, prec)
    d = dev(chain)
    kw = dict(method=method, dt=dt, k_spring=0.5, optimizer="vp", check_every=3)
    it, E, fm = s.path(d, max_iter=3, **kw)
    it2, E2, fm2 = s.path(d, max_iter=3, keep_velocity=True, **kw)
    assert it == 3 and it2 == 3
    ref, Er, fr, st = m.gneb_vp(chain, dt=dt, k=0.5, niter=3, climbing=method == "ci_gneb")
    ref, Er, fr, st = m.gneb_vp(ref, dt=dt, k=0.5, niter=3, climbing=method == "ci_gneb", state=st)
    got = d.cpu().numpy()
    assert np.array_equal(got[0], chain[0]) and np.array_equal(got[-1], chain[-1])
    assert np.abs(got - ref).max() < tol
    scale = max(1.0, np.abs(Er).max())
    assert np.abs(np.array(E2) - Er).max() < (1e-11 if prec == "fp64" else 1e-5) * scale
    assert fm2 == pytest.approx(fr, rel=1e-9 if prec == "fp64" else 1e-4)
    # without keep_velocity the second call starts at rest: a different chain
    d2 = dev(chain)
    s.path(d2, max_iter=3, **kw)
    s.path(d2, max_iter=3, **kw)
    rest, _, _, _ = m.gneb_vp(m.gneb_vp(chain, dt=dt, k=0.5, niter=3, climbing=method == "ci_gneb")[0], dt=dt,
                                k=0.5, niter=3, climbing=method == "ci_gneb")
    assert np.abs(d2.cpu().numpy() - rest).max() < tol
    assert np.abs(rest - ref).max() > 5 * tol


def test_vp_ci_gneb_converges_macrospin_faster():
    s, m = macrospin_pair()
    s.plan("gather", "fp64")
    chain = polar_chain(THETA0, np.pi - THETA0, 9, phi_bulge=0.8)
    d = dev(chain)
    it, E, fm = s.path(d, method="ci_gneb", dt=0.1, k_spring=1.0, tol=1e-10, max_iter=6000, check_every=10,
                       optimizer="vp")
    d2 = dev(chain)
    it_sd, _, _ = s.path(d2, method="ci_gneb", dt=0.1, k_spring=1.0, tol=1e-10, max_iter=6000, check_every=10)
    assert fm < 1e-10 and it < it_sd / 2
    top = int(np.argmax(E[1:-1])) + 1
    assert E[top] - E[0] == pytest.approx(K * (1 - H / (2 * K)) ** 2, abs=1e-12)
    with pytest.raises(sx.SxError) as e:
        s.path(d, method="string", optimizer="vp", max_iter=1)
    assert e.value.code == sx.SX_ERR_UNSUPPORTED
