"""Pins of the CPU oracle against results fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: textbook
coordination numbers, closed-form lattice sums for ferromagnets, spirals,
cycloids and helices, the derivative relation b = -dE/dS, the analytic
single-spin LLG solution, the invariants of undamped dynamics, the Langevin
function of a thermal spin, and the statistics of the normal noise.
"""
import math

import numpy as np
import pytest

import oracle
from oracle.models import oracle_model
from workloads import A_NM, BCC_POS, SC_POS, cubic_cell, random_spins, uniform_spins

C = oracle.constants()
MU_B, GAMMA, K_B = C["mu_B"], C["gamma"], C["k_B"]


def test_paper_constants_golden():
    # tests/golden/paper_constants.txt: the paper rounds mu_B to 5.7884e-2 meV/T
    vals = {}
    with open(__file__.replace("test_oracle_pins.py", "golden/paper_constants.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()
                vals[k] = float(v)
    assert abs(MU_B - vals["mu_B_meV_per_T"]) < 0.5e-6
    assert vals["hopfion_J2_over_J1"] == 0.188


def _coordination(pos, shell, n=(9, 9, 9)):
    m = oracle.Model(n, (1, 1, 1), cubic_cell(1.0), pos, [1.0] * len(pos))
    m.add_shell_exchange(shell, 1.0)
    m.build()
    counts = set()
    for s in range(len(pos)):
        jj, JJ = m.site_pairs(s * n[0] * n[1] * n[2] + 40)
        counts.add(len(jj))
        assert np.allclose(JJ, np.eye(3)[None])
    assert len(counts) == 1
    return counts.pop(), m.shell_radii(shell)[-1]


@pytest.mark.parametrize("shell,count,radius", [(1, 6, 1.0), (2, 12, math.sqrt(2)), (3, 8, math.sqrt(3)),
                                                (4, 6, 2.0)])
def test_sc_shells(shell, count, radius):
    c, r = _coordination(SC_POS, shell)
    assert c == count and abs(r - radius) < 1e-12


@pytest.mark.parametrize("shell,count,radius", [(1, 8, math.sqrt(3) / 2), (2, 6, 1.0), (3, 12, math.sqrt(2)),
                                                (4, 24, math.sqrt(11) / 2)])
def test_bcc_shells(shell, count, radius):
    c, r = _coordination(BCC_POS, shell)
    assert c == count and abs(r - radius) < 1e-12


def test_open_boundary_drops_bonds():
    m = oracle.Model((4, 4, 4), (1, 1, 0), cubic_cell(), SC_POS, [1.0])
    m.add_shell_exchange(1, 1.0)
    m.build()
    assert len(m.site_pairs(0)[0]) == 5            # z = 0 face
    assert len(m.site_pairs(16)[0]) == 6           # z = 1 interior
    assert len(m.site_pairs(3 * 16 + 5)[0]) == 5   # z = 3 face
    assert m.npair() == 64 * 6 - 2 * 16


def test_bond_reverse_is_transpose():
    # an unordered bond between sublattices expands into two directed bonds,
    # the reverse one carrying the transposed tensor (J_ji^{ba} = J_ij^{ab})
    rng = np.random.default_rng(7)
    J = rng.normal(size=(3, 3))
    m = oracle.Model((5, 5, 5), (1, 1, 1), cubic_cell(), BCC_POS, [1.0, 1.0])
    m.add_bond(0, 1, (1, 0, -1), J)
    m.build()
    n3 = 125
    i = 2 * 25 + 2 * 5 + 2          # sublattice 0, cell (2,2,2)
    jj, JJ = m.site_pairs(i)
    assert len(jj) == 1 and jj[0] == n3 + 1 * 25 + 2 * 5 + 3 and np.array_equal(JJ[0], J)
    jb, Jb = m.site_pairs(n3 + 1 * 25 + 2 * 5 + 3)  # sublattice 1, cell (3,2,1) -> back to (2,2,2)
    assert len(jb) == 1 and jb[0] == i and np.array_equal(Jb[0], J.T)


def test_ferromagnet_closed_form():
    # uniform state: b = (sum_k z_k J_k) S + mu mu_B B + 2 K (S.n) n, per-site energy
    # -1/2 sum z_k J_k - mu mu_B B.S - K (S.n)^2 (bcc coordination 8, 6, 12, 24)
    n = (6, 6, 6)
    m, w = oracle_model("bcc_4shell", n, B=[0.3, -0.2, 1.5])
    d = np.array([0.3, -0.5, 0.8])
    d /= np.linalg.norm(d)
    S = uniform_spins(2, n, d)
    Jsum = sum(z * J for z, J in zip((8, 6, 12, 24), w["shells"]))
    K = w["K"][0]
    mu = w["mu"][0]
    expect = Jsum * d + mu * MU_B * np.array(w["B"]) + 2 * K * d[2] * np.array([0, 0, 1.0])
    b = m.field(S)
    assert np.abs(b - expect[:, None, None, None, None]).max() < 1e-12
    e = m.energy(S) / (2 * 216)
    e_expect = -0.5 * Jsum - mu * MU_B * np.dot(w["B"], d) - K * d[2] ** 2
    assert abs(e - e_expect) < 1e-12


def _spiral(pos, n, q):
    nx, ny, nz = n
    S = np.empty((3, len(pos), nz, ny, nx))
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for s, p in enumerate(pos):
        ph = q[0] * (x + p[0]) + q[1] * (y + p[1]) + q[2] * (z + p[2])
        S[0, s], S[1, s], S[2, s] = np.cos(ph), np.sin(ph), 0.0
    return S


def test_sc_spiral_closed_form():
    # flat spiral S = (cos q.r, sin q.r, 0): b = J(q) S with the simple-cubic lattice sums
    n = (12, 8, 6)
    J = [1.0, -0.3, 0.25, 0.1]
    m = oracle.Model(n, (1, 1, 1), cubic_cell(), SC_POS, [1.0])
    for k, Jk in enumerate(J):
        m.add_shell_exchange(k + 1, Jk)
    m.build()
    q = 2 * np.pi * np.array([1 / 12, 2 / 8, 1 / 6])
    cx, cy, cz = np.cos(q)
    Jq = (2 * J[0] * (cx + cy + cz) + 4 * J[1] * (cx * cy + cy * cz + cz * cx) + 8 * J[2] * cx * cy * cz
          + 2 * J[3] * (np.cos(2 * q[0]) + np.cos(2 * q[1]) + np.cos(2 * q[2])))
    S = _spiral(SC_POS, n, q)
    assert np.abs(m.field(S) - Jq * S).max() < 1e-12


def test_bcc_spiral_closed_form():
    n = (8, 8, 8)
    m, w = oracle_model("bcc_4shell", n, K=None)
    J = w["shells"]
    q = 2 * np.pi * np.array([1 / 8, 3 / 8, 2 / 8])
    c = np.cos(q)
    h = np.cos(q / 2)
    t = np.cos(3 * q / 2)
    Jq = (8 * J[0] * h[0] * h[1] * h[2] + 2 * J[1] * c.sum() + 4 * J[2] * (c[0] * c[1] + c[1] * c[2] + c[2] * c[0])
          + 8 * J[3] * (t[0] * h[1] * h[2] + h[0] * t[1] * h[2] + h[0] * h[1] * t[2]))
    S = _spiral(BCC_POS, n, q)
    assert np.abs(m.field(S) - Jq * S).max() < 1e-11


def test_interfacial_dmi_cycloid():
    # cycloid S = (sin qx, 0, cos qx) with interfacial D_ij = D (z x r_ij): b = (J(q) + 2 D sin q) S,
    # per-site energy -1/2 (J(q) + 2 D sin q) (pair energy -J S_i.S_j - D_ij.(S_i x S_j))
    n = (16, 4, 4)
    J1, D = 1.3, 0.4
    m = oracle.Model(n, (1, 1, 1), cubic_cell(), SC_POS, [1.0])
    m.add_shell_exchange(1, J1)
    m.add_dmi(1, 0, D)
    m.build()
    q = 2 * np.pi * 3 / 16
    x = np.arange(16)[None, None, :] * np.ones((4, 4, 1))
    S = np.stack([np.sin(q * x), np.zeros_like(x), np.cos(q * x)])[:, None]
    lam = 2 * J1 * (np.cos(q) + 2) + 2 * D * np.sin(q)
    assert np.abs(m.field(S) - lam * S).max() < 1e-12
    assert abs(m.energy(S) / 256 + 0.5 * lam) < 1e-12


def test_bulk_dmi_helix():
    # helix S = (cos qz, sin qz, 0) with bulk D_ij = D r_ij: b = (J(q) + 2 D sin q) S
    n = (4, 4, 16)
    J1, D = 0.7, -0.25
    m = oracle.Model(n, (1, 1, 1), cubic_cell(), SC_POS, [1.0])
    m.add_shell_exchange(1, J1)
    m.add_dmi(1, 1, D)
    m.build()
    q = 2 * np.pi * 5 / 16
    z = np.arange(16)[:, None, None] * np.ones((1, 4, 4))
    S = np.stack([np.cos(q * z), np.sin(q * z), np.zeros_like(z)])[:, None]
    lam = 2 * J1 * (np.cos(q) + 2) + 2 * D * np.sin(q)
    assert np.abs(m.field(S) - lam * S).max() < 1e-12


def test_field_is_minus_energy_gradient():
    # b_i = -dH/dS_i for every term (bilinear incl. a general non-symmetric tensor bond, DMI,
    # Zeeman, anisotropy), checked by central differences on a small open/periodic lattice
    n = (4, 5, 3)
    rng = np.random.default_rng(11)
    m, w = oracle_model("bcc_4shell", n, pbc=(1, 1, 0), B=[0.4, -1.0, 2.0], build=False)
    m.add_dmi(2, 1, 0.7)
    m.add_dmi(1, 1, -0.3)
    m.add_bond(0, 1, (0, -1, 1), rng.normal(size=(3, 3)))
    m.add_bond(1, 1, (1, 0, 0), rng.normal(size=(3, 3)))
    m.set_anisotropy(1, -0.8, [1.0, 1.0, 0.0])
    m.build()
    S = random_spins(2, n, 5)
    b = m.field(S)
    h = 1e-5
    for flat in rng.choice(S.size, 40, replace=False):
        Sp = S.copy().reshape(-1)
        Sm = S.copy().reshape(-1)
        Sp[flat] += h
        Sm[flat] -= h
        g = (m.energy(Sp) - m.energy(Sm)) / (2 * h)
        assert abs(-g - b.reshape(-1)[flat]) < 1e-6 * max(1.0, abs(g))


def _single_spin(B0, mu=1.0):
    m = oracle.Model((1, 1, 1), (0, 0, 0), cubic_cell(), SC_POS, [mu])
    m.set_zeeman([0.0, 0.0, B0])
    m.build()
    return m


def _larmor_rmse(dt, alpha=0.1, B0=10.0, t_end=100000.0, sample=1000.0):
    m = _single_spin(B0)
    th0 = math.pi / 3
    S = np.array([math.sin(th0), 0.0, math.cos(th0)]).reshape(3, 1, 1, 1, 1)
    gp = GAMMA / (1 + alpha * alpha)
    err2 = []
    per = int(round(sample / dt))
    for k in range(1, int(t_end / sample) + 1):
        S = m.heun(S, dt, alpha, nsteps=per)
        t = k * sample
        ph = gp * B0 * t
        th = 2 * math.atan(math.tan(th0 / 2) * math.exp(-alpha * gp * B0 * t))
        ex = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        err2.append(((S.reshape(3) - ex) ** 2).sum())
    return math.sqrt(np.mean(err2))


def test_larmor_precession_second_order():
    # single spin in B || z: phi = gamma' B t, tan(theta/2) = tan(theta0/2) exp(-alpha gamma' B t);
    # the Heun trajectory error falls as dt^2 (the fp64 curve of the single-spin benchmark)
    r = [_larmor_rmse(dt) for dt in (2.0, 4.0, 8.0)]
    assert r[0] < 1e-3
    for a, b in zip(r, r[1:]):
        assert 3.4 < b / a < 4.6


def test_undamped_invariants():
    # alpha = 0, T = 0: |S| = 1 to rounding, energy conserved up to O(dt^2)
    n = (6, 6, 6)
    m, w = oracle_model("sc_j123", n, pbc=(1, 1, 1), B=[0.0, 0.0, 3.0])
    S0 = random_spins(1, n, 21)
    E0 = m.energy(S0)
    drifts = []
    # random spins are strongly chaotic: the dt^2 regime starts below ~0.5 fs
    for dt, steps in ((0.25, 1600), (0.125, 3200)):
        S = m.heun(S0, dt, 0.0, nsteps=steps)
        assert np.abs(np.sqrt((S ** 2).sum(0)) - 1).max() < 1e-14
        drifts.append(abs(m.energy(S) - E0))
    assert drifts[0] < 1e-4 * abs(E0)
    assert 3.0 < drifts[0] / drifts[1] < 5.0


def test_isotropic_exchange_conserves_total_spin():
    n = (6, 6, 6)
    m, w = oracle_model("sc_j123", n, pbc=(1, 1, 1))
    S0 = random_spins(1, n, 22)
    M0 = S0.reshape(3, -1).sum(1)
    d = []
    for dt, steps in ((1.0, 200), (0.5, 400)):
        S = m.heun(S0, dt, 0.0, nsteps=steps)
        d.append(np.abs(S.reshape(3, -1).sum(1) - M0).max())
    # the Heun error of the total spin is at least second order (here it is third)
    assert d[0] < 1e-4 * 216
    assert d[0] / d[1] > 3.5


def _langevin(x):
    return 1.0 / math.tanh(x) - 1.0 / x


@pytest.mark.slow
def test_thermal_spin_langevin_function():
    # independent spins in B at temperature T: <S_z> -> L(mu mu_B B / kB T) (Langevin function),
    # which pins the thermal-field amplitude sigma = sqrt(2 alpha kB T / (gamma mu mu_B dt))
    n = (16, 16, 16)
    B0, alpha, dt = 5.0, 1.0, 1.0
    x = 1.0
    T = MU_B * B0 / (K_B * x)
    m = oracle.Model(n, (1, 1, 1), cubic_cell(), SC_POS, [1.0])
    m.set_zeeman([0.0, 0.0, B0])
    m.build()
    S = uniform_spins(1, n, [0, 0, 1])
    S = m.heun(S, dt, alpha, T=T, seed=99, step0=0, nsteps=7000)
    acc = []
    step = 7000
    for _ in range(40):
        S = m.heun(S, dt, alpha, T=T, seed=99, step0=step, nsteps=500)
        step += 500
        acc.append(S[2].mean())
    assert abs(np.mean(acc) - _langevin(x)) < 0.015


def test_normal_noise_statistics():
    from scipy import stats
    eta = oracle.normals(12345, 3, 1000, 100000, 17).astype(np.float64)
    N = eta.size
    assert abs(eta.mean()) < 5 / math.sqrt(N)
    assert abs(eta.var() - 1) < 5 * math.sqrt(2 / N)
    assert abs(stats.kurtosis(eta.reshape(-1), fisher=False) - 3) < 5 * math.sqrt(24 / N)
    for c in range(3):
        assert stats.kstest(eta[:, c], "norm").pvalue > 1e-3
    cc = np.corrcoef(eta.T)
    assert np.abs(cc - np.eye(3)).max() < 5 / math.sqrt(eta.shape[0])


def test_box_muller_transform_is_accurate():
    # the FP32 normals equal the Box-Muller transform of the same Philox words evaluated in FP64 with
    # libm's log, cos and sin, to a few FP32 ulps: pins the project-written log and sincos
    rng = np.random.default_rng(3)
    for site in rng.integers(0, 2 ** 40, size=4000):
        site = int(site)
        x = oracle.philox4x32_10((site & 0xFFFFFFFF, site >> 32, 11, 2 << 8), (77, 0))
        u = [(2 * (w >> 9) + 1) * 2.0 ** -24 for w in x]
        r0, r1 = math.sqrt(-2 * math.log(u[0])), math.sqrt(-2 * math.log(u[2]))
        ref = np.array([r0 * math.cos(2 * math.pi * u[1]), r0 * math.sin(2 * math.pi * u[1]),
                        r1 * math.cos(2 * math.pi * u[3])])
        got = oracle.normals(77, 2, site, 1, 11)[0].astype(np.float64)
        assert np.abs(got - ref).max() <= 4e-7 * max(1.0, np.abs(ref).max())


def test_noise_is_counter_based():
    a = oracle.normals(7, 0, 50, 10, 3)
    b = oracle.normals(7, 0, 55, 5, 3)
    assert np.array_equal(a[5:], b)
    assert not np.array_equal(oracle.normals(7, 0, 50, 10, 4), a)
    assert not np.array_equal(oracle.normals(8, 0, 50, 10, 3), a)
    assert not np.array_equal(oracle.normals(7, 1, 50, 10, 3), a)


def test_philox_words_uniform():
    from scipy import stats
    words = np.array([oracle.philox4x32_10((i, 0, 5, 0), (1, 2)) for i in range(20000)], dtype=np.float64)
    u = (words + 0.5) / 2.0 ** 32
    for c in range(4):
        assert stats.kstest(u[:, c], "uniform").pvalue > 1e-3
    bits = np.unpackbits(np.array(words, dtype=np.uint32).view(np.uint8))
    assert abs(bits.mean() - 0.5) < 5 * 0.5 / math.sqrt(bits.size)


def test_philox_known_answer_vectors():
    # tests/golden/philox4x32_10_kat.txt: the generator's published known-answer vectors
    # (Salmon et al., SC'11, Random123 kat_vectors); a wrong multiplier, Weyl constant,
    # round count or word permutation changes every output word
    rows = []
    with open(__file__.replace("test_oracle_pins.py", "golden/philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append([int(v, 16) for v in line.split()])
    assert len(rows) == 3
    for r in rows:
        assert oracle.philox4x32_10(r[0:4], r[4:6]) == r[6:10]


@pytest.mark.parametrize("name,n,pbc", [("bcc_4shell", (5, 4, 6), (1, 0, 1)), ("sc_j123_dmi", (6, 5, 4), None)])
def test_heun_at_sites_equals_full_step(name, n, pbc):
    # the sampled-site Heun step (used for checks at full lattice size) is the same arithmetic as a full step
    m, w = oracle_model(name, n, pbc=pbc)
    S = random_spins(m.nsub, n, 44)
    full = m.heun(S, w["dt"], w["alpha"], T=w["T"] or 30.0, seed=5, replica=2, step0=17, nsteps=1).reshape(3, -1)
    sites = np.arange(m.nsite)
    part = m.heun_sites(S, sites, w["dt"], w["alpha"], T=w["T"] or 30.0, seed=5, replica=2, step=17)
    assert np.array_equal(part.T, full)


@pytest.mark.parametrize("name,n,pbc,dipolar", [("bcc_4shell", (5, 4, 6), (1, 0, 1), False),
                                                 ("sc_j123_dmi", (6, 5, 4), None, False),
                                                 ("sc_j123_dmi", (4, 4, 4), (1, 1, 1), True),
                                                 ("sc_nn", (4, 3, 5), (0, 0, 0), True)])
def test_field_at_sites_equals_full_field(name, n, pbc, dipolar):
    # the sampled-site field (used for checks at full lattice size, dipolar included) is the full field
    # restricted to those sites, on periodic, mixed and open faces
    m, w = oracle_model(name, n, pbc=pbc, dipolar=dipolar)
    S = random_spins(m.nsub, n, 45)
    full = m.field(S).reshape(3, -1)
    sites = np.arange(m.nsite)[::-1].copy()
    part = m.field_sites(S, sites)
    assert np.abs(part.T - full[:, sites]).max() <= 1e-14 * np.abs(full).max()


def _single_spins(theta, phi):
    return np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)]).reshape(
        3, 1, 1, 1, len(theta))


def test_torque_max_single_spins_closed_form():
    # uncoupled spins (open chain, no bonds) at polar angles theta: in B || z the torque is
    # |S x b| = mu mu_B B sin(theta); with uniaxial K along z it is 2K |cos(theta)| sin(theta)
    theta = np.array([0.3, 1.1, 2.9, 0.7, 1.9])
    phi = np.array([0.0, 2.0, -1.0, 0.5, 4.0])
    n = (len(theta), 1, 1)
    S = _single_spins(theta, phi)
    mu, B = 2.0, 1.5
    m = oracle.Model(n, (0, 0, 0), cubic_cell(), SC_POS, [mu])
    m.set_zeeman([0.0, 0.0, B])
    m.build()
    expect = mu * MU_B * B * np.sin(theta).max()       # the last site, sin(1.9)
    assert abs(m.torque_max(S) - expect) < 1e-15
    K = 0.25
    m = oracle.Model(n, (0, 0, 0), cubic_cell(), SC_POS, [mu])
    m.set_anisotropy(0, K, [0.0, 0.0, 1.0])
    m.build()
    expect = (2 * K * np.abs(np.cos(theta)) * np.sin(theta)).max()   # the fourth site, theta = 0.7
    assert abs(m.torque_max(S) - expect) < 1e-15


def test_torque_max_cycloid_in_field():
    # interfacial-DMI cycloid S = (sin qx, 0, cos qx) with exchange and DMI has b_bil = lambda S (no
    # bilinear torque); adding B || z leaves |S x b| = mu mu_B B |sin qx|, largest over the sites
    n = (16, 4, 4)
    J1, D, B = 1.3, 0.4, 0.8
    m = oracle.Model(n, (1, 1, 1), cubic_cell(), SC_POS, [1.0])
    m.add_shell_exchange(1, J1)
    m.add_dmi(1, 0, D)
    m.set_zeeman([0.0, 0.0, B])
    m.build()
    q = 2 * np.pi * 3 / 16
    x = np.arange(16)[None, None, :] * np.ones((4, 4, 1))
    S = np.stack([np.sin(q * x), np.zeros_like(x), np.cos(q * x)])[:, None]
    expect = MU_B * B * np.abs(np.sin(q * np.arange(16))).max()
    assert abs(m.torque_max(S) - expect) < 1e-13


def test_stochastic_step_uses_same_noise_in_both_stages():
    # with J = 0 one stochastic Heun step of a single spin equals the deterministic Heun step in the
    # constant field B_ext + sigma*eta (eta from the site/step counter), which is only true if the
    # predictor and corrector share eta
    n = (2, 1, 1)
    m = oracle.Model(n, (1, 1, 1), cubic_cell(), SC_POS, [2.0])
    m.set_zeeman([0.1, 0.2, 1.0])
    m.build()
    S0 = random_spins(1, n, 3)
    dt, alpha, T = 0.5, 0.3, 80.0
    S1 = m.heun(S0, dt, alpha, T=T, seed=42, step0=9, nsteps=1)
    eta = oracle.normals(42, 0, 0, 2, 9).astype(np.float64)
    sigma = math.sqrt(2 * alpha * K_B * T / (GAMMA * 2.0 * MU_B * dt))
    for i in range(2):
        mi = oracle.Model((1, 1, 1), (0, 0, 0), cubic_cell(), SC_POS, [2.0])
        mi.set_zeeman(np.array([0.1, 0.2, 1.0]) + sigma * eta[i])
        mi.build()
        ref = mi.heun(S0[:, :, :, :, i:i + 1], dt, alpha, nsteps=1)
        assert np.abs(ref.reshape(3) - S1[:, 0, 0, 0, i]).max() < 1e-15


# ---------------------------------------------------------------- dipolar

def test_mu_b_and_dipolar_prefactor_from_first_principles():
    # mu_B = e hbar / (2 m_e) from the exact SI e and h (hbar = h / 2 pi) and CODATA 2018 m_e (relative
    # uncertainty 3e-10); mu0/4pi = 1e-7 T m/A to 1e-10
    e, h, me = 1.602176634e-19, 6.62607015e-34, 9.1093837015e-31
    mu_b_JT = e * (h / (2 * math.pi)) / (2 * me)
    assert abs(MU_B / (mu_b_JT / e * 1e3) - 1) < 1e-9                  # meV/T
    pref = 1e-7 * mu_b_JT ** 2 / e * 1e3 * 1e27                        # J m^3 -> meV nm^3
    assert abs(C["dip_pref"] / pref - 1) < 2e-9


def test_two_dipoles_textbook_field():
    # b_1 = (mu0 mu_B^2/4pi) mu_1 mu_2 (3 (S_2.e) e - S_2) / r^3 for two moments on an open lattice
    a = 0.3
    m = oracle.Model((2, 1, 1), (0, 0, 0), cubic_cell(a), SC_POS, [2.0])
    m.set_dipolar(True)
    m.build()
    S = np.zeros((3, 1, 1, 1, 2))
    S[:, 0, 0, 0, 0] = [0.0, 0.6, 0.8]
    S[:, 0, 0, 0, 1] = [0.48, 0.6, 0.64]
    b = m.field(S)
    ex = np.array([1.0, 0.0, 0.0])
    S2 = S[:, 0, 0, 0, 1]
    expect = C["dip_pref"] * 4.0 * (3 * ex * (ex @ S2) - S2) / a ** 3
    assert np.abs(b[:, 0, 0, 0, 0] - expect).max() < 1e-14 * np.abs(expect).max() + 1e-18


@pytest.mark.parametrize("L", [4, 5, 6])
def test_uniform_state_zero_dipolar_field_in_periodic_cube(L):
    # uniform magnetisation in a periodic cubic box: the minimum-image sum (with half-period images split
    # evenly) is cubic-symmetric, so the dipolar field vanishes (sum of (3 e e - I)/r^3 is traceless and
    # isotropic)
    m = oracle.Model((L, L, L), (1, 1, 1), cubic_cell(), SC_POS, [2.2])
    m.set_dipolar(True)
    m.build()
    d = np.array([0.3, -0.5, 0.8])
    S = uniform_spins(1, (L, L, L), d)
    b = m.field(S)
    scale = C["dip_pref"] * 2.2 ** 2 / A_NM ** 3
    assert np.abs(b).max() < 1e-12 * scale
    # a non-uniform state does feel a dipolar field
    S2 = random_spins(1, (L, L, L), 3)
    assert np.abs(m.field(S2)).max() > 1e-3 * scale


def test_dipolar_energy_gradient():
    n = (3, 4, 2)
    m = oracle.Model(n, (1, 0, 1), cubic_cell(), [[0, 0, 0], [0.5, 0.5, 0.5]], [2.2, 1.5])
    m.add_shell_exchange(1, 0.3)
    m.set_dipolar(True)
    m.build()
    S = random_spins(2, n, 12)
    b = m.field(S)
    h = 1e-5
    rng = np.random.default_rng(2)
    for flat in rng.choice(S.size, 12, replace=False):
        Sp, Sm = S.copy().reshape(-1), S.copy().reshape(-1)
        Sp[flat] += h
        Sm[flat] -= h
        g = (m.energy(Sp) - m.energy(Sm)) / (2 * h)
        assert abs(-g - b.reshape(-1)[flat]) < 1e-6 * max(1.0, abs(g))
