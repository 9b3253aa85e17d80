"""CPU tests of the C ABI: the library loads, exports what include/sx.h
declares, validates arguments, and builds the same directed couplings as the
oracle's brute-force pair list (host logic only: no CUDA call is made)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2605_26016_gb300 as sx
from oracle.models import oracle_model
from paper_2605_26016_gb300.build import build
from workloads import BCC_POS, SC_POS, cubic_cell

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    build()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sx.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sx_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol():
    names = declared_functions()
    assert len(names) >= 18
    assert sorted(sx.EXPORTS) == names
    L = ctypes.CDLL(sx.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n


def _ctx(n=(4, 4, 4), pbc=(1, 1, 1), pos=SC_POS, mu=None):
    return sx.sx_create(n, pbc, cubic_cell(), pos, mu or [1.0] * len(pos))


def test_create_rejects_bad_lattices():
    with pytest.raises(sx.SxError) as e:
        sx.sx_create((0, 4, 4), (1, 1, 1), cubic_cell(), SC_POS, [1.0])
    assert e.value.code == sx.SX_ERR_ARG
    with pytest.raises(sx.SxError):
        sx.sx_create((4, 4, 4), (1, 1, 1), [[1, 0, 0], [2, 0, 0], [0, 0, 1]], SC_POS, [1.0])
    with pytest.raises(sx.SxError):
        sx.sx_create((4, 4, 4), (1, 1, 1), cubic_cell(), SC_POS, [0.0])


def test_hamiltonian_argument_checks():
    c = _ctx()
    try:
        for bad in (lambda: sx.sx_add_shell_exchange(c, 0, 1.0), lambda: sx.sx_add_shell_exchange(c, 99, 1.0),
                    lambda: sx.sx_add_dmi(c, 1, 7, 1.0), lambda: sx.sx_add_bonds(c, [(0, 0, (0, 0, 0), np.eye(3))]),
                    lambda: sx.sx_add_bonds(c, [(0, 1, (1, 0, 0), np.eye(3))]),
                    lambda: sx.sx_add_bonds(c, [(0, 0, (5, 0, 0), np.eye(3))]),
                    lambda: sx.sx_set_anisotropy(c, 1, 1.0, (0, 0, 1)),
                    lambda: sx.sx_set_anisotropy(c, 0, 1.0, (0, 0, 0))):
            with pytest.raises(sx.SxError) as e:
                bad()
            assert e.value.code == sx.SX_ERR_ARG
        # device calls before a plan are refused without touching the GPU
        assert sx.lib().sx_field(c, None, None, sx.SX_PREC_FP64, None) == sx.SX_ERR_STATE
        assert sx.lib().sx_energy(c, None, None, None) == sx.SX_ERR_STATE
        # unsupported combinations are refused before any CUDA call
        with pytest.raises(sx.SxError) as e:
            sx.sx_plan(c, "gather", "bf16")
        assert e.value.code == sx.SX_ERR_UNSUPPORTED
        sx.sx_set_dipolar(c, True)
        with pytest.raises(sx.SxError) as e:
            sx.sx_plan(c, "gather", "fp32")
        assert e.value.code == sx.SX_ERR_UNSUPPORTED
    finally:
        sx.sx_destroy(c)


@pytest.mark.parametrize("pos,radii", [(SC_POS, [1, 2 ** 0.5, 3 ** 0.5, 2]),
                                       (BCC_POS, [3 ** 0.5 / 2, 1, 2 ** 0.5, 11 ** 0.5 / 2])])
def test_shell_radii(pos, radii):
    c = sx.sx_create((4, 4, 4), (1, 1, 1), cubic_cell(1.0), pos, [1.0] * len(pos))
    try:
        got = [sx.sx_shell_radius(c, k + 1) for k in range(4)]
        assert np.allclose(got, radii, rtol=0, atol=1e-12)
    finally:
        sx.sx_destroy(c)


def _taps_vs_oracle(name, n, extra_lib, extra_orc, **override):
    s, w = sx.system_from_workload(name, n, **override)
    extra_lib(s)
    m, _ = oracle_model(name, n, build=False, **override)
    extra_orc(m)
    m.build()
    nx, ny, nz = n
    for a in range(s.nsub):
        taps = s.taps(a)
        i = ((a * nz + nz // 2) * ny + ny // 2) * nx + nx // 2   # an interior site
        jj, JJ = m.site_pairs(i)
        expect = {}
        for j, J in zip(jj, JJ):
            b, rem = divmod(int(j), nz * ny * nx)
            z, rem = divmod(rem, ny * nx)
            y, x = divmod(rem, nx)
            expect[(b, x - nx // 2, y - ny // 2, z - nz // 2)] = J
        got = {(b,) + tuple(d): np.array(J) for b, d, J in taps}
        assert set(got) == set(expect)
        for k in got:
            assert np.abs(got[k] - expect[k]).max() < 1e-13


def test_taps_match_oracle_pairs_bcc_dmi_bonds():
    rng = np.random.default_rng(3)
    J1 = rng.normal(size=(3, 3))
    J2 = rng.normal(size=(3, 3))

    def lib_extra(s):
        s.add_dmi(2, sx.SX_DMI_BULK, 0.3)
        s.add_dmi(3, sx.SX_DMI_INTERFACIAL, -0.2)
        s.add_bonds([(0, 1, (1, -1, 0), J1), (1, 1, (0, 2, -1), J2)])

    def orc_extra(m):
        m.add_dmi(2, 1, 0.3)
        m.add_dmi(3, 0, -0.2)
        m.add_bond(0, 1, (1, -1, 0), J1)
        m.add_bond(1, 1, (0, 2, -1), J2)

    _taps_vs_oracle("bcc_4shell", (11, 10, 9), lib_extra, orc_extra)


def test_taps_match_oracle_pairs_sc_dmi():
    _taps_vs_oracle("sc_j123_dmi", (9, 9, 9), lambda s: None, lambda m: None)


def test_tap_counts():
    s, _ = sx.system_from_workload("bcc_4shell", (8, 8, 8))
    assert len(s.taps(0)) == 50 and len(s.taps(1)) == 50
    s2, _ = sx.system_from_workload("sc_j123", (8, 8, 8))
    assert len(s2.taps(0)) == 26
    s3, _ = sx.system_from_workload("sc_j123_dmi", (8, 8, 8))
    assert len(s3.taps(0)) == 26


def test_proposer_size_and_argument_checks():
    L = sx.lib()
    assert L.sx_cnn_num_params() == 19491
    h = ctypes.c_void_p()
    for n, mb in (((0, 4, 4), 1), ((4, 4, 5000), 1), ((4, 4, 4), 0), ((4, 4, 4), 65536)):
        rc = L.sx_cnn_create(ctypes.byref(h), (ctypes.c_int * 3)(*n), mb)
        assert rc == sx.SX_ERR_ARG and not h.value
    assert L.sx_cnn_adam_step(None, None, None, None) == sx.SX_ERR_ARG
    assert L.sx_cnn_interpolate(None, None, 5, None) == sx.SX_ERR_ARG
    L.sx_cnn_destroy(None)
