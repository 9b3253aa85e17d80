"""CPU FP64 oracle for the spin field, energy and Heun-LLG step (test infrastructure).

This package is test infrastructure: only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py`` may import it.  It wraps
``sx_oracle.c`` (plain C, FP64, OpenMP), which shares no code with the CUDA
library.  Every routine follows the Methods section of arXiv 2605.26016:

* pair list built by brute force over lattice translations, distance shells
  sorted by radius ("Hopfion calculation": couplings on neighbour shells);
* reduced field b_i = sum_p J_p S_{j_p} (pair-list equation, "Backend
  representations") plus Zeeman mu mu_B B and anisotropy 2K(S.n)n (derivatives
  of H_Z and H_ani, "Spin Hamiltonian and effective fields");
* energy in the ordered-pair form with the factor 1/2;
* normalised Heun predictor/corrector of the LLG equation ("Atomistic spin
  dynamics") with the thermal field sigma*eta ("Stochastic LLG simulations");
* Philox4x32-10 (Salmon et al., SC'11) + Box-Muller noise, written here.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sx_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")

_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_fp = ctypes.POINTER(ctypes.c_float)


def build(force=False):
    """Compile sx_oracle.c into liboracle.so next to it (gcc, OpenMP, no FP contraction)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", _SO + ".tmp", _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [_ip, _ip, _dp, ctypes.c_int, _dp, _dp]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_nshell.argtypes = [ctypes.c_void_p]
        L.orc_shell_radius.restype = ctypes.c_double
        L.orc_shell_radius.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_add_shell_exchange.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double]
        L.orc_add_dmi.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double]
        L.orc_add_bond.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _ip, _dp]
        L.orc_set_zeeman.argtypes = [ctypes.c_void_p, _dp]
        L.orc_set_anisotropy.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, _dp]
        L.orc_set_dipolar.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_build.argtypes = [ctypes.c_void_p]
        L.orc_npair.restype = ctypes.c_int64
        L.orc_npair.argtypes = [ctypes.c_void_p]
        L.orc_site_pairs.restype = ctypes.c_int64
        L.orc_site_pairs.argtypes = [ctypes.c_void_p, ctypes.c_int64, _i64p, _dp, ctypes.c_int64]
        L.orc_field.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.orc_field_sites.argtypes = [ctypes.c_void_p, _dp, _i64p, ctypes.c_int64, _dp]
        L.orc_energy.restype = ctypes.c_double
        L.orc_energy.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.orc_torque_max.restype = ctypes.c_double
        L.orc_torque_max.argtypes = [ctypes.c_void_p, _dp]
        L.orc_heun.argtypes = [ctypes.c_void_p, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                               ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64]
        L.orc_heun_sites.argtypes = [ctypes.c_void_p, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, _i64p, ctypes.c_int64, _dp]
        L.orc_vp.argtypes = [ctypes.c_void_p, _dp, ctypes.c_double, ctypes.c_int64, _dp, _dp, ctypes.c_int]
        L.orc_geodesic.restype = ctypes.c_double
        L.orc_geodesic.argtypes = [ctypes.c_int64, _dp, _dp]
        L.orc_gneb.argtypes = [ctypes.c_void_p, _dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                               ctypes.c_int64, _dp, _dp]
        L.orc_gneb_vp.argtypes = [ctypes.c_void_p, _dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                  ctypes.c_int64, _dp, _dp, _dp, _dp, ctypes.c_int]
        L.orc_string.argtypes = [ctypes.c_void_p, _dp, ctypes.c_int, ctypes.c_double, ctypes.c_int64, _dp, _dp]
        L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.orc_normals_block.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64,
                                        ctypes.c_uint64, _fp]
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_constants.argtypes = [_dp]
        _lib = L
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(t)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


class Model:
    """A lattice + Hamiltonian in the oracle.  Spins are float64 arrays of shape
    (3, nsub, nz, ny, nx) (component planes, x fastest)."""

    def __init__(self, n, pbc, A, pos, mu):
        L = lib()
        self.n = tuple(int(v) for v in n)
        self.nsub = len(pos)
        n_ = (ctypes.c_int * 3)(*self.n)
        p_ = (ctypes.c_int * 3)(*[1 if v else 0 for v in pbc])
        A_ = np.ascontiguousarray(np.asarray(A, dtype=np.float64).reshape(9))
        pos_ = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1))
        mu_ = np.ascontiguousarray(np.asarray(mu, dtype=np.float64).reshape(-1))
        self.h = L.orc_create(n_, p_, _ptr(A_, _dp), self.nsub, _ptr(pos_, _dp), _ptr(mu_, _dp))
        if not self.h:
            raise ValueError("oracle: bad lattice")
        self.nsite = self.nsub * self.n[0] * self.n[1] * self.n[2]
        self.shape = (3, self.nsub, self.n[2], self.n[1], self.n[0])

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_destroy(self.h)
            self.h = None

    # --- Hamiltonian ---
    def shell_radii(self, k):
        L = lib()
        return [L.orc_shell_radius(self.h, i) for i in range(k)]

    def add_shell_exchange(self, shell, J):
        _check(lib().orc_add_shell_exchange(self.h, int(shell), float(J)), "add_shell_exchange")

    def add_dmi(self, shell, kind, D):
        _check(lib().orc_add_dmi(self.h, int(shell), int(kind), float(D)), "add_dmi")

    def add_bond(self, a, b, d, J):
        d_ = (ctypes.c_int * 3)(*[int(v) for v in d])
        J_ = np.ascontiguousarray(np.asarray(J, dtype=np.float64).reshape(9))
        _check(lib().orc_add_bond(self.h, int(a), int(b), d_, _ptr(J_, _dp)), "add_bond")

    def set_zeeman(self, B):
        B_ = np.ascontiguousarray(np.asarray(B, dtype=np.float64))
        lib().orc_set_zeeman(self.h, _ptr(B_, _dp))

    def set_anisotropy(self, sub, K, axis):
        a_ = np.ascontiguousarray(np.asarray(axis, dtype=np.float64))
        _check(lib().orc_set_anisotropy(self.h, int(sub), float(K), _ptr(a_, _dp)), "set_anisotropy")

    def set_dipolar(self, on):
        lib().orc_set_dipolar(self.h, 1 if on else 0)

    def build(self):
        _check(lib().orc_build(self.h), "build")

    def npair(self):
        return lib().orc_npair(self.h)

    def site_pairs(self, i, cap=4096):
        jj = np.zeros(cap, dtype=np.int64)
        JJ = np.zeros((cap, 9), dtype=np.float64)
        c = lib().orc_site_pairs(self.h, int(i), _ptr(jj, _i64p), _ptr(JJ, _dp), cap)
        return jj[:c].copy(), JJ[:c].reshape(-1, 3, 3).copy()

    # --- evaluation ---
    def _spins(self, S):
        S = np.ascontiguousarray(np.asarray(S, dtype=np.float64))
        if S.size != 3 * self.nsite:
            raise ValueError("spin array has the wrong size")
        return S

    def field(self, S):
        S = self._spins(S)
        b = np.empty_like(S)
        _check(lib().orc_field(self.h, _ptr(S, _dp), _ptr(b, _dp)), "field")
        return b.reshape(self.shape)

    def field_sites(self, S, sites):
        S = self._spins(S)
        sites = np.ascontiguousarray(np.asarray(sites, dtype=np.int64))
        out = np.empty((len(sites), 3), dtype=np.float64)
        _check(lib().orc_field_sites(self.h, _ptr(S, _dp), _ptr(sites, _i64p), len(sites), _ptr(out, _dp)),
               "field_sites")
        return out

    def energy(self, S, terms=False):
        S = self._spins(S)
        t = np.zeros(4, dtype=np.float64)
        e = lib().orc_energy(self.h, _ptr(S, _dp), _ptr(t, _dp))
        return (e, t) if terms else e

    def torque_max(self, S):
        return lib().orc_torque_max(self.h, _ptr(self._spins(S), _dp))

    def heun_sites(self, S, sites, dt, alpha, T=0.0, seed=0, replica=0, step=0):
        """One Heun step evaluated at the given sites only: (len(sites), 3)."""
        S = self._spins(S)
        sites = np.ascontiguousarray(np.asarray(sites, dtype=np.int64))
        out = np.empty((len(sites), 3), dtype=np.float64)
        _check(lib().orc_heun_sites(self.h, _ptr(S, _dp), float(dt), float(alpha), float(T), int(seed), int(replica),
                                    int(step), _ptr(sites, _i64p), len(sites), _ptr(out, _dp)), "heun_sites")
        return out

    def vp(self, S, dt, niter, state=None):
        """Velocity-projection minimisation; returns (S, state) where state carries (v, f_prev)."""
        S = self._spins(S).copy()
        first = state is None
        if first:
            state = (np.zeros(3 * self.nsite), np.zeros(3 * self.nsite))
        v, fp = state
        _check(lib().orc_vp(self.h, _ptr(S, _dp), float(dt), int(niter), _ptr(v, _dp), _ptr(fp, _dp),
                            1 if first else 0), "vp")
        return S.reshape(self.shape), (v, fp)

    def _chain(self, images):
        img = np.ascontiguousarray(np.asarray(images, dtype=np.float64)).copy()
        if img.size % (3 * self.nsite) or img.size // (3 * self.nsite) < 3:
            raise ValueError("a chain needs at least 3 images of %d spins" % self.nsite)
        return img.reshape(-1, 3 * self.nsite)

    def gneb(self, images, dt, k, niter, climbing=False):
        """niter geodesic-NEB iterations (endpoints fixed); returns (images, energies, max force)."""
        img = self._chain(images)
        E = np.zeros(img.shape[0])
        fm = ctypes.c_double(0.0)
        _check(lib().orc_gneb(self.h, _ptr(img, _dp), img.shape[0], float(dt), float(k), 1 if climbing else 0,
                              int(niter), _ptr(E, _dp), ctypes.byref(fm)), "gneb")
        return img.reshape((img.shape[0],) + self.shape), E, fm.value

    def gneb_vp(self, images, dt, k, niter, climbing=False, state=None):
        """niter geodesic-NEB iterations with velocity projection on the chain's force; returns (images,
        energies, max force, state); pass the returned state back to continue with the same velocity."""
        img = self._chain(images)
        E = np.zeros(img.shape[0])
        fm = ctypes.c_double(0.0)
        first = state is None
        if first:
            state = (np.zeros(img.shape), np.zeros(img.shape))
        _check(lib().orc_gneb_vp(self.h, _ptr(img, _dp), img.shape[0], float(dt), float(k), 1 if climbing else 0,
                                 int(niter), _ptr(E, _dp), ctypes.byref(fm), _ptr(state[0], _dp),
                                 _ptr(state[1], _dp), 1 if first else 0), "gneb_vp")
        return img.reshape((img.shape[0],) + self.shape), E, fm.value, state

    def string(self, images, dt, niter):
        """niter string-method iterations (step, then equal-arc-length redistribution);
        returns (images, energies, max force)."""
        img = self._chain(images)
        E = np.zeros(img.shape[0])
        fm = ctypes.c_double(0.0)
        _check(lib().orc_string(self.h, _ptr(img, _dp), img.shape[0], float(dt), int(niter), _ptr(E, _dp),
                                ctypes.byref(fm)), "string")
        return img.reshape((img.shape[0],) + self.shape), E, fm.value

    def heun(self, S, dt, alpha, T=0.0, seed=0, replica=0, step0=0, nsteps=1):
        """Return a new spin array after nsteps normalised Heun steps."""
        S = self._spins(S).copy()
        _check(lib().orc_heun(self.h, _ptr(S, _dp), float(dt), float(alpha), float(T), int(seed), int(replica),
                              int(step0), int(nsteps)), "heun")
        return S.reshape(self.shape)


def geodesic(A, B):
    """Geodesic distance between two spin fields: sqrt(sum_i arccos^2(A_i . B_i))."""
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float64).reshape(3, -1))
    B = np.ascontiguousarray(np.asarray(B, dtype=np.float64).reshape(3, -1))
    if A.shape != B.shape:
        raise ValueError("spin fields differ in size")
    return lib().orc_geodesic(A.shape[1], _ptr(A, _dp), _ptr(B, _dp))


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [o[i] for i in range(4)]


def normals(seed, replica, site0, n, step):
    """(n, 3) float32 standard normals for sites site0 .. site0+n-1 at one step."""
    out = np.empty((n, 3), dtype=np.float32)
    lib().orc_normals_block(int(seed), int(replica), int(site0), int(n), int(step), _ptr(out, _fp))
    return out


def constants():
    out = np.zeros(4, dtype=np.float64)
    lib().orc_constants(_ptr(out, _dp))
    return {"mu_B": out[0], "gamma": out[1], "k_B": out[2], "dip_pref": out[3]}


def num_threads():
    return lib().orc_num_threads()
