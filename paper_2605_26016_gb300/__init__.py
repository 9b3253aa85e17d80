"""Thin Python binding of the GB300 atomistic spin library (include/sx.h).

Every function here only marshals arguments for the C ABI of libsx.so; all
computation happens in the library's CUDA kernels.  PyTorch supplies device
memory and streams.  Importing works without a GPU; the library must have been
built (``python -m paper_2605_26016_gb300.build`` or ``__graft_entry__.build()``)
and there is no fallback: calls fail loudly if libsx.so is missing.

Spin fields are float64 CUDA tensors of shape (3, nsub, nz, ny, nx) (or any
contiguous tensor with 3*nsite elements in that order).
"""
import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libsx.so")

SX_OK, SX_ERR_ARG, SX_ERR_UNSUPPORTED, SX_ERR_OOM, SX_ERR_CUDA, SX_ERR_TIMEOUT, SX_ERR_NUMERIC, SX_ERR_STATE = \
    0, -1, -2, -3, -4, -5, -6, -7
SX_BACKEND_GATHER, SX_BACKEND_STENCIL, SX_BACKEND_IGEMM_TC, SX_BACKEND_FFT = 0, 1, 2, 3
SX_PREC_FP64, SX_PREC_FP32, SX_PREC_TF32, SX_PREC_BF16 = 0, 1, 2, 3
SX_DMI_INTERFACIAL, SX_DMI_BULK = 0, 1
SX_MAX_SUB = 8

BACKENDS = {"gather": SX_BACKEND_GATHER, "stencil": SX_BACKEND_STENCIL, "igemm_tc": SX_BACKEND_IGEMM_TC,
            "fft": SX_BACKEND_FFT}
PRECISIONS = {"fp64": SX_PREC_FP64, "fp32": SX_PREC_FP32, "tf32": SX_PREC_TF32, "bf16": SX_PREC_BF16}

# names exported by libsx.so, exactly the functions declared in include/sx.h
EXPORTS = ("sx_create", "sx_destroy", "sx_last_error", "sx_num_shells", "sx_shell_radius", "sx_add_shell_exchange",
           "sx_add_dmi", "sx_add_bonds", "sx_set_zeeman", "sx_set_anisotropy", "sx_set_dipolar", "sx_get_taps",
           "sx_plan", "sx_field", "sx_llg_heun_step", "sx_llg_heun_step_out", "sx_llg_heun_host", "sx_energy", "sx_torque_max",
           "sx_thermal_normals", "sx_plan_info", "sx_torque_max_noalloc", "sx_minimise", "sx_path_step",
           "sx_geodesic", "sx_set_stencil_scheme", "sx_autotune", "sx_plan_tiles", "sx_set_tiles", "sx_device_status",
           "sx_batch_create", "sx_batch_destroy", "sx_batch_heun_step", "sx_batch_create_with_images",
           "sx_batch_bind", "sx_batch_run", "sx_batch_status", "sx_batch_info",
           "sx_cnn_num_params", "sx_cnn_create", "sx_cnn_destroy", "sx_cnn_set_params", "sx_cnn_get_params",
           "sx_cnn_pack", "sx_cnn_forward", "sx_cnn_loss_grad", "sx_cnn_adam_step", "sx_cnn_interpolate",
           "sx_cnn_propose")
SX_STENCIL_AUTO, SX_STENCIL_FUSED, SX_STENCIL_TWO_PASS = 0, 1, 2
STENCIL_SCHEMES = {"auto": SX_STENCIL_AUTO, "fused": SX_STENCIL_FUSED, "two_pass": SX_STENCIL_TWO_PASS}
SX_MIN_VP, SX_MIN_DAMPED_LLG = 0, 1
SX_PATH_STRING, SX_PATH_GNEB, SX_PATH_CI_GNEB = 0, 1, 2
PATH_METHODS = {"string": SX_PATH_STRING, "gneb": SX_PATH_GNEB, "ci_gneb": SX_PATH_CI_GNEB}
SX_PATH_STEEPEST, SX_PATH_VP = 0, 1
PATH_OPTIMIZERS = {"steepest": SX_PATH_STEEPEST, "vp": SX_PATH_VP}


class sx_lattice(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("pbc", ctypes.c_int * 3), ("a", (ctypes.c_double * 3) * 3),
                ("nsub", ctypes.c_int), ("sub_pos", (ctypes.c_double * 3) * SX_MAX_SUB),
                ("mu", ctypes.c_double * SX_MAX_SUB)]


class sx_bond(ctypes.Structure):
    _fields_ = [("a", ctypes.c_int), ("b", ctypes.c_int), ("d", ctypes.c_int * 3), ("J", ctypes.c_double * 9)]


sx_tap = sx_bond


class sx_llg_params(ctypes.Structure):
    _fields_ = [("dt_fs", ctypes.c_double), ("alpha", ctypes.c_double), ("T_kelvin", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("replica", ctypes.c_uint32)]


class sx_min_params(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("dt", ctypes.c_double), ("alpha", ctypes.c_double), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("check_every", ctypes.c_int)]


class sx_path_params(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("dt", ctypes.c_double), ("k_spring", ctypes.c_double),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("check_every", ctypes.c_int),
                ("optimizer", ctypes.c_int), ("keep_velocity", ctypes.c_int)]


class sx_adam_params(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double)]


class SxError(RuntimeError):
    def __init__(self, code, fn, msg):
        super().__init__(f"{fn} failed ({code}): {msg}")
        self.code = code


_lib = None


def lib():
    """Load libsx.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2605_26016_gb300.build`")
        try:  # share the CUDA runtime torch already loaded
            import torch  # noqa: F401
        except ImportError:
            pass
        L = ctypes.CDLL(LIB_PATH)
        vp, dp, i64 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64
        sig = {
            "sx_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.POINTER(sx_lattice)]),
            "sx_destroy": (None, [vp]),
            "sx_last_error": (ctypes.c_char_p, []),
            "sx_num_shells": (ctypes.c_int, [vp]),
            "sx_shell_radius": (ctypes.c_double, [vp, ctypes.c_int]),
            "sx_add_shell_exchange": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_double]),
            "sx_add_dmi": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_double]),
            "sx_add_bonds": (ctypes.c_int, [vp, ctypes.POINTER(sx_bond), ctypes.c_size_t]),
            "sx_set_zeeman": (ctypes.c_int, [vp, dp]),
            "sx_set_anisotropy": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_double, dp]),
            "sx_set_dipolar": (ctypes.c_int, [vp, ctypes.c_int]),
            "sx_get_taps": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(sx_tap), ctypes.c_int]),
            "sx_plan": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int]),
            "sx_field": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, vp]),
            "sx_llg_heun_step": (ctypes.c_int, [vp, vp, vp, ctypes.POINTER(sx_llg_params), ctypes.c_uint64,
                                                ctypes.c_int, vp]),
            "sx_llg_heun_step_out": (ctypes.c_int, [vp, vp, vp, ctypes.POINTER(sx_llg_params), ctypes.c_uint64, vp]),
            "sx_llg_heun_host": (ctypes.c_int, [vp, vp, ctypes.POINTER(sx_llg_params), ctypes.c_uint64,
                                                ctypes.c_int, vp]),
            "sx_energy": (ctypes.c_int, [vp, vp, dp, vp]),
            "sx_torque_max": (ctypes.c_int, [vp, vp, dp, vp]),
            "sx_thermal_normals": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, i64,
                                                  ctypes.c_uint64, vp, vp]),
            "sx_plan_info": (ctypes.c_int, [vp, ctypes.POINTER(i64)]),
            "sx_torque_max_noalloc": (ctypes.c_int, [vp, vp, i64, dp, vp]),
            "sx_minimise": (ctypes.c_int, [vp, vp, vp, ctypes.POINTER(sx_min_params), ctypes.POINTER(ctypes.c_int),
                                           dp, vp]),
            "sx_path_step": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.POINTER(sx_path_params),
                                            ctypes.POINTER(ctypes.c_int), dp, dp, vp]),
            "sx_geodesic": (ctypes.c_int, [vp, vp, vp, dp, vp]),
            "sx_set_stencil_scheme": (ctypes.c_int, [vp, ctypes.c_int]),
            "sx_device_status": (ctypes.c_int, [vp, vp]),
            "sx_batch_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_int]),
            "sx_batch_destroy": (None, [vp]),
            "sx_batch_heun_step": (ctypes.c_int, [vp, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                                  ctypes.POINTER(sx_llg_params), ctypes.c_uint64, vp]),
            "sx_batch_create_with_images": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_int, vp,
                                                           ctypes.c_int]),
            "sx_batch_bind": (ctypes.c_int, [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp, vp, ctypes.c_uint32]),
            "sx_batch_run": (ctypes.c_int, [vp, ctypes.POINTER(sx_llg_params), ctypes.c_uint64, ctypes.c_int, vp]),
            "sx_batch_status": (ctypes.c_int, [vp, vp]),
            "sx_batch_info": (ctypes.c_int, [vp, ctypes.POINTER(i64)]),
            "sx_autotune": (ctypes.c_int, [vp, vp, vp, ctypes.POINTER(sx_llg_params), ctypes.c_int, dp, vp]),
            "sx_plan_tiles": (ctypes.c_int, [vp, ctypes.POINTER(i64)]),
            "sx_set_tiles": (ctypes.c_int, [vp, ctypes.POINTER(i64)]),
            "sx_cnn_num_params": (i64, []),
            "sx_cnn_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
            "sx_cnn_destroy": (None, [vp]),
            "sx_cnn_set_params": (ctypes.c_int, [vp, vp]),
            "sx_cnn_get_params": (ctypes.c_int, [vp, vp]),
            "sx_cnn_pack": (ctypes.c_int, [vp, vp, i64, vp, vp, i64, vp, ctypes.c_int, vp, vp]),
            "sx_cnn_forward": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, vp, vp]),
            "sx_cnn_loss_grad": (ctypes.c_int, [vp, vp, vp, vp, ctypes.c_int, vp, dp, vp]),
            "sx_cnn_adam_step": (ctypes.c_int, [vp, vp, ctypes.POINTER(sx_adam_params), vp]),
            "sx_cnn_interpolate": (ctypes.c_int, [vp, vp, ctypes.c_int, vp]),
            "sx_cnn_propose": (ctypes.c_int, [vp, vp, ctypes.c_int, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def last_error():
    return lib().sx_last_error().decode(errors="replace")


def _chk(rc, fn):
    if rc != SX_OK:
        raise SxError(rc, fn, last_error())
    return rc


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, nelem, dtype_name="float64"):
    if not t.is_cuda or not t.is_contiguous() or str(t.dtype) != "torch." + dtype_name or t.numel() != nelem:
        raise ValueError(f"expected a contiguous CUDA {dtype_name} tensor with {nelem} elements")
    return ctypes.c_void_p(t.data_ptr())


def _dbl3(v):
    return (ctypes.c_double * 3)(*[float(x) for x in v])


def make_lattice(n, pbc, cell, pos, mu):
    L = sx_lattice()
    for k in range(3):
        L.n[k] = int(n[k])
        L.pbc[k] = 1 if pbc[k] else 0
        for j in range(3):
            L.a[k][j] = float(cell[k][j])
    L.nsub = len(pos)
    for s, p in enumerate(pos):
        for j in range(3):
            L.sub_pos[s][j] = float(p[j])
        L.mu[s] = float(mu[s])
    return L


# ---------------------------------------------------------------- C-ABI mirrors

def sx_create(n, pbc, cell, pos, mu):
    h = ctypes.c_void_p()
    L = make_lattice(n, pbc, cell, pos, mu)
    _chk(lib().sx_create(ctypes.byref(h), ctypes.byref(L)), "sx_create")
    return h


def sx_destroy(ctx):
    if ctx is not None and ctx.value:
        lib().sx_destroy(ctx)


def sx_num_shells(ctx):
    return lib().sx_num_shells(ctx)


def sx_shell_radius(ctx, shell):
    return lib().sx_shell_radius(ctx, int(shell))


def sx_add_shell_exchange(ctx, shell, J):
    return _chk(lib().sx_add_shell_exchange(ctx, int(shell), float(J)), "sx_add_shell_exchange")


def sx_add_dmi(ctx, shell, kind, D):
    return _chk(lib().sx_add_dmi(ctx, int(shell), int(kind), float(D)), "sx_add_dmi")


def sx_add_bonds(ctx, bonds):
    """bonds: iterable of (a, b, (dx, dy, dz), J 3x3)."""
    bonds = list(bonds)
    arr = (sx_bond * max(1, len(bonds)))()
    for i, (a, b, d, J) in enumerate(bonds):
        arr[i].a, arr[i].b = int(a), int(b)
        for k in range(3):
            arr[i].d[k] = int(d[k])
        flat = [float(x) for row in J for x in row]
        for k in range(9):
            arr[i].J[k] = flat[k]
    return _chk(lib().sx_add_bonds(ctx, arr, len(bonds)), "sx_add_bonds")


def sx_set_zeeman(ctx, B):
    return _chk(lib().sx_set_zeeman(ctx, _dbl3(B)), "sx_set_zeeman")


def sx_set_anisotropy(ctx, sub, K, axis):
    return _chk(lib().sx_set_anisotropy(ctx, int(sub), float(K), _dbl3(axis)), "sx_set_anisotropy")


def sx_set_dipolar(ctx, enable):
    return _chk(lib().sx_set_dipolar(ctx, 1 if enable else 0), "sx_set_dipolar")


def sx_get_taps(ctx, a):
    n = lib().sx_get_taps(ctx, int(a), None, 0)
    if n < 0:
        raise SxError(n, "sx_get_taps", last_error())
    arr = (sx_tap * max(1, n))()
    _ = lib().sx_get_taps(ctx, int(a), arr, n)
    return [(t.b, tuple(t.d), [list(t.J[0:3]), list(t.J[3:6]), list(t.J[6:9])]) for t in arr[:n]]


def sx_plan(ctx, backend, precision):
    b = BACKENDS.get(backend, backend)
    p = PRECISIONS.get(precision, precision)
    return _chk(lib().sx_plan(ctx, int(b), int(p)), "sx_plan")


def sx_plan_info(ctx):
    out = (ctypes.c_int64 * 8)()
    _chk(lib().sx_plan_info(ctx, out), "sx_plan_info")
    keys = ("nsite", "max_taps", "rx", "ry", "rz", "backend", "precision", "launches_per_step")
    return dict(zip(keys, list(out)))


def llg_params(dt_fs, alpha, T=0.0, seed=0, replica=0):
    p = sx_llg_params()
    p.dt_fs, p.alpha, p.T_kelvin, p.seed, p.replica = float(dt_fs), float(alpha), float(T), int(seed), int(replica)
    return p


def sx_field(ctx, S, b, nsite, stream=None):
    """The field of S into b: a float64 tensor (FP64 output) or a float32 tensor (FP32 output)."""
    fp32 = str(b.dtype) == "torch.float32"
    return _chk(lib().sx_field(ctx, _dev_ptr(S, 3 * nsite), _dev_ptr(b, 3 * nsite, "float32" if fp32 else "float64"),
                               SX_PREC_FP32 if fp32 else SX_PREC_FP64, _stream(stream)), "sx_field")


def sx_llg_heun_step(ctx, S, S_scratch, params, step0, nsteps, nsite, stream=None):
    return _chk(lib().sx_llg_heun_step(ctx, _dev_ptr(S, 3 * nsite), _dev_ptr(S_scratch, 3 * nsite),
                                       ctypes.byref(params), int(step0), int(nsteps), _stream(stream)),
                "sx_llg_heun_step")


def sx_llg_heun_step_out(ctx, S_in, S_out, params, step, nsite, stream=None):
    return _chk(lib().sx_llg_heun_step_out(ctx, _dev_ptr(S_in, 3 * nsite), _dev_ptr(S_out, 3 * nsite),
                                           ctypes.byref(params), int(step), _stream(stream)), "sx_llg_heun_step_out")


def sx_llg_heun_host(ctx, S_host, params, step0, nsteps, nsite, stream=None):
    """S_host: contiguous float64 CPU torch tensor (pinned for full bandwidth) or numpy array."""
    if hasattr(S_host, "data_ptr"):
        if S_host.is_cuda or not S_host.is_contiguous() or S_host.numel() != 3 * nsite:
            raise ValueError("S_host must be a contiguous CPU tensor with 3*nsite elements")
        ptr = ctypes.c_void_p(S_host.data_ptr())
    else:
        if S_host.size != 3 * nsite or not S_host.flags["C_CONTIGUOUS"]:
            raise ValueError("S_host must be a contiguous array with 3*nsite elements")
        ptr = ctypes.c_void_p(S_host.ctypes.data)
    return _chk(lib().sx_llg_heun_host(ctx, ptr, ctypes.byref(params), int(step0), int(nsteps), _stream(stream)),
                "sx_llg_heun_host")


def sx_energy(ctx, S, nsite, stream=None):
    out = (ctypes.c_double * 5)()
    _chk(lib().sx_energy(ctx, _dev_ptr(S, 3 * nsite), out, _stream(stream)), "sx_energy")
    return {"total": out[0], "bilinear": out[1], "zeeman": out[2], "anisotropy": out[3], "dipolar": out[4]}


def sx_torque_max(ctx, S, nsite, stream=None):
    out = ctypes.c_double()
    _chk(lib().sx_torque_max(ctx, _dev_ptr(S, 3 * nsite), ctypes.byref(out), _stream(stream)), "sx_torque_max")
    return out.value


def sx_torque_max_noalloc(S, b, nsite, stream=None):
    """max_i |S_i x b_i| for caller-provided spins and fields; the library allocates nothing for it
    (scratch lives in a fixed array in the library image)."""
    out = ctypes.c_double()
    _chk(lib().sx_torque_max_noalloc(_dev_ptr(S, 3 * nsite), _dev_ptr(b, 3 * nsite), int(nsite), ctypes.byref(out),
                                     _stream(stream)), "sx_torque_max_noalloc")
    return out.value


def sx_minimise(ctx, S, S_scratch, nsite, method="vp", dt=0.05, alpha=1.0, tol=1e-8, max_iter=1000, check_every=50,
                stream=None):
    """Minimise in place; returns (iterations, last measured max |S x b| in meV)."""
    p = sx_min_params()
    p.method = {"vp": SX_MIN_VP, "damped_llg": SX_MIN_DAMPED_LLG}.get(method, method)
    p.dt, p.alpha, p.tol, p.max_iter, p.check_every = float(dt), float(alpha), float(tol), int(max_iter), int(check_every)
    it = ctypes.c_int()
    tq = ctypes.c_double()
    _chk(lib().sx_minimise(ctx, _dev_ptr(S, 3 * nsite), _dev_ptr(S_scratch, 3 * nsite), ctypes.byref(p),
                           ctypes.byref(it), ctypes.byref(tq), _stream(stream)), "sx_minimise")
    return it.value, tq.value


def sx_path_step(ctx, images, nimg, nsite, method="gneb", dt=0.05, k_spring=1.0, tol=0.0, max_iter=100,
                 check_every=50, optimizer="steepest", keep_velocity=False, stream=None):
    """Path-method iterations on a chain (nimg images back to back, in place; endpoints fixed).
    Returns (iterations, image energies in meV as a list, largest site force of the last measured
    iteration in meV)."""
    p = sx_path_params()
    p.method = PATH_METHODS.get(method, method)
    p.dt, p.k_spring, p.tol = float(dt), float(k_spring), float(tol)
    p.max_iter, p.check_every = int(max_iter), int(check_every)
    p.optimizer = PATH_OPTIMIZERS.get(optimizer, optimizer)
    p.keep_velocity = 1 if keep_velocity else 0
    it = ctypes.c_int()
    E = (ctypes.c_double * max(1, int(nimg)))()
    fm = ctypes.c_double()
    _chk(lib().sx_path_step(ctx, _dev_ptr(images, 3 * nsite * int(nimg)), int(nimg), ctypes.byref(p),
                            ctypes.byref(it), E, ctypes.byref(fm), _stream(stream)), "sx_path_step")
    return it.value, [E[i] for i in range(int(nimg))], fm.value


def sx_geodesic(ctx, A, B, nsite, stream=None):
    """Geodesic distance between two spin fields (FP64)."""
    out = ctypes.c_double()
    _chk(lib().sx_geodesic(ctx, _dev_ptr(A, 3 * nsite), _dev_ptr(B, 3 * nsite), ctypes.byref(out),
                           _stream(stream)), "sx_geodesic")
    return out.value


class Batch:
    """Replicas sharing one Hamiltonian (SpinSystem objects with stencil plans), advanced together by
    sx_batch_heun_step, and optionally nimg images of `image_system`'s lattice whose fields sx_batch_run
    evaluates in the same launch.  Keeps the systems (and the buffers given to bind) alive while it exists."""

    def __init__(self, systems, image_system=None, nimg=0):
        self.systems = list(systems)
        self.image_system = image_system
        self.nimg = nimg if image_system is not None else 0
        arr = (ctypes.c_void_p * len(self.systems))(*[s.ctx for s in self.systems])
        h = ctypes.c_void_p()
        if image_system is None:
            _chk(lib().sx_batch_create(ctypes.byref(h), arr, len(self.systems)), "sx_batch_create")
        else:
            _chk(lib().sx_batch_create_with_images(ctypes.byref(h), arr, len(self.systems), image_system.ctx, int(nimg)),
                 "sx_batch_create_with_images")
        self.h = h
        self._bound = None

    def close(self):
        if getattr(self, "h", None):
            lib().sx_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def bind(self, S_a, S_b, images=None, fields=None, replica0=0):
        """Device buffers of run(): replica r alternates between S_a[r] and S_b[r]; images (nimg x 3 x
        nsite of the image system, float64) in, their FP64 fields out."""
        n = len(self.systems)
        a = (ctypes.c_void_p * n)(*[_dev_ptr(x, 3 * s.nsite).value for x, s in zip(S_a, self.systems)])
        b = (ctypes.c_void_p * n)(*[_dev_ptr(x, 3 * s.nsite).value for x, s in zip(S_b, self.systems)])
        ip = fp = None
        if self.nimg:
            m = self.nimg * 3 * self.image_system.nsite
            ip, fp = _dev_ptr(images, m), _dev_ptr(fields, m)
        _chk(lib().sx_batch_bind(self.h, a, b, ip, fp, int(replica0)), "sx_batch_bind")
        self._bound = (list(S_a), list(S_b), images, fields)

    def run(self, params, step0, nsteps, stream=None):
        return _chk(lib().sx_batch_run(self.h, ctypes.byref(params), int(step0), int(nsteps), _stream(stream)),
                    "sx_batch_run")

    def status(self, stream=None):
        return _chk(lib().sx_batch_status(self.h, _stream(stream)), "sx_batch_status")

    def info(self):
        out = (ctypes.c_int64 * 4)()
        _chk(lib().sx_batch_info(self.h, out), "sx_batch_info")
        return {"replicas": out[0], "images": out[1], "persistent": bool(out[2])}

    def heun_step(self, S_in, S_out, params, step, stream=None):
        n = len(self.systems)
        a = (ctypes.c_void_p * n)(*[_dev_ptr(x, 3 * s.nsite).value for x, s in zip(S_in, self.systems)])
        b = (ctypes.c_void_p * n)(*[_dev_ptr(x, 3 * s.nsite).value for x, s in zip(S_out, self.systems)])
        return _chk(lib().sx_batch_heun_step(self.h, a, b, ctypes.byref(params), int(step), _stream(stream)),
                    "sx_batch_heun_step")


def sx_device_status(ctx, stream=None):
    """Synchronise and raise SxError(SX_ERR_TIMEOUT) if a bounded device wait gave up since the last check."""
    return _chk(lib().sx_device_status(ctx, _stream(stream)), "sx_device_status")


def sx_set_stencil_scheme(ctx, scheme):
    """Choose the stencil Heun scheme ("auto", "fused" or "two_pass")."""
    return _chk(lib().sx_set_stencil_scheme(ctx, STENCIL_SCHEMES.get(scheme, scheme)), "sx_set_stencil_scheme")


def sx_autotune(ctx, S, S_scratch, p, nsite, steps=5, stream=None):
    """Time the plan's candidate tile shapes on S (unchanged) and keep the fastest; returns
    (chosen scheme name, {"fused": ms, "two_pass": ms}) -- for a tensor-core plan "fused" holds the best time."""
    t = (ctypes.c_double * 2)()
    rc = lib().sx_autotune(ctx, _dev_ptr(S, 3 * nsite), _dev_ptr(S_scratch, 3 * nsite), ctypes.byref(p), int(steps),
                           t, _stream(stream))
    if rc < 0:
        _chk(rc, "sx_autotune")
    name = {v: k for k, v in STENCIL_SCHEMES.items()}[rc]
    return name, {"fused": t[0], "two_pass": t[1]}


def sx_set_tiles(ctx, scheme, zchunk_or_ring, sched_or_ctas=0, regen_noise=0, tma_staging=None):
    """Set the tile shape (see include/sx.h): stencil (scheme, z chunk, two-pass launch shape, regenerate
    normals, plane-staging mask: bit 0 predictor and field passes, bit 1 corrector use tensor copies) or tensor
    core (0, ring depth, CTAs per SM, 0, 0); scheme may be "fused" / "two_pass".  tma_staging None keeps the
    plan's current staging."""
    if tma_staging is None:
        tma_staging = sx_plan_tiles(ctx)["tma_staging"]
    v = (ctypes.c_int64 * 5)(STENCIL_SCHEMES.get(scheme, scheme), int(zchunk_or_ring), int(sched_or_ctas),
                             int(regen_noise), int(tma_staging))
    return _chk(lib().sx_set_tiles(ctx, v), "sx_set_tiles")


def sx_plan_tiles(ctx):
    out = (ctypes.c_int64 * 8)()
    _chk(lib().sx_plan_tiles(ctx, out), "sx_plan_tiles")
    keys = ("scheme", "tile_x", "tile_y", "tile_z", "ctas", "ring_or_schedule", "regen_noise", "tma_staging")
    return dict(zip(keys, list(out)))


def sx_thermal_normals(seed, replica, site0, n, step, eta, stream=None):
    return _chk(lib().sx_thermal_normals(int(seed), int(replica), int(site0), int(n), int(step),
                                         _dev_ptr(eta, 3 * n, "float32"), _stream(stream)), "sx_thermal_normals")


class Proposer:
    """The convolutional chain proposer of include/sx.h (sx_cnn_*) for grids n = (nx, ny, nz) and batches of
    up to max_batch samples.  Images are float64 CUDA tensors with 3*ncell elements per sample ([c][z][y][x]);
    packed inputs are int16 CUDA tensors (BF16 bit patterns) of shape (nb, ncell, 16)."""

    def __init__(self, n, max_batch):
        self.n = tuple(int(v) for v in n)
        self.ncell = self.n[0] * self.n[1] * self.n[2]
        self.max_batch = int(max_batch)
        self.nparams = int(lib().sx_cnn_num_params())
        h = ctypes.c_void_p()
        _chk(lib().sx_cnn_create(ctypes.byref(h), (ctypes.c_int * 3)(*self.n), self.max_batch), "sx_cnn_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().sx_cnn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat):
        import numpy as np
        a = np.ascontiguousarray(flat, dtype=np.float32)
        if a.size != self.nparams:
            raise ValueError(f"expected {self.nparams} parameters")
        return _chk(lib().sx_cnn_set_params(self.h, a.ctypes.data_as(ctypes.c_void_p)), "sx_cnn_set_params")

    def get_params(self):
        import numpy as np
        a = np.empty(self.nparams, dtype=np.float32)
        _chk(lib().sx_cnn_get_params(self.h, a.ctypes.data_as(ctypes.c_void_p)), "sx_cnn_get_params")
        return a

    def new_packed(self, nb):
        import torch
        return torch.empty((nb, self.ncell, 16), dtype=torch.int16, device="cuda")

    def pack(self, I, A, B, s, X, shared_endpoints=False, stream=None):
        """X <- packed samples (I[b], A[b], B[b], s[b]); with shared_endpoints A and B are single images."""
        nb = X.shape[0]
        m = 3 * self.ncell
        ab = m if not shared_endpoints else 0
        return _chk(lib().sx_cnn_pack(self.h, _dev_ptr(I, nb * m), m, _dev_ptr(A, m if shared_endpoints else nb * m),
                                      _dev_ptr(B, m if shared_endpoints else nb * m), ab, _dev_ptr(s, nb),
                                      nb, _dev_ptr(X, nb * self.ncell * 16, "int16"), _stream(stream)), "sx_cnn_pack")

    def forward(self, X, I, P, stream=None):
        nb = X.shape[0]
        m = 3 * self.ncell
        return _chk(lib().sx_cnn_forward(self.h, _dev_ptr(X, nb * self.ncell * 16, "int16"), _dev_ptr(I, nb * m), nb,
                                         _dev_ptr(P, nb * m), _stream(stream)), "sx_cnn_forward")

    def loss_grad(self, X, I, T, grad=None, stream=None):
        """Returns the loss; the gradient goes to grad (float32 CUDA tensor) or stays in the proposer."""
        nb = X.shape[0]
        m = 3 * self.ncell
        loss = ctypes.c_double()
        g = _dev_ptr(grad, self.nparams, "float32") if grad is not None else None
        _chk(lib().sx_cnn_loss_grad(self.h, _dev_ptr(X, nb * self.ncell * 16, "int16"), _dev_ptr(I, nb * m),
                                    _dev_ptr(T, nb * m), nb, g, ctypes.byref(loss), _stream(stream)),
             "sx_cnn_loss_grad")
        return loss.value

    def adam_step(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, grad=None, stream=None):
        p = sx_adam_params(lr, beta1, beta2, eps)
        g = _dev_ptr(grad, self.nparams, "float32") if grad is not None else None
        return _chk(lib().sx_cnn_adam_step(self.h, g, ctypes.byref(p), _stream(stream)), "sx_cnn_adam_step")

    def interpolate(self, chain, stream=None):
        nimg = chain.shape[0]
        return _chk(lib().sx_cnn_interpolate(self.h, _dev_ptr(chain, nimg * 3 * self.ncell), nimg, _stream(stream)),
                    "sx_cnn_interpolate")

    def propose(self, chain, stream=None):
        nimg = chain.shape[0]
        return _chk(lib().sx_cnn_propose(self.h, _dev_ptr(chain, nimg * 3 * self.ncell), nimg, _stream(stream)),
                    "sx_cnn_propose")


# ---------------------------------------------------------------- convenience

class SpinSystem:
    """Owns one context.  Convenience over the sx_* functions above."""

    def __init__(self, n, pbc, cell, pos, mu):
        self.ctx = sx_create(n, pbc, cell, pos, mu)
        self.n = tuple(int(v) for v in n)
        self.nsub = len(pos)
        self.nsite = self.nsub * self.n[0] * self.n[1] * self.n[2]
        self.shape = (3, self.nsub, self.n[2], self.n[1], self.n[0])

    def close(self):
        if getattr(self, "ctx", None) is not None:
            sx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_shell_exchange(self, shell, J):
        sx_add_shell_exchange(self.ctx, shell, J)

    def add_dmi(self, shell, kind, D):
        sx_add_dmi(self.ctx, shell, kind, D)

    def add_bonds(self, bonds):
        sx_add_bonds(self.ctx, bonds)

    def set_zeeman(self, B):
        sx_set_zeeman(self.ctx, B)

    def set_anisotropy(self, sub, K, axis):
        sx_set_anisotropy(self.ctx, sub, K, axis)

    def set_dipolar(self, on):
        sx_set_dipolar(self.ctx, on)

    def taps(self, a):
        return sx_get_taps(self.ctx, a)

    def plan(self, backend="stencil", precision="fp32"):
        sx_plan(self.ctx, backend, precision)
        return sx_plan_info(self.ctx)

    def info(self):
        return sx_plan_info(self.ctx)

    def field(self, S, out=None, stream=None, dtype=None):
        """The field of S: into `out` (float64 or float32), else a new tensor of `dtype` (default float64)."""
        import torch
        if out is None:
            out = torch.empty_like(S, dtype=dtype or torch.float64)
        sx_field(self.ctx, S, out, self.nsite, stream)
        return out

    def heun(self, S, scratch, dt, alpha, T=0.0, seed=0, replica=0, step0=0, nsteps=1, stream=None):
        sx_llg_heun_step(self.ctx, S, scratch, llg_params(dt, alpha, T, seed, replica), step0, nsteps, self.nsite,
                         stream)
        return S

    def heun_host(self, S_host, dt, alpha, T=0.0, seed=0, replica=0, step0=0, nsteps=1, stream=None):
        sx_llg_heun_host(self.ctx, S_host, llg_params(dt, alpha, T, seed, replica), step0, nsteps, self.nsite, stream)
        return S_host

    def energy(self, S, stream=None):
        return sx_energy(self.ctx, S, self.nsite, stream)

    def minimise(self, S, scratch=None, stream=None, **kw):
        import torch
        if scratch is None:
            scratch = torch.empty_like(S)
        return sx_minimise(self.ctx, S, scratch, self.nsite, stream=stream, **kw)

    def torque_max(self, S, stream=None):
        return sx_torque_max(self.ctx, S, self.nsite, stream)

    def path(self, images, method="gneb", stream=None, **kw):
        """Path-method iterations on a chain tensor of shape (nimg, 3, nsub, nz, ny, nx), in place."""
        return sx_path_step(self.ctx, images, images.shape[0], self.nsite, method=method, stream=stream, **kw)

    def geodesic(self, A, B, stream=None):
        return sx_geodesic(self.ctx, A, B, self.nsite, stream)


def system_from_workload(workload, n, pbc=None, cell=None, **override):
    """SpinSystem (not yet planned) for a workload description: a dict with keys pos, mu, shells,
    dmi, B, K, pbc (see workloads.py at the repository root), or the name of one there."""
    if isinstance(workload, str):
        from workloads import WORKLOADS, cubic_cell
        w = dict(WORKLOADS[workload])
        cell = cell or cubic_cell()
    else:
        w = dict(workload)
    if cell is None:
        raise ValueError("cell vectors are required with a workload dict")
    w.update(override)
    s = SpinSystem(n, pbc if pbc is not None else w["pbc"], cell, w["pos"], w["mu"])
    for k, J in enumerate(w["shells"]):
        if J != 0.0:
            s.add_shell_exchange(k + 1, J)
    if w["dmi"]:
        shell, kind, D = w["dmi"]
        s.add_dmi(shell, kind, D)
    s.set_zeeman(w["B"])
    if w["K"]:
        K, axis = w["K"]
        for sub in range(len(w["pos"])):
            s.set_anisotropy(sub, K, axis)
    return s, w
