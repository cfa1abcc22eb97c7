"""ctypes binding of libddlpb.so (argument marshalling only).

Every computation runs in the CUDA library; this module converts Python
arguments to the C ABI declared in include/ddlpb.h and back.  Device buffers
are PyTorch CUDA tensors (plumbing only).  If the library has not been built,
importing works but every call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libddlpb.so")

DDLPB_VDW, DDLPB_SAS = 0, 1
DDLPB_FP64, DDLPB_MIXED = 0, 1
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ENOTCONV", 4: "ECUDA", 5: "EORDER"}

# Operators of ddlpb_apply_device
OP_L, OP_LT, OP_AB, OP_ABT, OP_C, OP_CT = range(6)
OP_FP32 = 8          # added to an op code: the FP32 operators of the mixed-precision form
OP_AB_F16, OP_ABT_F16 = 16, 17   # A/B and transpose as the mixed-precision preconditioner applies them


class Options(C.Structure):
    _fields_ = [("eta", C.c_double), ("tol", C.c_double), ("max_iter", C.c_int), ("gmres_restart", C.c_int),
                ("precision", C.c_int), ("fmm_order", C.c_int), ("cuda_stream", C.c_void_p),
                ("precond_tol", C.c_double), ("kernel_timing", C.c_int), ("precond_coupling", C.c_int),
                ("precond_fp16", C.c_int), ("fmm_theta", C.c_double)]


class Info(C.Structure):
    _fields_ = [("n_atoms", C.c_int), ("lmax", C.c_int), ("n_lebedev", C.c_int),
                ("n_neighbour_pairs", C.c_longlong), ("n_hits", C.c_longlong), ("n_external", C.c_longlong),
                ("solve_iterations", C.c_int), ("adjoint_iterations", C.c_int), ("solve_residual", C.c_double),
                ("adjoint_residual", C.c_double), ("refinement_steps", C.c_int),
                ("inner_iterations", C.c_int), ("n_sources", C.c_int),
                ("kernel_launches", C.c_longlong), ("fmm_nodes", C.c_longlong), ("fmm_m2l", C.c_longlong),
                ("fmm_near_pairs", C.c_longlong), ("fmm_m2l_flops", C.c_double)]


class DDLPBError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


_lib = None

EXPORTS = ["ddlpb_default_options", "ddlpb_setup", "ddlpb_setup_device", "ddlpb_solve", "ddlpb_adjoint",
           "ddlpb_energy", "ddlpb_energy_device", "ddlpb_forces", "ddlpb_forces_device", "ddlpb_apply_device",
           "ddlpb_get_vector_device", "ddlpb_get_info", "ddlpb_last_error", "ddlpb_last_setup_error", "ddlpb_free",
           "ddlpb_kernel_time", "ddlpb_kernel_time_reset", "ddlpb_energy_noalloc", "ddlpb_noalloc_last_error",
           "ddlpb_set_vector_device"]


def library():
    """Load libddlpb.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libddlpb.so is not built (run paper_2203_00552_gb300.build.build()); "
                           "there is no CPU fallback")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    dp = C.POINTER(C.c_double)
    lib.ddlpb_default_options.argtypes = [C.POINTER(Options)]
    lib.ddlpb_default_options.restype = None
    for name in ("ddlpb_setup", "ddlpb_setup_device"):
        f = getattr(lib, name)
        f.argtypes = [C.c_int, P, P, P, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int,
                      C.POINTER(Options), C.POINTER(P)]
        f.restype = C.c_int
    for name in ("ddlpb_solve", "ddlpb_adjoint"):
        getattr(lib, name).argtypes = [P]
        getattr(lib, name).restype = C.c_int
    for name in ("ddlpb_energy", "ddlpb_energy_device", "ddlpb_forces", "ddlpb_forces_device"):
        getattr(lib, name).argtypes = [P, P]
        getattr(lib, name).restype = C.c_int
    lib.ddlpb_apply_device.argtypes = [P, C.c_int, P, P]
    lib.ddlpb_apply_device.restype = C.c_int
    lib.ddlpb_get_vector_device.argtypes = [P, C.c_int, P]
    lib.ddlpb_get_vector_device.restype = C.c_int
    lib.ddlpb_set_vector_device.argtypes = [P, C.c_int, P]
    lib.ddlpb_set_vector_device.restype = C.c_int
    lib.ddlpb_get_info.argtypes = [P, C.POINTER(Info)]
    lib.ddlpb_get_info.restype = C.c_int
    lib.ddlpb_last_error.argtypes = [P]
    lib.ddlpb_last_error.restype = C.c_char_p
    lib.ddlpb_last_setup_error.argtypes = []
    lib.ddlpb_last_setup_error.restype = C.c_char_p
    lib.ddlpb_free.argtypes = [P]
    lib.ddlpb_free.restype = None
    lib.ddlpb_kernel_time.argtypes = [P, C.c_char_p, C.POINTER(C.c_longlong), C.POINTER(C.c_double)]
    lib.ddlpb_kernel_time.restype = C.c_int
    lib.ddlpb_kernel_time_reset.argtypes = [P]
    lib.ddlpb_kernel_time_reset.restype = C.c_int
    lib.ddlpb_energy_noalloc.argtypes = [C.c_int, C.c_int, P, P, P, P]
    lib.ddlpb_energy_noalloc.restype = C.c_int
    lib.ddlpb_noalloc_last_error.argtypes = []
    lib.ddlpb_noalloc_last_error.restype = C.c_char_p
    _lib = lib
    return lib


def default_options(**kw) -> Options:
    o = Options()
    library().ddlpb_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ptr(a):
    """Address of a contiguous numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"] and a.dtype == np.float64
        return a.ctypes.data_as(C.c_void_p)
    assert a.is_contiguous()
    return C.c_void_p(a.data_ptr())


def energy_noalloc(n, lmax, charges_dev, X_dev, stream=None) -> float:
    """E_s from device buffers through the allocation-free entry point (see include/ddlpb.h)."""
    lib = library()
    e = np.zeros(1)
    st = lib.ddlpb_energy_noalloc(int(n), int(lmax), _ptr(charges_dev), _ptr(X_dev), _ptr(e),
                                  C.c_void_p(stream) if stream else None)
    if st != 0:
        raise DDLPBError(st, lib.ddlpb_noalloc_last_error().decode())
    return float(e[0])


class Context:
    """One solute on the current CUDA device (wraps a ddlpb_ctx*)."""

    def __init__(self, centres, radii, charges, eps_solvent, kappa, lmax, n_lebedev, surface="vdw",
                 stream=None, **options):
        lib = library()
        opt = default_options(**options)
        if stream is not None:
            opt.cuda_stream = C.c_void_p(stream)
        surf = {"vdw": DDLPB_VDW, "sas": DDLPB_SAS}[surface]
        self._h = C.c_void_p()
        on_device = not isinstance(centres, np.ndarray)
        if on_device:
            n = int(centres.shape[0])
            st = lib.ddlpb_setup_device(n, _ptr(centres), _ptr(radii), _ptr(charges), float(eps_solvent),
                                        float(kappa), int(lmax), int(n_lebedev), surf, C.byref(opt),
                                        C.byref(self._h))
        else:
            centres = np.ascontiguousarray(centres, dtype=np.float64)
            radii = np.ascontiguousarray(radii, dtype=np.float64)
            charges = np.ascontiguousarray(charges, dtype=np.float64)
            n = int(centres.shape[0])
            st = lib.ddlpb_setup(n, _ptr(centres), _ptr(radii), _ptr(charges), float(eps_solvent), float(kappa),
                                 int(lmax), int(n_lebedev), surf, C.byref(opt), C.byref(self._h))
        if st != 0:
            raise DDLPBError(st, lib.ddlpb_last_setup_error().decode())
        self.n = n
        self.lmax = int(lmax)
        self.nb = (self.lmax + 1) ** 2
        self.nvec = 2 * n * self.nb

    def _check(self, st):
        if st != 0:
            raise DDLPBError(st, library().ddlpb_last_error(self._h).decode())

    def solve(self):
        self._check(library().ddlpb_solve(self._h))

    def adjoint(self):
        self._check(library().ddlpb_adjoint(self._h))

    def energy(self) -> float:
        e = np.zeros(1)
        self._check(library().ddlpb_energy(self._h, _ptr(e)))
        return float(e[0])

    def energy_device(self, out):
        self._check(library().ddlpb_energy_device(self._h, _ptr(out)))
        return out

    def forces(self) -> np.ndarray:
        f = np.zeros((self.n, 3))
        self._check(library().ddlpb_forces(self._h, _ptr(f)))
        return f

    def forces_device(self, out):
        self._check(library().ddlpb_forces_device(self._h, _ptr(out)))
        return out

    def apply(self, op: int, x, y):
        """y = op(x) on device tensors of length 2*n*(lmax+1)^2."""
        self._check(library().ddlpb_apply_device(self._h, int(op), _ptr(x), _ptr(y)))
        return y

    def vector(self, which: int, out):
        """Copy g (0), X (1) or X_adj (2) into the device tensor out."""
        self._check(library().ddlpb_get_vector_device(self._h, int(which), _ptr(out)))
        return out

    def set_vector(self, which: int, x):
        """Initial guess for the next solve: X (1) or X_adj (2), from the device tensor x."""
        self._check(library().ddlpb_set_vector_device(self._h, int(which), _ptr(x)))

    def info(self) -> dict:
        i = Info()
        self._check(library().ddlpb_get_info(self._h, C.byref(i)))
        return {k: getattr(i, k) for k, _ in Info._fields_}

    def kernel_time(self, name: str):
        """(launches, total ms) of one hot kernel since the last reset (needs kernel_timing=1)."""
        n = C.c_longlong()
        ms = C.c_double()
        self._check(library().ddlpb_kernel_time(self._h, name.encode(), C.byref(n), C.byref(ms)))
        return int(n.value), float(ms.value)

    def kernel_time_reset(self):
        self._check(library().ddlpb_kernel_time_reset(self._h))

    def close(self):
        if self._h:
            library().ddlpb_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
