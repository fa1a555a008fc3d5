"""Thin Python binding of liblcbp.so (ctypes).

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind the C ABI declared in ``include/lcbp.h``.  There is no CPU
fallback: if the library is not built, or no GPU is present, calls raise.

PyTorch supplies device memory and streams: by default a lattice lives in a
``torch.uint8`` CUDA tensor (``lcbp_create_on_buffers``) and runs on a stream
owned by that lattice.  Field buffers may be numpy arrays (host) or torch
tensors (host or device); shapes follow the boundary layout
``[component, z, y, x]``.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "liblcbp.so")

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, ESTATE, EIO = 0, -1, -2, -3, -4, -5, -6, -7
F32, F64 = 0, 1
BPII, CHOL_X, CHOL_Y, CHOL_Z, ISO_NOISE, SLAB_BPII_IN_CHOL, SLAB_BPII_IN_ISO, SLAB_BPII_IN_CHOL_Z = range(8)
JACOBI, GAUSS_SEIDEL = 0, 1
PATH_AUTO, PATH_GENERIC, PATH_FAST1, PATH_FAST2 = 0, 1, 2, 3
CONV_AUTO, CONV_TAPS, CONV_WINDOW = 0, 1, 2
CONV_DW_CUDA_CORES = 4  # OR-ed into a kind: weight gradients on the CUDA-core kernel

_lib = None

_c_int, _c_double, _c_void_p, _c_size_t = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
_P = ctypes.c_void_p  # opaque handle

_SIGNATURES = {
    "lcbp_strerror": (ctypes.c_char_p, [_c_int]),
    "lcbp_last_error": (ctypes.c_char_p, []),
    "lcbp_version": (_c_int, []),
    "lcbp_create": (_c_int, [_c_int, _c_int, _c_int, _c_int, ctypes.POINTER(_P)]),
    "lcbp_workspace_bytes": (_c_size_t, [_c_int, _c_int, _c_int, _c_int]),
    "lcbp_create_on_buffers": (_c_int, [_c_int, _c_int, _c_int, _c_int, _c_void_p, _c_size_t, _c_void_p,
                                        ctypes.POINTER(_P)]),
    "lcbp_destroy": (_c_int, [_P]),
    "lcbp_get_info": (_c_int, [_P, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int),
                               ctypes.POINTER(ctypes.c_longlong)]),
    "lcbp_set_ldg": (_c_int, [_P, _c_double, _c_double, _c_double, _c_double]),
    "lcbp_set_ldg_kappa_tau": (_c_int, [_P, _c_double, _c_double, _c_double, _c_double]),
    "lcbp_set_flow": (_c_int, [_P, _c_double, _c_double, _c_double, _c_double, _c_int, _c_int]),
    "lcbp_params_kappa_tau": (_c_int, [_c_double, _c_double, _c_double, _c_double, _c_double, _c_double,
                                       _c_double, _c_void_p]),
    "lcbp_snapshot_bytes": (_c_size_t, [_P]),
    "lcbp_snapshot": (_c_int, [_P, _c_void_p]),
    "lcbp_restore": (_c_int, [_P, _c_void_p]),
    "lcbp_init_q": (_c_int, [_P, _c_int, _c_double, _c_double, ctypes.c_uint64, ctypes.POINTER(_c_int)]),
    "lcbp_set_q": (_c_int, [_P, _c_void_p, _c_int]),
    "lcbp_init_f_equilibrium": (_c_int, [_P, _c_double, _c_void_p, _c_int]),
    "lcbp_set_f": (_c_int, [_P, _c_void_p, _c_int]),
    "lcbp_set_body_force": (_c_int, [_P, _c_void_p, _c_int]),
    "lcbp_step": (_c_int, [_P, _c_int]),
    "lcbp_synchronize": (_c_int, [_P]),
    "lcbp_check_wait_timeout": (_c_int, [_c_double, ctypes.POINTER(_c_int)]),
    "lcbp_set_path": (_c_int, [_P, _c_int]),
    "lcbp_get_path": (_c_int, [_P, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int), ctypes.POINTER(_c_int)]),
    "lcbp_profile_steps": (_c_int, [_P, _c_int, ctypes.POINTER(_c_double), _c_int, ctypes.POINTER(_c_int)]),
    "lcbp_read_q": (_c_int, [_P, _c_void_p, _c_int]),
    "lcbp_read_u": (_c_int, [_P, _c_void_p, _c_int]),
    "lcbp_read_rho": (_c_int, [_P, _c_void_p, _c_int]),
    "lcbp_read_f": (_c_int, [_P, _c_void_p, _c_int]),
    "lcbp_free_energy": (_c_int, [_P, ctypes.POINTER(_c_double)]),
    "lcbp_totals": (_c_int, [_P, ctypes.POINTER(_c_double), ctypes.POINTER(_c_double)]),
    "lcbp_defect_fraction": (_c_int, [_P, _c_double, ctypes.POINTER(_c_double)]),
    "lcbp_optics_default": (_c_int, [_P]),
    "lcbp_set_walls": (_c_int, [_P, _c_int, _P]),
    "lcbp_set_l2": (_c_int, [_P, _c_int, _c_double]),
    "lcbp_texture": (_c_int, [_P, _P, _P]),
    "lcbp_save": (_c_int, [_P, ctypes.c_char_p]),
    "lcbp_load": (_c_int, [_P, ctypes.c_char_p]),
    "lcbp_reequilibrate_f": (_c_int, [_P]),
    "lcbp_get_tuning": (_c_int, [_P, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int), ctypes.POINTER(_c_int),
                                 ctypes.POINTER(_c_int)]),
    "lcbp_free_energy_noalloc": (_c_int, [_c_void_p, _c_int, _c_int, _c_int, _c_int, _c_double, _c_double,
                                          _c_double, _c_double, _c_void_p, ctypes.POINTER(_c_double)]),
    "lcbp_surrogate_param_count": (_c_size_t, []),
    "lcbp_surrogate_create": (_c_int, [_c_int, _c_int, _c_int, _c_int, ctypes.POINTER(_P)]),
    "lcbp_surrogate_destroy": (_c_int, [_P]),
    "lcbp_surrogate_set_scales": (_c_int, [_P, _c_double, _c_double, _c_double]),
    "lcbp_surrogate_set_conv_kernel": (_c_int, [_P, _c_int]),
    "lcbp_surrogate_set_params": (_c_int, [_P, _c_void_p, _c_size_t]),
    "lcbp_surrogate_get_params": (_c_int, [_P, _c_void_p, _c_size_t]),
    "lcbp_surrogate_get_grads": (_c_int, [_P, _c_void_p, _c_size_t]),
    "lcbp_surrogate_forward": (_c_int, [_P, _c_void_p, _c_void_p, _c_void_p, _c_double, _c_double, _c_int,
                                        _c_void_p]),
    "lcbp_surrogate_step": (_c_int, [_P, _P, _c_double, _c_double, _c_int]),
    "lcbp_surrogate_train_step": (_c_int, [_P, _c_void_p, _c_void_p, _c_void_p, _c_double, _c_double, _c_void_p,
                                           _c_void_p, _c_int, _c_double, ctypes.POINTER(_c_double)]),
    "lcbp_read_rate": (_c_int, [_P, _c_void_p, _c_int]),
    "lcbp_surrogate_set_steps": (_c_int, [_P, _c_int]),
    "lcbp_surrogate_get_steps": (_c_int, [_P, ctypes.POINTER(_c_int)]),
    "lcbp_surrogate_save": (_c_int, [_P, ctypes.c_char_p]),
    "lcbp_surrogate_load": (_c_int, [_P, ctypes.c_char_p]),
    "lcbp_judge_create": (_c_int, [_P, _P, _c_void_p, ctypes.POINTER(_P)]),
    "lcbp_judge_destroy": (_c_int, [_P]),
    "lcbp_judge_advance": (_c_int, [_P, ctypes.c_longlong, _c_int, _c_double, _c_void_p, _c_void_p, _c_void_p,
                                    _c_int, ctypes.POINTER(_c_int)]),
    "lcbp_judge_get_stats": (_c_int, [_P, _c_void_p]),
    "lcbp_batch_create": (_c_int, [_c_int, ctypes.POINTER(_c_int), _c_void_p, _c_int, ctypes.POINTER(_P)]),
    "lcbp_batch_destroy": (_c_int, [_P]),
    "lcbp_batch_set_flow": (_c_int, [_P, _c_int, _c_int]),
    "lcbp_batch_init_q": (_c_int, [_P, _c_int, _c_int, _c_double, _c_double, ctypes.c_uint64,
                                   ctypes.POINTER(_c_int)]),
    "lcbp_batch_set_q": (_c_int, [_P, _c_int, _c_void_p, _c_int]),
    "lcbp_batch_init_f_equilibrium": (_c_int, [_P, _c_double]),
    "lcbp_batch_step": (_c_int, [_P, _c_int]),
    "lcbp_batch_synchronize": (_c_int, [_P]),
    "lcbp_batch_read_q": (_c_int, [_P, _c_int, _c_void_p, _c_int]),
    "lcbp_batch_read_u": (_c_int, [_P, _c_int, _c_void_p, _c_int]),
    "lcbp_batch_free_energy": (_c_int, [_P, _c_int, ctypes.POINTER(_c_double)]),
    "lcbp_batch_totals": (_c_int, [_P, _c_int, ctypes.POINTER(_c_double), ctypes.POINTER(_c_double)]),
    "lcbp_batch_defect_fraction": (_c_int, [_P, _c_int, _c_double, ctypes.POINTER(_c_double)]),
    "lcbp_batch_set_path": (_c_int, [_P, _c_int]),
    "lcbp_batch_get_path": (_c_int, [_P, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int)]),
    "lcbp_batch_get_info": (_c_int, [_P, ctypes.POINTER(_c_int), ctypes.POINTER(ctypes.c_longlong),
                                     ctypes.POINTER(_c_int), ctypes.POINTER(_c_int),
                                     ctypes.POINTER(ctypes.c_longlong)]),
}


class Params(ctypes.Structure):
    """lcbp_params: per-replica parameters of a batch."""
    _fields_ = [(k, _c_double) for k in ("A0", "gamma", "K", "q0", "tau_f", "xi", "Gamma")]

    @classmethod
    def _fields_names(cls):
        return [f[0] for f in cls._fields_]


def params_kappa_tau(A0: float, q0: float, kappa: float, tau: float, tau_f: float = 2.0, xi: float = 0.7,
                     Gamma: float = 0.3) -> dict:
    """Per-replica parameters from the reduced chirality and temperature
    (lcbp_params_kappa_tau: gamma and K are derived by the library)."""
    p = Params()
    check(lib().lcbp_params_kappa_tau(A0, q0, kappa, tau, tau_f, xi, Gamma, ctypes.byref(p)))
    return {k: getattr(p, k) for k in Params._fields_names()}


class LcbpError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{message} (status {code})")
        self.code = code


def lib() -> ctypes.CDLL:
    """Load liblcbp.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: run paper_0901_3293_gb300.build.build() "
                               "(or __graft_entry__.build()); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(rc: int) -> None:
    if rc != OK:
        msg = lib().lcbp_last_error().decode() or lib().lcbp_strerror(rc).decode()
        raise LcbpError(rc, msg)


def _dtype_code(a) -> int:
    name = str(a.dtype)
    if name.endswith("float32"):
        return F32
    if name.endswith("float64"):
        return F64
    raise TypeError(f"buffers must be float32 or float64, got {name}")


def _ptr(a):
    """(pointer, dtype code, keep-alive) of a numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a)
        return a.ctypes.data, _dtype_code(a), a
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            a = a.contiguous()
        if a.is_cuda:
            import torch
            # the library works on its own stream: finish pending torch work on the tensor
            torch.cuda.synchronize(a.device)
        return a.data_ptr(), _dtype_code(a), a
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a.ctypes.data, F64, a


def _raw_buffer(a, nbytes: int) -> int:
    """Address of a contiguous buffer (torch tensor or numpy array) of at least nbytes bytes."""
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous or a.nbytes < nbytes:
            raise ValueError(f"need a contiguous buffer of {nbytes} bytes")
        return a.ctypes.data
    if not a.is_contiguous() or a.numel() * a.element_size() < nbytes:
        raise ValueError(f"need a contiguous buffer of {nbytes} bytes")
    if a.is_cuda:
        import torch
        torch.cuda.synchronize(a.device)
    return a.data_ptr()


class Optics(ctypes.Structure):
    """lcbp_optics: wavelengths and weights, indices, layer thickness, polariser angles."""
    _fields_ = [("nlambda", _c_int), ("lambda_", _c_double * 4), ("weight", _c_double * 4),
                ("n_o", _c_double), ("n_e", _c_double), ("h", _c_double),
                ("phi_in", _c_double), ("phi_out", _c_double)]

    @classmethod
    def default(cls) -> "Optics":
        """The values of the paper's rendering: lambda 16, 18, 20 with weights 0.2, 0.6, 0.2,
        n_o 1.5, n_e 2.0, h 1, crossed polarisers at 0 and pi/2."""
        o = cls()
        check(lib().lcbp_optics_default(ctypes.byref(o)))
        return o


def write_pgm(img: np.ndarray, path: str, vmax: float | None = None) -> None:
    """Write a grayscale image (e.g. a texture) as binary 8-bit PGM, scaled to [0, vmax]."""
    a = np.asarray(img, dtype=np.float64)
    top = float(vmax) if vmax else (float(a.max()) if a.max() > 0 else 1.0)
    g = np.clip(np.rint(255.0 * a / top), 0, 255).astype(np.uint8)
    with open(path, "wb") as fh:
        fh.write(b"P5\n%d %d\n255\n" % (g.shape[1], g.shape[0]))
        fh.write(g.tobytes())


class Lattice:
    """A periodic nx * ny * nz lattice on the current CUDA device.

    memory="torch" (default): state lives in a torch CUDA tensor and work runs
    on a torch stream owned by the lattice; memory="library": lcbp_create
    allocates with cudaMalloc and owns its stream.
    """

    def __init__(self, nx: int, ny: int, nz: int, dtype: str = "f32", memory: str = "torch", device=None):
        self.dims = (int(nx), int(ny), int(nz))
        self.n = self.dims[0] * self.dims[1] * self.dims[2]
        self.state_dtype = {"f32": F32, "f64": F64}[dtype]
        self.np_dtype = np.float32 if self.state_dtype == F32 else np.float64
        self._h = _P()
        self._ws = None
        self._stream = None
        L = lib()
        if memory == "torch":
            import torch
            dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
            nbytes = L.lcbp_workspace_bytes(*self.dims, self.state_dtype)
            if nbytes == 0:
                raise LcbpError(EINVAL, "invalid lattice size")
            with torch.cuda.device(dev):
                self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
                self._stream = torch.cuda.Stream(device=dev)
                base = self._ws.data_ptr()
                off = (-base) % 256
                check(L.lcbp_create_on_buffers(*self.dims, self.state_dtype, base + off, nbytes,
                                               self._stream.cuda_stream, ctypes.byref(self._h)))
        elif memory == "library":
            check(L.lcbp_create(*self.dims, self.state_dtype, ctypes.byref(self._h)))
        else:
            raise ValueError(memory)

    # -- lifetime -----------------------------------------------------------
    def close(self) -> None:
        if self._h:
            check(lib().lcbp_destroy(self._h))
            self._h = _P()
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- parameters ---------------------------------------------------------
    def set_ldg(self, A0: float, gamma: float, K: float, q0: float) -> "Lattice":
        check(lib().lcbp_set_ldg(self._h, A0, gamma, K, q0))
        return self

    def set_ldg_kappa_tau(self, A0: float, q0: float, kappa: float, tau: float) -> "Lattice":
        check(lib().lcbp_set_ldg_kappa_tau(self._h, A0, q0, kappa, tau))
        return self

    def set_flow(self, tau_f: float = 2.0, xi: float = 0.7, Gamma: float = 0.3, flow_on: bool = True,
                 coupling: int = JACOBI, rho0: float = 1.0) -> "Lattice":
        check(lib().lcbp_set_flow(self._h, tau_f, rho0, xi, Gamma, int(bool(flow_on)), coupling))
        return self

    # -- state ----------------------------------------------------------------
    def set_l2(self, L2: float | None) -> "Lattice":
        """Energy with -((K - L2)/2)|div Q|^2 added (L2 = 0: exactly as printed); None: one-constant."""
        check(lib().lcbp_set_l2(self._h, 0 if L2 is None else 1, 0.0 if L2 is None else float(L2)))
        return self

    def set_walls(self, walls: bool = True, q_wall=None) -> "Lattice":
        """Solid walls below z = 0 and above z = Nz-1 (bounce-back, strong anchoring to q_wall, q5 order)."""
        qw = None if q_wall is None else np.ascontiguousarray(np.asarray(q_wall, dtype=np.float64).reshape(5))
        check(lib().lcbp_set_walls(self._h, 1 if walls else 0, qw.ctypes.data if qw is not None else None))
        return self

    def init_q(self, kind: int, amplitude: float, noise: float = 0.0, seed: int = 0, z0: int | None = None):
        region = (ctypes.c_int * 1)(z0) if z0 is not None else None
        check(lib().lcbp_init_q(self._h, kind, amplitude, noise, seed, region))
        return self

    def set_q(self, q5) -> "Lattice":
        p, d, keep = _ptr(q5)
        self._check_size(keep, 5)
        check(lib().lcbp_set_q(self._h, p, d))
        return self

    def init_f_equilibrium(self, rho0: float = 1.0, u3=None) -> "Lattice":
        if u3 is None:
            check(lib().lcbp_init_f_equilibrium(self._h, rho0, None, F64))
        else:
            p, d, keep = _ptr(u3)
            self._check_size(keep, 3)
            check(lib().lcbp_init_f_equilibrium(self._h, rho0, p, d))
        return self

    def set_f(self, f15) -> "Lattice":
        p, d, keep = _ptr(f15)
        self._check_size(keep, 15)
        check(lib().lcbp_set_f(self._h, p, d))
        return self

    def set_body_force(self, b3) -> "Lattice":
        if b3 is None:
            check(lib().lcbp_set_body_force(self._h, None, F64))
        else:
            p, d, keep = _ptr(b3)
            self._check_size(keep, 3)
            check(lib().lcbp_set_body_force(self._h, p, d))
        return self

    def step(self, nsteps: int = 1) -> "Lattice":
        check(lib().lcbp_step(self._h, int(nsteps)))
        return self

    def profile_steps(self, nsteps: int):
        """Advance nsteps steps kernel by kernel; mean device ms per kernel."""
        ms = (_c_double * 8)()
        nk = _c_int()
        check(lib().lcbp_profile_steps(self._h, int(nsteps), ms, 8, ctypes.byref(nk)))
        return list(ms[:nk.value])

    def set_path(self, path: int) -> "Lattice":
        check(lib().lcbp_set_path(self._h, path))
        return self

    def path(self):
        """(fast path in use, autotuned planes per CTA, sites per thread)."""
        fast = _c_int()
        zc = _c_int()
        spt = _c_int()
        check(lib().lcbp_get_path(self._h, ctypes.byref(fast), ctypes.byref(zc), ctypes.byref(spt)))
        return bool(fast.value), zc.value, spt.value

    def tuning(self):
        """(planes per CTA and sites per thread of the LB kernel, sites per
        thread and planes per CTA of the field kernel)."""
        zc, sl, sq, zq = _c_int(), _c_int(), _c_int(), _c_int()
        check(lib().lcbp_get_tuning(self._h, ctypes.byref(zc), ctypes.byref(sl), ctypes.byref(sq), ctypes.byref(zq)))
        return zc.value, sl.value, sq.value, zq.value

    def synchronize(self) -> None:
        check(lib().lcbp_synchronize(self._h))

    def reequilibrate_f(self) -> "Lattice":
        check(lib().lcbp_reequilibrate_f(self._h))
        return self

    def _check_size(self, a, comps: int) -> None:
        if int(np.prod(a.shape)) != comps * self.n:
            raise LcbpError(EINVAL, f"expected {comps} x {self.n} values, got shape {tuple(a.shape)}")

    def _read(self, fn, comps: int, dtype, out=None):
        shape = (comps, self.dims[2], self.dims[1], self.dims[0])
        if out is None:
            out = np.empty(shape, dtype=dtype)
        p, d, keep = _ptr(out)
        check(fn(self._h, p, d))
        return out

    def read_q(self, dtype=np.float64, out=None):
        return self._read(lib().lcbp_read_q, 5, dtype, out)

    def read_u(self, dtype=np.float64, out=None):
        return self._read(lib().lcbp_read_u, 3, dtype, out)

    def read_rho(self, dtype=np.float64, out=None):
        return self._read(lib().lcbp_read_rho, 1, dtype, out)[0] if out is None else \
            self._read(lib().lcbp_read_rho, 1, dtype, out)

    def read_f(self, dtype=np.float64, out=None):
        return self._read(lib().lcbp_read_f, 15, dtype, out)

    def read_rate(self, dtype=np.float64, out=None):
        """Beris-Edwards rate dQ/dt = Gamma H + S - u.grad Q of the current state."""
        return self._read(lib().lcbp_read_rate, 5, dtype, out)

    # -- diagnostics ------------------------------------------------------------
    def free_energy(self) -> float:
        F = _c_double()
        check(lib().lcbp_free_energy(self._h, ctypes.byref(F)))
        return F.value

    def totals(self):
        m = _c_double()
        P = (_c_double * 3)()
        check(lib().lcbp_totals(self._h, ctypes.byref(m), P))
        return m.value, np.array(P[:])

    def defect_fraction(self, threshold: float = 0.19) -> float:
        fr = _c_double()
        check(lib().lcbp_defect_fraction(self._h, threshold, ctypes.byref(fr)))
        return fr.value

    def texture(self, optics: "Optics | None" = None) -> np.ndarray:
        """Polarised-light texture [ny, nx] (FP32) of the current Q between crossed polarisers."""
        o = optics if optics is not None else Optics.default()
        nx, ny, _ = self.dims
        img = np.empty((ny, nx), dtype=np.float32)
        check(lib().lcbp_texture(self._h, ctypes.byref(o), img.ctypes.data))
        return img

    def info(self):
        dims = (_c_int * 3)()
        dt = _c_int()
        st = ctypes.c_longlong()
        check(lib().lcbp_get_info(self._h, dims, ctypes.byref(dt), ctypes.byref(st)))
        return tuple(dims), dt.value, st.value

    def save(self, path: str) -> None:
        check(lib().lcbp_save(self._h, os.fsencode(path)))

    def snapshot_bytes(self) -> int:
        return int(lib().lcbp_snapshot_bytes(self._h))

    def snapshot(self, out) -> None:
        """Raw state (f, rho u, Q) into `out`: a contiguous CUDA tensor or numpy
        array of at least snapshot_bytes() bytes, any element type.  restore()
        brings it back bitwise."""
        check(lib().lcbp_snapshot(self._h, _raw_buffer(out, self.snapshot_bytes())))

    def restore(self, src) -> "Lattice":
        check(lib().lcbp_restore(self._h, _raw_buffer(src, self.snapshot_bytes())))
        return self

    def load(self, path: str) -> None:
        check(lib().lcbp_load(self._h, os.fsencode(path)))


class Batch:
    """R replicas of uneven sizes and per-replica parameters, stepped together.

    dims: list of (nx, ny, nz); params: list of dicts with keys A0, gamma, K,
    q0, tau_f, xi, Gamma.
    """

    def __init__(self, dims, params, dtype: str = "f32"):
        self.R = len(dims)
        self.dims = [tuple(int(v) for v in d) for d in dims]
        arr = (_c_int * (3 * self.R))(*[v for d in self.dims for v in d])
        ps = (Params * self.R)(*[Params(**{k: float(p[k]) for k in Params._fields_names()}) for p in params])
        self._h = _P()
        self.state_dtype = {"f32": F32, "f64": F64}[dtype]
        check(lib().lcbp_batch_create(self.R, arr, ctypes.cast(ps, _c_void_p), self.state_dtype,
                                      ctypes.byref(self._h)))

    def close(self) -> None:
        if self._h:
            check(lib().lcbp_batch_destroy(self._h))
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_flow(self, flow_on: bool = True, coupling: int = JACOBI) -> "Batch":
        check(lib().lcbp_batch_set_flow(self._h, int(bool(flow_on)), coupling))
        return self

    def set_path(self, path: int) -> "Batch":
        check(lib().lcbp_batch_set_path(self._h, path))
        return self

    def path(self):
        """(fast kernels in use, tuned planes per CTA or 0)."""
        fast = _c_int()
        zc = _c_int()
        check(lib().lcbp_batch_get_path(self._h, ctypes.byref(fast), ctypes.byref(zc)))
        return bool(fast.value), zc.value

    def init_q(self, r: int, kind: int, amplitude: float, noise: float = 0.0, seed: int = 0, z0=None) -> "Batch":
        region = (_c_int * 1)(z0) if z0 is not None else None
        check(lib().lcbp_batch_init_q(self._h, r, kind, amplitude, noise, seed, region))
        return self

    def set_q(self, r: int, q5) -> "Batch":
        p, d, keep = _ptr(q5)
        check(lib().lcbp_batch_set_q(self._h, r, p, d))
        return self

    def init_f_equilibrium(self, rho0: float = 1.0) -> "Batch":
        check(lib().lcbp_batch_init_f_equilibrium(self._h, rho0))
        return self

    def step(self, nsteps: int = 1) -> "Batch":
        check(lib().lcbp_batch_step(self._h, int(nsteps)))
        return self

    def synchronize(self) -> None:
        check(lib().lcbp_batch_synchronize(self._h))

    def _read(self, fn, r, comps, dtype):
        if not 0 <= r < self.R:
            raise LcbpError(EINVAL, f"replica {r} out of range [0, {self.R})")
        nx, ny, nz = self.dims[r]
        out = np.empty((comps, nz, ny, nx), dtype=dtype)
        p, d, keep = _ptr(out)
        check(fn(self._h, r, p, d))
        return out

    def read_q(self, r: int, dtype=np.float64):
        return self._read(lib().lcbp_batch_read_q, r, 5, dtype)

    def read_u(self, r: int, dtype=np.float64):
        return self._read(lib().lcbp_batch_read_u, r, 3, dtype)

    def free_energy(self, r: int) -> float:
        F = _c_double()
        check(lib().lcbp_batch_free_energy(self._h, r, ctypes.byref(F)))
        return F.value

    def totals(self, r: int):
        m = _c_double()
        P = (_c_double * 3)()
        check(lib().lcbp_batch_totals(self._h, r, ctypes.byref(m), P))
        return m.value, np.array(P[:])

    def defect_fraction(self, r: int, threshold: float = 0.19) -> float:
        fr = _c_double()
        check(lib().lcbp_batch_defect_fraction(self._h, r, threshold, ctypes.byref(fr)))
        return fr.value

    def info(self):
        R = _c_int()
        tot = ctypes.c_longlong()
        tile = (_c_int * 3)()
        ctas = _c_int()
        st = ctypes.c_longlong()
        check(lib().lcbp_batch_get_info(self._h, ctypes.byref(R), ctypes.byref(tot), tile, ctypes.byref(ctas),
                                        ctypes.byref(st)))
        return {"R": R.value, "sites": tot.value, "tile": tuple(tile), "persistent_ctas": ctas.value,
                "step": st.value}


def check_wait_timeout(limit_ms: float) -> bool:
    """Self-test of the bounded device-side wait: True if a wait on a barrier
    that nothing arrives on gave up after limit_ms and reported it."""
    out = _c_int()
    check(lib().lcbp_check_wait_timeout(limit_ms, ctypes.byref(out)))
    return bool(out.value)


def free_energy_noalloc(q5_device, nx: int, ny: int, nz: int, A0: float, gamma: float, K: float, q0: float,
                        stream=None) -> float:
    """F_h of a device Q field without any device allocation (lcbp_free_energy_noalloc).

    q5_device: a CUDA tensor of 5 * nx * ny * nz float32 or float64 values;
    stream: a torch.cuda.Stream or None (legacy default stream)."""
    F = _c_double()
    dt = _dtype_code(q5_device)
    sp = stream.cuda_stream if stream is not None else None
    check(lib().lcbp_free_energy_noalloc(q5_device.data_ptr(), dt, nx, ny, nz, A0, gamma, K, q0, sp,
                                         ctypes.byref(F)))
    return F.value


class Surrogate:
    """Convolutional surrogate advancing Q by 10 solver steps (tensor-core kernels)."""

    def __init__(self, nx: int, ny: int, nz: int, training: bool = False):
        self.dims = (int(nx), int(ny), int(nz))
        self.n = self.dims[0] * self.dims[1] * self.dims[2]
        self.count = int(lib().lcbp_surrogate_param_count())
        self._h = _P()
        check(lib().lcbp_surrogate_create(*self.dims, int(bool(training)), ctypes.byref(self._h)))

    def close(self) -> None:
        if self._h:
            check(lib().lcbp_surrogate_destroy(self._h))
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_scales(self, s_u: float = 1e-3, s_r: float = 1e-3, s_dq: float = 1e-3) -> "Surrogate":
        check(lib().lcbp_surrogate_set_scales(self._h, s_u, s_r, s_dq))
        return self

    def set_conv_kernel(self, kind: int) -> "Surrogate":
        """CONV_AUTO, CONV_TAPS (one shifted tile per tap) or CONV_WINDOW (one staged plane for all taps),
        optionally OR-ed with CONV_DW_CUDA_CORES (weight gradients on the CUDA-core kernel)."""
        check(lib().lcbp_surrogate_set_conv_kernel(self._h, kind))
        return self

    def set_params(self, v) -> "Surrogate":
        a = np.ascontiguousarray(np.asarray(v, dtype=np.float32))
        check(lib().lcbp_surrogate_set_params(self._h, a.ctypes.data, a.size))
        return self

    def set_steps(self, k: int) -> "Surrogate":
        """Solver steps one call stands for (default 10)."""
        check(lib().lcbp_surrogate_set_steps(self._h, int(k)))
        return self

    def steps(self) -> int:
        k = _c_int()
        check(lib().lcbp_surrogate_get_steps(self._h, ctypes.byref(k)))
        return k.value

    def save(self, path: str) -> None:
        """Write the weights file (parameters and scales, versioned)."""
        check(lib().lcbp_surrogate_save(self._h, os.fsencode(path)))

    def load(self, path: str) -> "Surrogate":
        """Read a weights file written by save (any lattice size)."""
        check(lib().lcbp_surrogate_load(self._h, os.fsencode(path)))
        return self

    def get_params(self) -> np.ndarray:
        a = np.empty(self.count, dtype=np.float32)
        check(lib().lcbp_surrogate_get_params(self._h, a.ctypes.data, a.size))
        return a

    def get_grads(self) -> np.ndarray:
        a = np.empty(self.count, dtype=np.float32)
        check(lib().lcbp_surrogate_get_grads(self._h, a.ctypes.data, a.size))
        return a

    @staticmethod
    def _opt(a, dt):
        if a is None:
            return None, None
        p, d, keep = _ptr(a)
        if d != dt:
            raise TypeError("all field buffers must share a dtype")
        return p, keep

    def forward(self, q5, u3, r5, kappa: float, tau: float) -> np.ndarray:
        """Network output y for fields Q, u (or None), rate R (or None)."""
        pq, dq, kq = _ptr(q5)
        pu, ku = self._opt(u3, dq)
        pr, kr = self._opt(r5, dq)
        nx, ny, nz = self.dims
        out = np.empty((5, nz, ny, nx), dtype=np.float32)
        check(lib().lcbp_surrogate_forward(self._h, pq, pu, pr, kappa, tau, dq, out.ctypes.data))
        return out

    def step(self, lattice: "Lattice", kappa: float, tau: float, ncalls: int = 1) -> "Surrogate":
        check(lib().lcbp_surrogate_step(self._h, lattice._h, kappa, tau, int(ncalls)))
        return self

    def train_step(self, q5, u3, r5, kappa: float, tau: float, dq5, mask=None, lr: float = 1e-3) -> float:
        """One Adam step; dq5 is the true 10-step change of Q."""
        pq, dq, kq = _ptr(q5)
        pu, ku = self._opt(u3, dq)
        pr, kr = self._opt(r5, dq)
        pt, kt = self._opt(dq5, dq)
        pm, km = self._opt(mask, dq)
        loss = _c_double()
        check(lib().lcbp_surrogate_train_step(self._h, pq, pu, pr, kappa, tau, pt, pm, dq, lr, ctypes.byref(loss)))
        return loss.value


class JudgeConfig(ctypes.Structure):
    """lcbp_judge_config."""
    _fields_ = [("kappa", _c_double), ("tau", _c_double), ("calls_per_segment", _c_int), ("tol_F", _c_double),
                ("tol_Q", _c_double), ("warmup_steps", ctypes.c_longlong)]


class JudgeStats(ctypes.Structure):
    """lcbp_judge_stats."""
    _fields_ = [(k, ctypes.c_longlong) for k in ("t", "segments", "accepted", "fallbacks", "surrogate_calls",
                                                 "plain_steps")] + \
               [(k, _c_double) for k in ("last_gap_F", "last_gap_Q", "max_gap_F", "mean_gap_F", "mean_gap_Q")] + \
               [("judged", ctypes.c_longlong)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class Judge:
    """The judged surrogate run of the library (lcbp_judge_*): after
    `warmup_steps` plain steps, segments of `calls_per_segment` surrogate
    calls, each judged against k plain steps
    (relative F gap <= tol_F, and max |dQ| <= tol_Q if tol_Q > 0), rolled back
    and redone plainly when it fails.  Keeps references to the lattice and
    the surrogate."""

    def __init__(self, lattice: "Lattice", surrogate: "Surrogate", kappa: float, tau: float,
                 calls_per_segment: int = 49, tol_F: float = 1e-3, tol_Q: float = 0.0, warmup_steps: int = 0):
        self.lattice, self.surrogate = lattice, surrogate
        cfg = JudgeConfig(float(kappa), float(tau), int(calls_per_segment), float(tol_F), float(tol_Q),
                          int(warmup_steps))
        self._h = _P()
        check(lib().lcbp_judge_create(lattice._h, surrogate._h, ctypes.byref(cfg), ctypes.byref(self._h)))

    def advance(self, t_end: int, log_every: int = 0, defect_threshold: float = 0.19):
        """Advance to t_end; with log_every > 0 returns the log as arrays (t, F, defect fraction)."""
        if log_every <= 0:
            check(lib().lcbp_judge_advance(self._h, int(t_end), 0, defect_threshold, None, None, None, 0, None))
            return None
        cap = int(t_end) // log_every + 1
        t = np.zeros(cap, dtype=np.int64)
        F = np.zeros(cap)
        D = np.zeros(cap)
        n = _c_int()
        check(lib().lcbp_judge_advance(self._h, int(t_end), int(log_every), defect_threshold, t.ctypes.data,
                                       F.ctypes.data, D.ctypes.data, cap, ctypes.byref(n)))
        return t[:n.value], F[:n.value], D[:n.value]

    def stats(self) -> dict:
        st = JudgeStats()
        check(lib().lcbp_judge_get_stats(self._h, ctypes.byref(st)))
        return st.as_dict()

    def close(self) -> None:
        if self._h:
            check(lib().lcbp_judge_destroy(self._h))
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
