"""Plain FP64 CPU oracle of the ADG method (arXiv 2603.28710) -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  The product path (the CUDA library and its Python binding)
never touches it.  The C source ``adgref.c`` follows the paper's definitions literally:
dense quadrature of the weak form (Eq. 6), a dense mass-matrix solve (Eq. 7), the Rusanov
flux with the paper's dissipation parameter (Eq. 8-9), the two-register LSERK update
(Eq. 10, Table 2), delayed fluxes (Eq. 13), AT fluxes from the moment constraints
(Eq. 14-15) and the communication schedules of Algorithms 2 and 3.

Parity status per function (what pins it lives in ``tests/test_oracle_*.py``):
  gauss, lagrange(+deriv), at_coeffs, rk_tableau, euler_flux, llf, schedule, rhs,
  step (SYNC / STD / AT / AT_TRACE), conservation, init_vortex, l2_error_vortex: pinned.
  init_tgv, dt_from_cfl: pinned by closed forms (test_oracle_init_dt.py): the Taylor-Green
  initial condition (not in the paper) by its uniform temperature, zero z velocity, domain
  means and pressure variance worked by hand, and its divergence-free velocity; the CFL
  time step by hand-computed uniform states, the node maximum and the t_end rounding.

The all-cores timing variant (``Oracle(parallel=True)``) is the same C source compiled with
OpenMP over elements; its results equal the single-threaded build's.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "adgref.c")
_HDR = os.path.join(_HERE, "adgref.h")
_LIB_PATH = os.path.join(_HERE, "_build", "libadgref.so")
# all-cores variant: the same source with OpenMP over elements (timing only; same results)
_LIB_PATH_OMP = os.path.join(_HERE, "_build", "libadgref_omp.so")
_lock = threading.Lock()
_libs = {}

FLUX = {"sync": 0, "std": 1, "at": 2, "at_trace": 3}
DELAY = {"caa": 0, "random": 1}
RK = {"rk22": 0, "rk33": 1, "ck45": 2}


def build(force: bool = False, parallel: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction, no fast-math); parallel=True
    builds the OpenMP variant used for the all-cores timing."""
    path = _LIB_PATH_OMP if parallel else _LIB_PATH
    os.makedirs(os.path.dirname(path), exist_ok=True)
    stale = (not os.path.exists(path)) or any(
        os.path.getmtime(p) > os.path.getmtime(path) for p in (_SRC, _HDR))
    if force or stale:
        tmp = path + f".{os.getpid()}.tmp"
        extra = ["-fopenmp"] if parallel else []
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               *extra, "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, path)
    return path


class _Params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n_elem", ctypes.c_int * 3),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("degree", ctypes.c_int), ("P", ctypes.c_int * 3),
                ("max_delay", ctypes.c_int), ("flux", ctypes.c_int), ("rk", ctypes.c_int),
                ("delay_mode", ctypes.c_int), ("random_delay_max", ctypes.c_int),
                ("at_np", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("gamma", ctypes.c_double), ("dt", ctypes.c_double)]


def lib(parallel: bool = False):
    with _lock:
        if parallel not in _libs:
            L = ctypes.CDLL(build(parallel=parallel))
            D, I, I64, U64 = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64
            P = ctypes.c_void_p
            L.adgref_gauss.argtypes = [I, P, P]
            L.adgref_lagrange.argtypes = [I, P, I, D]
            L.adgref_lagrange.restype = D
            L.adgref_lagrange_deriv.argtypes = [I, P, I, D]
            L.adgref_lagrange_deriv.restype = D
            L.adgref_at_coeffs.argtypes = [I, D, P]
            L.adgref_rk_tableau.argtypes = [I, P, P, P, P, P]
            L.adgref_euler_flux.argtypes = [I, D, P, I, P]
            L.adgref_llf.argtypes = [I, D, P, P, P, P]
            L.adgref_splitmix64.argtypes = [U64]
            L.adgref_splitmix64.restype = U64
            L.adgref_schedule.argtypes = [I, I, I, I, P, I, U64, I, I64, I, P, P, P]
            L.adgref_num_interfaces.argtypes = [I, P]
            L.adgref_create.argtypes = [ctypes.POINTER(_Params)]
            L.adgref_create.restype = P
            L.adgref_destroy.argtypes = [P]
            L.adgref_state_size.argtypes = [P]
            L.adgref_state_size.restype = I64
            L.adgref_set_state.argtypes = [P, P]
            L.adgref_get_state.argtypes = [P, P]
            L.adgref_step.argtypes = [P, I]
            L.adgref_rhs.argtypes = [P, P, P]
            L.adgref_rhs_elements.argtypes = [P, P, P, I64, P]
            L.adgref_conservation.argtypes = [P, P, P]
            L.adgref_init_vortex.argtypes = [P, P, D, D, D, D]
            L.adgref_init_tgv.argtypes = [P, P, D]
            L.adgref_l2_error_vortex.argtypes = [P, P, D, D, D, D, P]
            L.adgref_dt_from_cfl.argtypes = [P, P, D, D]
            L.adgref_dt_from_cfl.restype = D
            L.adgref_info.argtypes = [P, P, P, P]
            L.adgref_threads.argtypes = []
            L.adgref_threads.restype = I
            _libs[parallel] = L
    return _libs[parallel]


def threads(parallel: bool = False) -> int:
    """Threads the oracle's element loops use (1 unless parallel)."""
    return int(lib(parallel).adgref_threads())


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def gauss(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    if lib().adgref_gauss(n, _ptr(x), _ptr(w)) != 0:
        raise ValueError("unsupported number of points")
    return x, w


def lagrange(x: np.ndarray, a: int, xi: float) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().adgref_lagrange(len(x), _ptr(x), a, xi)


def lagrange_deriv(x: np.ndarray, a: int, xi: float) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().adgref_lagrange_deriv(len(x), _ptr(x), a, xi)


def at_coeffs(np_: int, km: float) -> np.ndarray:
    c = np.zeros(np_ + 1)
    if lib().adgref_at_coeffs(np_, km, _ptr(c)) != 0:
        raise ValueError("AT system singular")
    return c


def rk_tableau(scheme: str):
    """Returns (a, b, c, butcher_A, butcher_b) of the low-storage scheme."""
    a = np.zeros(8); b = np.zeros(8); c = np.zeros(8); ba = np.zeros(64); bb = np.zeros(8)
    s = lib().adgref_rk_tableau(RK[scheme], _ptr(a), _ptr(b), _ptr(c), _ptr(ba), _ptr(bb))
    return a[:s], b[:s], c[:s], ba[:s * s].reshape(s, s), bb[:s]


def euler_flux(dim: int, gamma: float, w, direction: int) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.float64)
    f = np.zeros(dim + 2)
    lib().adgref_euler_flux(dim, gamma, _ptr(w), direction, _ptr(f))
    return f


def llf(dim: int, gamma: float, wm, wp, normal) -> np.ndarray:
    wm = np.ascontiguousarray(wm, dtype=np.float64)
    wp = np.ascontiguousarray(wp, dtype=np.float64)
    n = np.zeros(3)
    n[:dim] = normal
    f = np.zeros(dim + 2)
    lib().adgref_llf(dim, gamma, _ptr(wm), _ptr(wp), _ptr(n), _ptr(f))
    return f


def splitmix64(x: int) -> int:
    return int(lib().adgref_splitmix64(x & 0xFFFFFFFFFFFFFFFF))


def num_interfaces(dim: int, P) -> int:
    Pa = np.array(list(P) + [1] * (3 - len(P)), dtype=np.int32)
    return lib().adgref_num_interfaces(dim, _ptr(Pa))


def schedule(flux: str, delay_mode: str, max_delay: int, np_: int, P, dim: int, seed: int,
             dmax: int, n0: int, count: int):
    """(comm[count], k[count], iface_delay[count, n_iface]) for steps n0 .. n0+count-1."""
    Pa = np.array(list(P) + [1] * (3 - len(P)), dtype=np.int32)
    nif = num_interfaces(dim, P)
    comm = np.zeros(count, np.int32)
    k = np.zeros(count, np.int32)
    dl = np.zeros((count, max(nif, 1)), np.int32)
    lib().adgref_schedule(FLUX[flux], DELAY[delay_mode], max_delay, np_, _ptr(Pa), dim,
                          seed & 0xFFFFFFFFFFFFFFFF, dmax, n0, count, _ptr(comm), _ptr(k), _ptr(dl))
    return comm, k, dl[:, :nif]


class Oracle:
    """The oracle solver; mirrors the library's create/set_state/step/get_state calls."""

    def __init__(self, dim=2, n_elem=(16, 16), lo=(-5.0, -5.0), hi=(5.0, 5.0), degree=2,
                 P=(1, 1), max_delay=1, flux="sync", rk="ck45", delay_mode="caa",
                 random_delay_max=0, at_np=0, seed=0, gamma=1.4, dt=1e-3, parallel=False):
        pr = _Params()
        pr.dim = dim
        P = tuple(P) + (1,) * (3 - len(P))
        for i in range(3):
            pr.n_elem[i] = n_elem[i] if i < dim else 1
            pr.lo[i] = lo[i] if i < dim else 0.0
            pr.hi[i] = hi[i] if i < dim else 1.0
            pr.P[i] = P[i] if i < dim else 1
        pr.degree = degree
        pr.max_delay = max_delay
        pr.flux = FLUX[flux]
        pr.rk = RK[rk]
        pr.delay_mode = DELAY[delay_mode]
        pr.random_delay_max = random_delay_max
        pr.at_np = at_np
        pr.seed = seed & 0xFFFFFFFFFFFFFFFF
        pr.gamma = gamma
        pr.dt = dt
        self._L = lib(parallel)
        self._h = self._L.adgref_create(ctypes.byref(pr))
        if not self._h:
            raise ValueError("oracle rejected the parameters")
        self.dim, self.degree, self.nv = dim, degree, dim + 2
        self.n_elem = tuple(n_elem[:dim])
        self.ne = int(np.prod(self.n_elem))
        self.nd = (degree + 1) ** dim
        self.size = int(self._L.adgref_state_size(self._h))
        self.shape = (self.nv, self.ne, self.nd)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.adgref_destroy(h)
            self._h = None

    def _arr(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        if u.size != self.size:
            raise ValueError("state has the wrong size")
        return u

    def set_state(self, u):
        self._L.adgref_set_state(self._h, _ptr(self._arr(u)))

    def get_state(self) -> np.ndarray:
        u = np.zeros(self.size)
        self._L.adgref_get_state(self._h, _ptr(u))
        return u.reshape(self.shape)

    def step(self, n: int = 1):
        self._L.adgref_step(self._h, n)

    def rhs(self, u) -> np.ndarray:
        k = np.zeros(self.size)
        self._L.adgref_rhs(self._h, _ptr(self._arr(u)), _ptr(k))
        return k.reshape(self.shape)

    def rhs_elements(self, u, elems) -> np.ndarray:
        el = np.ascontiguousarray(elems, dtype=np.int64)
        k = np.zeros((len(el), self.nv, self.nd))
        self._L.adgref_rhs_elements(self._h, _ptr(self._arr(u)), _ptr(el), len(el), _ptr(k))
        return k

    def conservation(self, u) -> np.ndarray:
        s = np.zeros(self.nv)
        self._L.adgref_conservation(self._h, _ptr(self._arr(u)), _ptr(s))
        return s

    def init_vortex(self, t=0.0, beta=5.0, x0=0.0, y0=0.0) -> np.ndarray:
        u = np.zeros(self.size)
        self._L.adgref_init_vortex(self._h, _ptr(u), t, beta, x0, y0)
        return u.reshape(self.shape)

    def init_tgv(self, mach=0.1) -> np.ndarray:
        u = np.zeros(self.size)
        self._L.adgref_init_tgv(self._h, _ptr(u), mach)
        return u.reshape(self.shape)

    def l2_error_vortex(self, u, t, beta=5.0, x0=0.0, y0=0.0) -> np.ndarray:
        e = np.zeros(3)
        self._L.adgref_l2_error_vortex(self._h, _ptr(self._arr(u)), t, beta, x0, y0, _ptr(e))
        return e

    def dt_from_cfl(self, u, cfl, t_end=0.0) -> float:
        return float(self._L.adgref_dt_from_cfl(self._h, _ptr(self._arr(u)), cfl, t_end))

    def info(self):
        s = ctypes.c_int64()
        t = ctypes.c_double()
        dt = ctypes.c_double()
        self._L.adgref_info(self._h, ctypes.byref(s), ctypes.byref(t), ctypes.byref(dt))
        return s.value, t.value, dt.value
