"""Thin ctypes binding of the C ABI in include/adg.h.

Argument marshalling only: every step of the method runs in the CUDA library.  Device
buffers are torch tensors (their data_ptr() is passed with on_device=1); host buffers are
numpy arrays.  The binding raises if the compiled library is missing -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libadg.so")

FLUX = {"sync": 0, "std": 1, "at": 2, "at_trace": 3, "learned": 4}
DELAY = {"caa": 0, "random": 1}
RK = {"rk22": 0, "rk33": 1, "ck45": 2}
PREC = {"fp64": 0, "fp32": 1, "df64": 2}
PATH = {"auto": 0, "split": 1, "fused": 2, "element": 3}
STATUS = {0: "ADG_OK", 1: "ADG_ERR_INVALID", 2: "ADG_ERR_UNSUPPORTED", 3: "ADG_ERR_CUDA",
          4: "ADG_ERR_OOM", 5: "ADG_ERR_NONFINITE", 6: "ADG_ERR_TIMEOUT", 7: "ADG_ERR_STATE"}

# every symbol the header declares (tests check the library exports them all)
SYMBOLS = ["adg_default_options", "adg_create", "adg_set_state", "adg_init_vortex",
           "adg_init_tgv", "adg_step", "adg_get_state", "adg_rhs", "adg_get_schedule",
           "adg_info", "adg_conservation", "adg_l2_error_vortex", "adg_check_finite",
           "adg_last_error", "adg_destroy", "adg_set_profiling", "adg_get_profile", "adg_rhs_noalloc",
           "adg_checkpoint_bytes", "adg_checkpoint_save", "adg_checkpoint_restore",
           "adg_batch_create", "adg_batch_init_vortex", "adg_batch_set_state", "adg_batch_step",
           "adg_batch_autotune", "adg_batch_get_state", "adg_batch_info",
           "adg_batch_l2_error_vortex", "adg_batch_num_groups", "adg_batch_last_error",
           "adg_batch_destroy", "adg_mlp_num_params", "adg_mlp_grad", "adg_mlp_forward",
           "adg_mlp_adam", "adg_mlp_to_bf16", "adg_set_learned_model", "adg_set_trace_log",
           "adg_learned_samples", "adg_host_gauss", "adg_host_at_coeffs",
           "adg_host_rk", "adg_host_schedule", "adg_host_num_interfaces", "adg_measure_peak",
           "adg_probe_wait"]


class AdgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n_elem", ctypes.c_int * 3),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3)]


class Options(ctypes.Structure):
    _fields_ = [("rk", ctypes.c_int), ("dt", ctypes.c_double), ("cfl", ctypes.c_double),
                ("t_end", ctypes.c_double), ("gamma", ctypes.c_double),
                ("delay_mode", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("random_delay_max", ctypes.c_int), ("at_np", ctypes.c_int),
                ("precision", ctypes.c_int), ("cuda_stream", ctypes.c_void_p),
                ("kernel_path", ctypes.c_int)]


_lock = threading.Lock()
_lib = None


def lib():
    """Loads libadg.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        I, I64, D, P, U64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_uint64
        sig = {
            "adg_default_options": ([ctypes.POINTER(Options)], I),
            "adg_create": ([ctypes.POINTER(Mesh), I, P, I, I, ctypes.POINTER(Options),
                            ctypes.POINTER(ctypes.c_void_p)], I),
            "adg_set_state": ([P, P, I64, I], I),
            "adg_init_vortex": ([P, D, D, D, D], I),
            "adg_init_tgv": ([P, D], I),
            "adg_step": ([P, I], I),
            "adg_get_state": ([P, P, I64, I], I),
            "adg_rhs": ([P, P, P, I64, I], I),
            "adg_get_schedule": ([P, I64, I, P, P, P], I),
            "adg_info": ([P, P, P, P, P], I),
            "adg_conservation": ([P, P], I),
            "adg_l2_error_vortex": ([P, D, D, D, D, P], I),
            "adg_check_finite": ([P], I),
            "adg_last_error": ([P], ctypes.c_char_p),
            "adg_destroy": ([P], None),
            "adg_set_profiling": ([P, I], I),
            "adg_get_profile": ([P, P, P], I),
            "adg_rhs_noalloc": ([ctypes.POINTER(Mesh), I, D, P, P, I64, P], I),
            "adg_checkpoint_bytes": ([P, P], I),
            "adg_checkpoint_save": ([P, P, I64], I),
            "adg_checkpoint_restore": ([P, P, I64], I),
            "adg_batch_create": ([I, P, P, P, P, I, ctypes.POINTER(Options),
                                  ctypes.POINTER(ctypes.c_void_p)], I),
            "adg_batch_init_vortex": ([P, I, D, D, D], I),
            "adg_batch_set_state": ([P, I, P, I64, I], I),
            "adg_batch_step": ([P, I], I),
            "adg_batch_autotune": ([P, I, P], I),
            "adg_batch_get_state": ([P, I, P, I64, I], I),
            "adg_batch_info": ([P, I, P, P, P, P, P], I),
            "adg_batch_l2_error_vortex": ([P, I, D, D, D, D, P], I),
            "adg_batch_num_groups": ([P], I),
            "adg_batch_last_error": ([P], ctypes.c_char_p),
            "adg_batch_destroy": ([P], None),
            "adg_mlp_num_params": ([], I),
            "adg_mlp_grad": ([P, P, P, I64, P, P, P], I),
            "adg_mlp_forward": ([P, P, I64, P, P], I),
            "adg_mlp_adam": ([P, P, P, P, P, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                              ctypes.c_float, I, P], I),
            "adg_mlp_to_bf16": ([P, P, P], I),
            "adg_set_learned_model": ([P, P, ctypes.c_float], I),
            "adg_set_trace_log": ([P, P, I64, P], I),
            "adg_learned_samples": ([P, P, I64, P, I64, P, P, P], I),
            "adg_host_gauss": ([I, P, P], I),
            "adg_host_at_coeffs": ([I, D, P], I),
            "adg_host_rk": ([I, P, P, P, P], I),
            "adg_host_schedule": ([I, I, I, I, I, P, U64, I, I64, I, P, P, P], I),
            "adg_host_num_interfaces": ([I, P], I),
            "adg_measure_peak": ([I, P, P, P], I),
            "adg_probe_wait": ([I64, P, P], I),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
        return L


def _check(st, handle=None):
    if st != 0:
        msg = lib().adg_last_error(handle)
        raise AdgError(st, msg.decode() if msg else "")


def _np_ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _buf(a, writable=False):
    """(pointer, count, on_device) of a numpy array or a CUDA torch tensor (FP64)."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host buffers must be C-contiguous float64")
        if writable and not a.flags["WRITEABLE"]:
            raise ValueError("buffer is read-only")
        return _np_ptr(a), a.size, 0
    import torch
    if not isinstance(a, torch.Tensor):
        raise TypeError("expected a numpy array or a torch tensor")
    if a.dtype != torch.float64 or not a.is_contiguous():
        raise ValueError("tensors must be contiguous float64")
    if not a.is_cuda:
        return ctypes.c_void_p(a.data_ptr()), a.numel(), 0
    return ctypes.c_void_p(a.data_ptr()), a.numel(), 1


# ---- host-only helpers ----------------------------------------------------------------

def host_gauss(n):
    x, w = np.zeros(n), np.zeros(n)
    _check(lib().adg_host_gauss(n, _np_ptr(x), _np_ptr(w)))
    return x, w


def host_at_coeffs(np_, km):
    c = np.zeros(np_ + 1)
    _check(lib().adg_host_at_coeffs(np_, km, _np_ptr(c)))
    return c


def host_rk(scheme):
    s = ctypes.c_int()
    a, b, c = np.zeros(8), np.zeros(8), np.zeros(8)
    _check(lib().adg_host_rk(RK[scheme], ctypes.byref(s), _np_ptr(a), _np_ptr(b), _np_ptr(c)))
    n = s.value
    return a[:n], b[:n], c[:n]


def host_num_interfaces(dim, P):
    Pa = (ctypes.c_int * 3)(*(list(P) + [1] * (3 - len(P))))
    return lib().adg_host_num_interfaces(dim, Pa)


def host_schedule(flux, delay_mode, max_delay, np_, P, dim, seed, dmax, n0, count):
    Pa = (ctypes.c_int * 3)(*(list(P) + [1] * (3 - len(P))))
    nif = host_num_interfaces(dim, P)
    comm = np.zeros(count, np.int32)
    k = np.zeros(count, np.int32)
    dl = np.zeros((count, max(nif, 1)), np.int32)
    _check(lib().adg_host_schedule(FLUX[flux], DELAY[delay_mode], max_delay, np_, dim, Pa,
                                   seed & 0xFFFFFFFFFFFFFFFF, dmax, n0, count, _np_ptr(comm),
                                   _np_ptr(k), _np_ptr(dl)))
    return comm, k, dl[:, :nif]


PEAK_KINDS = {"fp64_fma": 0, "fp32_fma": 1, "fp64_mma": 2, "fp64_fma+mma": 3, "fp32x2_fma": 4,
              "fp64_add": 5, "fp64_mul": 6}


def measure_peak(kind):
    """Measured arithmetic rate of one instruction kind on the current device:
    (TFLOP/s, ms of the timed launch, SM MHz during it).  Kinds: PEAK_KINDS."""
    t, ms, mhz = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().adg_measure_peak(PEAK_KINDS[kind], ctypes.byref(t), ctypes.byref(ms),
                                  ctypes.byref(mhz)))
    return t.value, ms.value, mhz.value


def probe_wait(limit_cycles):
    """adg_probe_wait: (threads that gave up of 128, cycles thread 0 waited) for a bounded
    wait on a barrier nothing arrives at."""
    n, c = ctypes.c_int(), ctypes.c_int64()
    _check(lib().adg_probe_wait(int(limit_cycles), ctypes.byref(n), ctypes.byref(c)))
    return n.value, c.value


def rhs_noalloc(dim, n_elem, degree, u, k, lo=None, hi=None, gamma=1.4, stream=None):
    """adg_rhs_noalloc on CUDA torch tensors u (read) and k (written); no allocation."""
    lo = lo if lo is not None else ((-5.0,) * dim)
    hi = hi if hi is not None else ((5.0,) * dim)
    m = Mesh()
    m.dim = dim
    for i in range(3):
        m.n_elem[i] = n_elem[i] if i < dim else 1
        m.lo[i] = lo[i] if i < dim else 0.0
        m.hi[i] = hi[i] if i < dim else 1.0
    pu, n, du = _buf(u)
    pk, nk, dk = _buf(k, writable=True)
    if not (du and dk) or n != nk:
        raise ValueError("u and k must be CUDA tensors of the same size")
    if u.device != k.device:
        raise ValueError("u and k must be on the same CUDA device")
    import torch
    # the library works on the current device: make it the tensors' device
    with torch.cuda.device(u.device):
        if stream is None:
            stream = torch.cuda.current_stream(u.device).cuda_stream
        _check(lib().adg_rhs_noalloc(ctypes.byref(m), degree, gamma, pu, pk, n, stream))


# ---- solver ---------------------------------------------------------------------------

class Solver:
    """One ADG solver on the current CUDA device (see include/adg.h)."""

    def __init__(self, dim=2, n_elem=(16, 16), lo=None, hi=None, degree=2, P=(1, 1),
                 max_delay=1, flux="sync", rk="ck45", dt=0.0, cfl=0.1, t_end=0.0, gamma=1.4,
                 delay_mode="caa", seed=0, random_delay_max=0, at_np=0, precision="fp64",
                 stream=None, kernel_path="auto"):
        L = lib()
        lo = lo if lo is not None else ((-5.0,) * dim)
        hi = hi if hi is not None else ((5.0,) * dim)
        m = Mesh()
        m.dim = dim
        for i in range(3):
            m.n_elem[i] = n_elem[i] if i < dim else 1
            m.lo[i] = lo[i] if i < dim else 0.0
            m.hi[i] = hi[i] if i < dim else 1.0
        o = Options()
        _check(L.adg_default_options(ctypes.byref(o)))
        o.rk = RK[rk]
        o.dt = dt
        o.cfl = cfl
        o.t_end = t_end
        o.gamma = gamma
        o.delay_mode = DELAY[delay_mode]
        o.seed = seed & 0xFFFFFFFFFFFFFFFF
        o.random_delay_max = random_delay_max
        o.at_np = at_np
        o.precision = PREC[precision]
        o.kernel_path = PATH[kernel_path]
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
            except ImportError:
                stream = None
        o.cuda_stream = stream
        Pa = (ctypes.c_int * 3)(*(list(P) + [1] * (3 - len(P))))
        h = ctypes.c_void_p()
        _check(L.adg_create(ctypes.byref(m), degree, Pa, max_delay, FLUX[flux], ctypes.byref(o),
                            ctypes.byref(h)))
        self._h = h
        self._L = L
        self.dim, self.degree, self.nv = dim, degree, dim + 2
        self.n_elem = tuple(n_elem[:dim])
        self.ne = int(np.prod(self.n_elem))
        self.nd = (degree + 1) ** dim
        self.shape = (self.nv, self.ne, self.nd)
        self.n_dof = self.nv * self.ne * self.nd
        self.flux, self.delay_mode, self.P = flux, delay_mode, tuple(P)

    def close(self):
        if getattr(self, "_h", None):
            self._L.adg_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _chk(self, st):
        _check(st, self._h)

    def set_state(self, u):
        p, n, dev = _buf(u)
        self._chk(self._L.adg_set_state(self._h, p, n, dev))

    def init_vortex(self, t=0.0, beta=5.0, x0=0.0, y0=0.0):
        self._chk(self._L.adg_init_vortex(self._h, t, beta, x0, y0))

    def init_tgv(self, mach=0.1):
        self._chk(self._L.adg_init_tgv(self._h, mach))

    def step(self, n=1):
        self._chk(self._L.adg_step(self._h, n))

    def get_state(self, out=None):
        if out is None:
            out = np.empty(self.shape)
        p, n, dev = _buf(out, writable=True)
        self._chk(self._L.adg_get_state(self._h, p, n, dev))
        return out

    def rhs(self, u, out=None):
        if out is None:
            out = np.empty(self.shape)
        pu, n, du = _buf(u)
        pk, nk, dk = _buf(out, writable=True)
        if du != dk or n != nk:
            raise ValueError("u and out must both be host or both be device, same size")
        self._chk(self._L.adg_rhs(self._h, pu, pk, n, du))
        return out

    def schedule(self, n0, count):
        nif = host_num_interfaces(self.dim, self.P)
        comm = np.zeros(count, np.int32)
        k = np.zeros(count, np.int32)
        dl = np.zeros((count, max(nif, 1)), np.int32)
        self._chk(self._L.adg_get_schedule(self._h, n0, count, _np_ptr(comm), _np_ptr(k), _np_ptr(dl)))
        return comm, k, dl[:, :nif]

    def info(self):
        t, dt = ctypes.c_double(), ctypes.c_double()
        st, nd = ctypes.c_int64(), ctypes.c_int64()
        self._chk(self._L.adg_info(self._h, ctypes.byref(t), ctypes.byref(st), ctypes.byref(dt),
                                   ctypes.byref(nd)))
        return dict(t=t.value, step=st.value, dt=dt.value, n_dof=nd.value)

    def conservation(self):
        s = np.zeros(self.nv)
        self._chk(self._L.adg_conservation(self._h, _np_ptr(s)))
        return s

    def l2_error_vortex(self, t, beta=5.0, x0=0.0, y0=0.0):
        e = np.zeros(3)
        self._chk(self._L.adg_l2_error_vortex(self._h, t, beta, x0, y0, _np_ptr(e)))
        return e

    def set_profiling(self, enable=True):
        self._chk(self._L.adg_set_profiling(self._h, 1 if enable else 0))

    def get_profile(self):
        """{'flux': (ms, launches), 'vol': (ms, launches)} since profiling was enabled/read."""
        ms = np.zeros(2)
        n = np.zeros(2, np.int64)
        self._chk(self._L.adg_get_profile(self._h, _np_ptr(ms), _np_ptr(n)))
        return {"flux": (float(ms[0]), int(n[0])), "vol": (float(ms[1]), int(n[1]))}

    def checkpoint(self):
        """The run state (see adg_checkpoint_save) as a numpy uint8 array."""
        n = ctypes.c_int64()
        self._chk(self._L.adg_checkpoint_bytes(self._h, ctypes.byref(n)))
        buf = np.empty(n.value, np.uint8)
        self._chk(self._L.adg_checkpoint_save(self._h, _np_ptr(buf), n.value))
        return buf

    def restore(self, buf):
        """Continue from a checkpoint taken by a compatible handle."""
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        self._chk(self._L.adg_checkpoint_restore(self._h, _np_ptr(buf), buf.size))

    def set_learned_model(self, params_bf16, trust=1.0):
        """params_bf16: numpy uint16 array of adg_mlp_num_params() BF16 values."""
        a = np.ascontiguousarray(params_bf16, dtype=np.uint16)
        if a.size != lib().adg_mlp_num_params():
            raise ValueError("wrong number of parameters")
        self._chk(self._L.adg_set_learned_model(self._h, _np_ptr(a), trust))

    def set_trace_log(self, log_tensor=None, n_records=0):
        """Log subdomain-face traces of every stage input into a CUDA float64 tensor."""
        rl = ctypes.c_int64()
        ptr = ctypes.c_void_p(log_tensor.data_ptr()) if log_tensor is not None else None
        self._chk(self._L.adg_set_trace_log(self._h, ptr, n_records, ctypes.byref(rl)))
        return rl.value

    def learned_samples(self, log_tensor, n_records, picks, x, target, ok):
        """picks: CUDA int32 [n][4]; x: CUDA float32 [n][4]; target: [n]; ok: int32 [n]."""
        self._chk(self._L.adg_learned_samples(
            self._h, ctypes.c_void_p(log_tensor.data_ptr()), n_records,
            ctypes.c_void_p(picks.data_ptr()), picks.shape[0], ctypes.c_void_p(x.data_ptr()),
            ctypes.c_void_p(target.data_ptr()), ctypes.c_void_p(ok.data_ptr())))

    def check_finite(self):
        st = self._L.adg_check_finite(self._h)
        if st == 5:
            return False
        self._chk(st)
        return True


class Batch:
    """Batched solver (include/adg.h, adg_batch_*): instances given as a list of dicts with
    keys n_elem, degree, P, max_delay (and optionally lo, hi)."""

    def __init__(self, instances, dim=2, flux="at", rk="ck45", dt=0.0, cfl=0.1, gamma=1.4,
                 delay_mode="caa", seed=0, random_delay_max=0, at_np=0, precision="fp32",
                 stream=None, kernel_path="auto"):
        L = lib()
        n = len(instances)
        meshes = (Mesh * n)()
        degs = (ctypes.c_int * n)()
        Ps = (ctypes.c_int * (3 * n))()
        Ls = (ctypes.c_int * n)()
        for i, ins in enumerate(instances):
            ne = ins["n_elem"]
            lo = ins.get("lo", (-5.0,) * dim)
            hi = ins.get("hi", (5.0,) * dim)
            meshes[i].dim = dim
            for d in range(3):
                meshes[i].n_elem[d] = ne[d] if d < dim else 1
                meshes[i].lo[d] = lo[d] if d < dim else 0.0
                meshes[i].hi[d] = hi[d] if d < dim else 1.0
                Ps[3 * i + d] = ins.get("P", (1, 1, 1))[d] if d < dim else 1
            degs[i] = ins["degree"]
            Ls[i] = ins.get("max_delay", 1)
        o = Options()
        _check(L.adg_default_options(ctypes.byref(o)))
        o.rk, o.dt, o.cfl, o.gamma = RK[rk], dt, cfl, gamma
        o.delay_mode, o.seed = DELAY[delay_mode], seed & 0xFFFFFFFFFFFFFFFF
        o.random_delay_max, o.at_np, o.precision = random_delay_max, at_np, PREC[precision]
        o.kernel_path = PATH[kernel_path]
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        o.cuda_stream = stream
        h = ctypes.c_void_p()
        st = L.adg_batch_create(n, meshes, degs, Ps, Ls, FLUX[flux], ctypes.byref(o), ctypes.byref(h))
        if st != 0:
            msg = L.adg_batch_last_error(None)
            raise AdgError(st, msg.decode() if msg else "")
        self._h, self._L, self.n, self.dim = h, L, n, dim
        self.instances = instances

    def _chk(self, st):
        if st != 0:
            msg = self._L.adg_batch_last_error(self._h)
            raise AdgError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "_h", None):
            self._L.adg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def init_vortex(self, i, beta=5.0, x0=0.0, y0=0.0):
        self._chk(self._L.adg_batch_init_vortex(self._h, i, beta, x0, y0))

    def set_state(self, i, u):
        p, n, dev = _buf(u)
        self._chk(self._L.adg_batch_set_state(self._h, i, p, n, dev))

    def step(self, n=1):
        self._chk(self._L.adg_batch_step(self._h, n))

    def autotune(self, trials=3):
        g = self._L.adg_batch_num_groups(self._h)
        out = (ctypes.c_int * max(g, 1))()
        self._chk(self._L.adg_batch_autotune(self._h, trials, out))
        return list(out)[:g]

    def info(self, i):
        t, dt = ctypes.c_double(), ctypes.c_double()
        st, nd, deg = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        self._chk(self._L.adg_batch_info(self._h, i, ctypes.byref(t), ctypes.byref(st),
                                         ctypes.byref(dt), ctypes.byref(nd), ctypes.byref(deg)))
        return dict(t=t.value, step=st.value, dt=dt.value, n_dof=nd.value, degree=deg.value)

    def get_state(self, i, out=None):
        inf = self.info(i)
        if out is None:
            nd = (inf["degree"] + 1) ** self.dim
            out = np.empty((self.dim + 2, inf["n_dof"] // ((self.dim + 2) * nd), nd))
        p, n, dev = _buf(out, writable=True)
        self._chk(self._L.adg_batch_get_state(self._h, i, p, n, dev))
        return out

    def l2_error_vortex(self, i, t, beta=5.0, x0=0.0, y0=0.0):
        e = np.zeros(3)
        self._chk(self._L.adg_batch_l2_error_vortex(self._h, i, t, beta, x0, y0, _np_ptr(e)))
        return e
