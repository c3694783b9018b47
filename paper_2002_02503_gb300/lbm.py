"""Python binding of the C-ABI in ``include/lbm.h`` (ctypes; argument marshalling only).

Every function below has the C name and forwards to ``liblbm_gb300.so``; all
arithmetic of the method runs in the library's CUDA kernels.  PyTorch is used
only to own device memory (the workspace) and to supply CUDA streams.  If the
library is missing the import of any entry point raises: there is no CPU path.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# LBM_BOUNDS_CHECK=1 selects the bounds-check build (every kernel checks its indices; an index
# outside its buffer is reported as LBM_ERR_BOUNDS); built by build.build(bounds_check=True)
BOUNDS_CHECK = os.environ.get("LBM_BOUNDS_CHECK", "") not in ("", "0")
LIB_PATH = os.path.join(HERE, "liblbm_gb300_bounds.so" if BOUNDS_CHECK else "liblbm_gb300.so")

LBM_OK, LBM_ERR_INVALID_ARG, LBM_ERR_UNSUPPORTED, LBM_ERR_OUT_OF_MEMORY = 0, 1, 2, 3
LBM_ERR_CUDA, LBM_ERR_NONFINITE, LBM_ERR_TIMEOUT, LBM_ERR_BUSY, LBM_ERR_NOT_FOUND = 4, 5, 6, 7, 8
LBM_ERR_RANGE, LBM_ERR_BOUNDS = 9, 10
LATTICES = {"D2Q9": 0, "D3Q19": 1, "D3Q27": 2, "D3Q39": 3, "D3Q15": 4}
STORAGES = {"f32": 0, "f16": 1, "bf16": 2, "f64": 3, "q16": 4, "f16r": 5, "bf16r": 6}
STORAGE_BYTES = {"f32": 4, "f16": 2, "bf16": 2, "f64": 8, "q16": 2, "f16r": 2, "bf16r": 2}
# forms that store D planes of a per-cell reference velocity after the Q distribution planes
REFERENCE_FORMS = ("f16r", "bf16r")
MEM_HOST, MEM_DEVICE = 0, 1

# (name, restype, argtypes) of every exported entry point of include/lbm.h
_c = ctypes
_P = _c.c_void_p
_I64P = _c.POINTER(_c.c_int64)
_DP = _c.POINTER(_c.c_double)
_IP = _c.POINTER(_c.c_int)
SIGNATURES = [
    ("lbm_lattice_info", _c.c_int, [_c.c_int, _IP, _IP, _IP, _DP, _DP, _IP]),
    ("lbm_workspace_bytes", _c.c_size_t, [_c.c_int, _I64P, _c.c_int]),
    ("lbm_create", _c.c_int, [_c.c_int, _I64P, _c.c_double, _c.c_int, _c.c_int, _c.c_double, _P, _c.c_size_t, _P,
                              _c.POINTER(_P)]),
    ("lbm_set_fields", _c.c_int, [_P, _P, _P, _c.c_int]),
    ("lbm_step", _c.c_int, [_P, _c.c_int64]),
    ("lbm_get_moments", _c.c_int, [_P, _P, _P, _c.c_int]),
    ("lbm_get_f", _c.c_int, [_P, _P, _c.c_int]),
    ("lbm_conservation", _c.c_int, [_P, _DP]),
    ("lbm_mode_amplitude", _c.c_int, [_P, _I64P, _c.c_int, _DP]),
    ("lbm_get_distributions", _c.c_int, [_P, _P, _c.c_size_t, _c.c_int, _I64P]),
    ("lbm_set_distributions", _c.c_int, [_P, _P, _c.c_size_t, _c.c_int, _c.c_int64]),
    ("lbm_time", _c.c_int, [_P, _I64P]),
    ("lbm_set_kernel", _c.c_int, [_P, _c.c_int, _c.c_int, _c.c_int]),
    ("lbm_get_kernel", _c.c_int, [_P, _IP, _IP, _IP]),
    ("lbm_set_collision", _c.c_int, [_P, _c.c_int]),
    ("lbm_set_energy_flux", _c.c_int, [_P, _c.c_double]),
    ("lbm_set_storage_range", _c.c_int, [_P, _c.c_double]),
    ("lbm_get_storage_range", _c.c_int, [_P, _DP]),
    ("lbm_set_storage_reference", _c.c_int, [_P, _DP]),
    ("lbm_autotune", _c.c_int, [_P, _c.c_int, _DP]),
    ("lbm_conservation_noalloc", _c.c_int, [_c.c_int, _c.c_int, _I64P, _c.c_double, _P, _P, _c.c_int, _P]),
    ("lbm_bounds_checked", _c.c_int, []),
    ("lbm_bounds_walk", _c.c_int64, [_c.c_int, _c.c_int, _I64P, _c.c_int64, _c.POINTER(_c.c_int64)]),
    ("lbm_destroy", _c.c_int, [_P]),
    ("lbm_pool_request_bytes", _c.c_size_t, [_c.c_int, _I64P, _c.c_int]),
    ("lbm_pool_create", _c.c_int, [_c.c_int, _c.c_int, _c.c_int, _P, _c.c_size_t, _c.c_int, _P, _P, _c.POINTER(_P)]),
    ("lbm_pool_submit", _c.c_int, [_P, _I64P, _c.c_double, _c.c_double, _P, _P, _c.c_int, _c.c_int64,
                                   _c.POINTER(_c.c_int64)]),
    ("lbm_pool_advance", _c.c_int, [_P, _c.c_int64, _IP]),
    ("lbm_pool_poll", _c.c_int, [_P, _c.c_int64, _IP, _c.POINTER(_c.c_int64)]),
    ("lbm_pool_result", _c.c_int, [_P, _c.c_int64, _P, _P, _c.c_int]),
    ("lbm_pool_cancel", _c.c_int, [_P, _c.c_int64]),
    ("lbm_pool_sync", _c.c_int, [_P]),
    ("lbm_pool_stats", _c.c_int, [_P, _c.POINTER(_c.c_size_t), _IP, _IP]),
    ("lbm_pool_set_storage_range", _c.c_int, [_P, _c.c_double]),
    ("lbm_pool_get_storage_range", _c.c_int, [_P, _DP]),
    ("lbm_pool_request_range", _c.c_int, [_P, _c.c_int64, _DP]),
    ("lbm_pool_set_kernel", _c.c_int, [_P, _c.c_int, _c.c_int]),
    ("lbm_pool_get_kernel", _c.c_int, [_P, _IP, _IP]),
    ("lbm_pool_autotune", _c.c_int, [_P, _c.c_int, _DP]),
    ("lbm_pool_destroy", _c.c_int, [_P]),
    ("lbm_status_string", _c.c_char_p, [_c.c_int]),
    ("lbm_last_error", _c.c_char_p, []),
]

_lib = None


class LbmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s (status %d): %s" % (_status_name(status), status, message))
        self.status = status


def _status_name(status):
    names = {0: "LBM_OK", 1: "LBM_ERR_INVALID_ARG", 2: "LBM_ERR_UNSUPPORTED", 3: "LBM_ERR_OUT_OF_MEMORY",
             4: "LBM_ERR_CUDA", 5: "LBM_ERR_NONFINITE", 6: "LBM_ERR_TIMEOUT", 7: "LBM_ERR_BUSY",
             8: "LBM_ERR_NOT_FOUND", 9: "LBM_ERR_RANGE", 10: "LBM_ERR_BOUNDS"}
    return names.get(status, "LBM_STATUS_%d" % status)


def lib():
    """The loaded CUDA library.  Raises if it has not been built: there is no fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("%s is not built (run __graft_entry__.build(); the bounds-check build: "
                               "build.build(bounds_check=True)); the CUDA library is the only implementation"
                               % os.path.basename(LIB_PATH))
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != LBM_OK:
        msg = lib().lbm_last_error()
        raise LbmError(status, msg.decode() if msg else "")


def _lat(lattice):
    return LATTICES[lattice] if isinstance(lattice, str) else int(lattice)


def _st(storage):
    return STORAGES[storage] if isinstance(storage, str) else int(storage)


def _dims(dims):
    d = (list(dims) + [1, 1, 1])[:3]
    return (ctypes.c_int64 * 3)(*[int(x) for x in d])


def _ptr(a):
    """(pointer, mem) of a numpy array (host) or a torch tensor (host or CUDA)."""
    if a is None:
        return None, MEM_HOST
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data, MEM_HOST
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr(), (MEM_DEVICE if a.is_cuda else MEM_HOST)
    raise TypeError("expected a numpy array or a torch tensor")


# ----------------------------------------------------------------- C entry points
def lbm_lattice_info(lattice):
    D, Q, kmax = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    T0 = ctypes.c_double()
    c = (ctypes.c_int * (39 * 3))()
    w = (ctypes.c_double * 39)()
    _check(lib().lbm_lattice_info(_lat(lattice), ctypes.byref(D), ctypes.byref(Q), c, w, ctypes.byref(T0),
                                  ctypes.byref(kmax)))
    q = Q.value
    return {"D": D.value, "Q": q, "T0": T0.value, "kmax": kmax.value,
            "c": np.array(c[: 3 * q], dtype=np.int64).reshape(q, 3), "w": np.array(w[:q])}


def lbm_workspace_bytes(lattice, dims, storage):
    return int(lib().lbm_workspace_bytes(_lat(lattice), _dims(dims), _st(storage)))


def lbm_create(lattice, dims, tau, truncation_order, storage, rho0, workspace_ptr, workspace_bytes, stream_ptr):
    h = ctypes.c_void_p()
    _check(lib().lbm_create(_lat(lattice), _dims(dims), float(tau), int(truncation_order), _st(storage), float(rho0),
                            ctypes.c_void_p(workspace_ptr), int(workspace_bytes), ctypes.c_void_p(stream_ptr),
                            ctypes.byref(h)))
    return h


def lbm_set_fields(h, rho, u):
    pr, mr = _ptr(rho)
    pu, mu = _ptr(u)
    if mr != mu:
        raise ValueError("rho and u must both be host or both be device memory")
    _check(lib().lbm_set_fields(h, pr, pu, mr))


def lbm_step(h, n):
    _check(lib().lbm_step(h, int(n)))


def lbm_get_moments(h, rho, u):
    pr, mr = _ptr(rho)
    pu, mu = _ptr(u)
    mem = mr if rho is not None else mu
    _check(lib().lbm_get_moments(h, pr, pu, mem))


def lbm_get_f(h, f):
    p, m = _ptr(f)
    _check(lib().lbm_get_f(h, p, m))


def lbm_conservation(h):
    out = (ctypes.c_double * 4)()
    _check(lib().lbm_conservation(h, out))
    return np.array(out[:])


def lbm_mode_amplitude(h, k, component):
    out = (ctypes.c_double * 2)()
    _check(lib().lbm_mode_amplitude(h, _dims(k), int(component), out))
    return complex(out[0], out[1])


def lbm_get_distributions(h, dst):
    p, m = _ptr(dst)
    t = ctypes.c_int64()
    nbytes = dst.nbytes if isinstance(dst, np.ndarray) else dst.numel() * dst.element_size()
    _check(lib().lbm_get_distributions(h, p, nbytes, m, ctypes.byref(t)))
    return t.value


def lbm_set_distributions(h, src, t):
    p, m = _ptr(src)
    nbytes = src.nbytes if isinstance(src, np.ndarray) else src.numel() * src.element_size()
    _check(lib().lbm_set_distributions(h, p, nbytes, m, int(t)))


def lbm_time(h):
    t = ctypes.c_int64()
    _check(lib().lbm_time(h, ctypes.byref(t)))
    return t.value


def lbm_set_kernel(h, variant=-1, cells_per_thread=0, block_threads=0):
    _check(lib().lbm_set_kernel(h, int(variant), int(cells_per_thread), int(block_threads)))


def lbm_get_kernel(h):
    v, c, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().lbm_get_kernel(h, ctypes.byref(v), ctypes.byref(c), ctypes.byref(b)))
    return v.value, c.value, b.value


COLLISIONS = {"filtered": 0, "bgk": 1}


def lbm_set_collision(h, model):
    _check(lib().lbm_set_collision(h, COLLISIONS[model] if isinstance(model, str) else int(model)))


def lbm_set_energy_flux(h, theta):
    _check(lib().lbm_set_energy_flux(h, float(theta)))


def lbm_set_storage_range(h, R):
    _check(lib().lbm_set_storage_range(h, float(R)))


def lbm_set_storage_reference(h, U):
    arr = (ctypes.c_double * 3)(*[float(x) for x in (list(U) + [0.0, 0.0, 0.0])[:3]])
    _check(lib().lbm_set_storage_reference(h, arr))


def lbm_get_storage_range(h):
    r = ctypes.c_double()
    _check(lib().lbm_get_storage_range(h, ctypes.byref(r)))
    return r.value


def lbm_autotune(h, iters=10):
    us = ctypes.c_double()
    _check(lib().lbm_autotune(h, int(iters), ctypes.byref(us)))
    return us.value


def lbm_conservation_noalloc(lattice, storage, dims, rho0, distributions, out, stream_ptr=0):
    """Allocation-free conservation sums over caller-owned stored distributions (device).

    ``out``: a float64 array/tensor of 4 elements (host or device)."""
    pd, md = _ptr(distributions)
    if md != MEM_DEVICE:
        raise ValueError("distributions must be device memory")
    po, mo = _ptr(out)
    _check(lib().lbm_conservation_noalloc(_lat(lattice), _st(storage), _dims(dims), float(rho0), pd, po, mo,
                                          ctypes.c_void_p(stream_ptr)))


def lbm_bounds_checked():
    return bool(lib().lbm_bounds_checked())


def lbm_bounds_walk(lattice, cells_per_thread, dims, P):
    """(accesses outside their plane, accesses checked) of one register-pull launch (host only)."""
    n = ctypes.c_int64()
    bad = lib().lbm_bounds_walk(_lat(lattice), int(cells_per_thread), _dims(dims), int(P), ctypes.byref(n))
    if bad < 0:
        raise LbmError(LBM_ERR_INVALID_ARG, "lbm_bounds_walk: invalid arguments")
    return int(bad), int(n.value)


def lbm_destroy(h):
    _check(lib().lbm_destroy(h))


# ----------------------------------------------------------------- convenience owner
class Solver:
    """Owns a solver handle plus its device workspace (a torch uint8 tensor).

    ``stream`` is a ``torch.cuda.Stream`` (default: the current stream).  ``storage_range``
    sets the range of the fixed-point storage ("q16"; a power of two, default 1, 0 = automatic)
    and ``storage_reference`` its reference velocity (the shift of the stored values)."""

    def __init__(self, lattice, dims, tau, K, storage="f32", rho0=1.0, stream=None, device=None,
                 storage_range=None, storage_reference=None):
        import torch

        self.lattice = lattice
        self.dims = tuple((list(dims) + [1, 1, 1])[:3])
        self.info = lbm_lattice_info(lattice)
        self.storage = storage
        self.C = int(np.prod(self.dims))
        nbytes = lbm_workspace_bytes(lattice, self.dims, storage)
        if nbytes == 0:
            raise LbmError(LBM_ERR_INVALID_ARG, "invalid lattice, dims or storage")
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.handle = lbm_create(lattice, self.dims, tau, K, storage, rho0, self.workspace.data_ptr(), nbytes,
                                 self.stream.cuda_stream)
        if storage_range is not None:
            lbm_set_storage_range(self.handle, storage_range)
        if storage_reference is not None:
            lbm_set_storage_reference(self.handle, storage_reference)

    def close(self):
        if getattr(self, "handle", None) is not None:
            lbm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_fields(self, rho, u):
        lbm_set_fields(self.handle, rho, u)

    def step(self, n=1):
        lbm_step(self.handle, n)

    def moments(self):
        D = self.info["D"]
        rho = np.empty(self.C)
        u = np.empty((D, self.C))
        lbm_get_moments(self.handle, rho, u)
        return rho, u

    def f(self):
        out = np.empty((self.info["Q"], self.C))
        lbm_get_f(self.handle, out)
        return out

    def conservation(self):
        return lbm_conservation(self.handle)

    def mode(self, k, component):
        return lbm_mode_amplitude(self.handle, k, component)

    def time(self):
        return lbm_time(self.handle)

    def raw_bytes(self):
        planes = self.info["Q"] + (self.info["D"] if self.storage in REFERENCE_FORMS else 0)
        return planes * self.C * STORAGE_BYTES[self.storage]

    def autotune(self, iters=10):
        return lbm_autotune(self.handle, iters)

    def set_kernel(self, variant=-1, cells_per_thread=0, block_threads=0):
        lbm_set_kernel(self.handle, variant, cells_per_thread, block_threads)

    def kernel(self):
        return lbm_get_kernel(self.handle)

    def set_collision(self, model):
        lbm_set_collision(self.handle, model)

    def set_energy_flux(self, theta):
        lbm_set_energy_flux(self.handle, theta)

    def checkpoint(self):
        """(raw stored distributions as a uint8 array, step counter)."""
        raw = np.empty(self.raw_bytes(), dtype=np.uint8)
        t = lbm_get_distributions(self.handle, raw)
        return raw, t

    def restore(self, raw, t):
        lbm_set_distributions(self.handle, raw, t)


# ----------------------------------------------------------------- pool (batched / served solves)
def lbm_pool_request_bytes(lattice, dims, storage):
    return int(lib().lbm_pool_request_bytes(_lat(lattice), _dims(dims), _st(storage)))


def lbm_pool_create(lattice, truncation_order, storage, arena_ptr, arena_bytes, max_slots, compute_stream_ptr=0,
                    io_stream_ptr=0):
    h = ctypes.c_void_p()
    _check(lib().lbm_pool_create(_lat(lattice), int(truncation_order), _st(storage), ctypes.c_void_p(arena_ptr),
                                 int(arena_bytes), int(max_slots), ctypes.c_void_p(compute_stream_ptr),
                                 ctypes.c_void_p(io_stream_ptr), ctypes.byref(h)))
    return h


def lbm_pool_submit(h, dims, tau, rho0, rho, u, steps):
    """Returns the request id, or None when the pool is busy (LBM_ERR_BUSY)."""
    pr, mr = _ptr(rho)
    pu, mu = _ptr(u)
    if mr != mu:
        raise ValueError("rho and u must both be host or both be device memory")
    rid = ctypes.c_int64()
    st = lib().lbm_pool_submit(h, _dims(dims), float(tau), float(rho0), pr, pu, mr, int(steps), ctypes.byref(rid))
    if st == LBM_ERR_BUSY:
        return None
    _check(st)
    return rid.value


def lbm_pool_advance(h, chunk_steps):
    n = ctypes.c_int()
    _check(lib().lbm_pool_advance(h, int(chunk_steps), ctypes.byref(n)))
    return n.value


def lbm_pool_poll(h, rid):
    d = ctypes.c_int()
    sd = ctypes.c_int64()
    _check(lib().lbm_pool_poll(h, int(rid), ctypes.byref(d), ctypes.byref(sd)))
    return bool(d.value), sd.value


def lbm_pool_result(h, rid, rho, u):
    pr, mr = _ptr(rho)
    pu, mu = _ptr(u)
    mem = mr if rho is not None else mu
    _check(lib().lbm_pool_result(h, int(rid), pr, pu, mem))


def lbm_pool_sync(h):
    _check(lib().lbm_pool_sync(h))


def lbm_pool_stats(h):
    fb = ctypes.c_size_t()
    res, dn = ctypes.c_int(), ctypes.c_int()
    _check(lib().lbm_pool_stats(h, ctypes.byref(fb), ctypes.byref(res), ctypes.byref(dn)))
    return {"free_bytes": fb.value, "resident": res.value, "done": dn.value}


def lbm_pool_cancel(h, rid):
    _check(lib().lbm_pool_cancel(h, int(rid)))


def lbm_pool_set_storage_range(h, R):
    _check(lib().lbm_pool_set_storage_range(h, float(R)))


def lbm_pool_get_storage_range(h):
    r = ctypes.c_double()
    _check(lib().lbm_pool_get_storage_range(h, ctypes.byref(r)))
    return r.value


def lbm_pool_request_range(h, rid):
    r = ctypes.c_double()
    _check(lib().lbm_pool_request_range(h, int(rid), ctypes.byref(r)))
    return r.value


def lbm_pool_set_kernel(h, cells_per_thread=0, block_threads=0):
    _check(lib().lbm_pool_set_kernel(h, int(cells_per_thread), int(block_threads)))


def lbm_pool_get_kernel(h):
    cpt, block = ctypes.c_int(), ctypes.c_int()
    _check(lib().lbm_pool_get_kernel(h, ctypes.byref(cpt), ctypes.byref(block)))
    return cpt.value, block.value


def lbm_pool_autotune(h, iters=5):
    us = ctypes.c_double()
    _check(lib().lbm_pool_autotune(h, int(iters), ctypes.byref(us)))
    return us.value


def lbm_pool_destroy(h):
    _check(lib().lbm_pool_destroy(h))


class Pool:
    """Owns a pool handle plus its device arena (a torch uint8 tensor) and two streams
    (compute: the batched steps; io: uploads and result downloads).  ``storage_range`` sets
    the range of a fixed-point pool ("q16")."""

    def __init__(self, lattice, K, storage, arena_bytes, max_slots=256, device=None, storage_range=None):
        import torch

        self.lattice = lattice
        self.info = lbm_lattice_info(lattice)
        self.storage = storage
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.compute = torch.cuda.Stream(dev)
        self.io = torch.cuda.Stream(dev)
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=dev)
        self.handle = lbm_pool_create(lattice, K, storage, self.arena.data_ptr(), int(arena_bytes), max_slots,
                                      self.compute.cuda_stream, self.io.cuda_stream)
        if storage_range is not None:
            lbm_pool_set_storage_range(self.handle, storage_range)

    def close(self):
        if getattr(self, "handle", None) is not None:
            lbm_pool_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, dims, tau, rho, u, steps, rho0=1.0):
        return lbm_pool_submit(self.handle, dims, tau, rho0, rho, u, steps)

    def advance(self, chunk):
        return lbm_pool_advance(self.handle, chunk)

    def poll(self, rid):
        return lbm_pool_poll(self.handle, rid)

    def result(self, rid, C):
        rho = np.empty(C)
        u = np.empty((self.info["D"], C))
        lbm_pool_result(self.handle, rid, rho, u)
        return rho, u

    def sync(self):
        lbm_pool_sync(self.handle)

    def stats(self):
        return lbm_pool_stats(self.handle)

    def cancel(self, rid):
        lbm_pool_cancel(self.handle, rid)

    def autotune(self, iters=5):
        return lbm_pool_autotune(self.handle, iters)

    def set_kernel(self, cells_per_thread=0, block_threads=0):
        lbm_pool_set_kernel(self.handle, cells_per_thread, block_threads)

    def kernel(self):
        return lbm_pool_get_kernel(self.handle)
