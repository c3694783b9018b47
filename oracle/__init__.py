"""FP64 CPU oracle for the Galilean-invariant filtered LB collision (arXiv 2002.02503).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the CUDA product path, and it
shares no code with it.  The arithmetic lives in ``lbm_oracle.c`` (see its
header for the paper's steps it follows); this module only marshals numpy
arrays through ctypes.

Array conventions: distributions ``f`` are ``[Q, C]`` float64 with
``cell = x + nx*(y + ny*z)``; ``rho`` is ``[C]``; ``u`` is ``[D, C]``.  The
velocity ordering is the oracle's own (``lattice(name)["c"]``).
"""
import ctypes
import os

import numpy as np

from . import build as _build

LATTICES = {"D2Q9": 0, "D3Q19": 1, "D3Q27": 2, "D3Q39": 3, "D3Q15": 4}
MAX_K = 10

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.orc_lattice.argtypes = [ctypes.c_int, ip, ip, dp, ip, dp]
        lib.orc_hermite.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
        lib.orc_feq.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp]
        lib.orc_fneq_hat.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
        lib.orc_collide.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp, dp, dp, dp, dp, dp]
        lib.orc_init_eq.argtypes = [ctypes.c_int, ctypes.c_int, i64p, dp, dp, dp, ctypes.c_int]
        lib.orc_moments.argtypes = [ctypes.c_int, i64p, dp, dp, dp]
        lib.orc_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, i64p, dp, ctypes.c_int64, ctypes.c_int]
        lib.orc_run_model.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                      i64p, dp, ctypes.c_int64, ctypes.c_int]
        lib.orc_fneq_hat_q.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
        lib.orc_collide_theta.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp, dp,
                                          dp]
        lib.orc_collide_bgk.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp]
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc, what):
    if rc != 0:
        raise ValueError("oracle %s failed with code %d" % (what, rc))


def _lat(name):
    if name not in LATTICES:
        raise ValueError("unknown lattice %r" % (name,))
    return LATTICES[name]


def lattice(name):
    """Tables of the named lattice: dict(D, Q, T0, c [Q,3] int, w [Q])."""
    lib = _load()
    D, Q, T0 = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    c = np.zeros((39, 3), dtype=np.int32)
    w = np.zeros(39)
    rc = lib.orc_lattice(_lat(name), ctypes.byref(D), ctypes.byref(Q), ctypes.byref(T0),
                         c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w))
    _check(rc, "lattice")
    q = Q.value
    return {"D": D.value, "Q": q, "T0": T0.value, "c": c[:q].copy(), "w": w[:q].copy()}


def hermite(name, i, n):
    """Tensor Hermite polynomial H^(n)(xi_i) of velocity i (Eq. recurG), shape (D,)*n."""
    lat = lattice(name)
    D = lat["D"]
    out = np.zeros(D ** n)
    _check(_load().orc_hermite(_lat(name), int(i), int(n), _dp(out)), "hermite")
    return out.reshape((D,) * n) if n > 0 else out.reshape(())


def _u3(u):
    v = np.zeros(3)
    v[: len(u)] = u
    return v


def feq(name, K, rho, u):
    """Truncated equilibrium of Eq. hermite at one cell (float64 [Q])."""
    Q = lattice(name)["Q"]
    out = np.zeros(Q)
    uu = _u3(u)
    _check(_load().orc_feq(_lat(name), int(K), float(rho), _dp(uu), _dp(out)), "feq")
    return out


def fneq_hat(name, K, u, Pi):
    """Truncated filtered non-equilibrium part of Eq. hermite-coll at one cell."""
    Q = lattice(name)["Q"]
    out = np.zeros(Q)
    uu = _u3(u)
    P = np.zeros((3, 3))
    Pi = np.asarray(Pi, dtype=np.float64)
    P[: Pi.shape[0], : Pi.shape[1]] = Pi
    _check(_load().orc_fneq_hat(_lat(name), int(K), _dp(uu), _dp(P), _dp(out)), "fneq_hat")
    return out


def collide(name, K, tau, f):
    """One cell through Eq. mme, hermite, neq, Pi_def, hermite-coll and lbe-reg.

    Returns dict(fpost, rho, u, feq, Pi, fhat)."""
    Q = lattice(name)["Q"]
    f = np.ascontiguousarray(f, dtype=np.float64)
    fpost, feq_, fhat = np.zeros(Q), np.zeros(Q), np.zeros(Q)
    rho = ctypes.c_double()
    u = np.zeros(3)
    Pi = np.zeros(9)
    rc = _load().orc_collide(_lat(name), int(K), float(tau), _dp(f), _dp(fpost),
                             ctypes.cast(ctypes.byref(rho), ctypes.POINTER(ctypes.c_double)),
                             _dp(u), _dp(feq_), _dp(Pi), _dp(fhat))
    _check(rc, "collide")
    return {"fpost": fpost, "rho": rho.value, "u": u, "feq": feq_, "Pi": Pi.reshape(3, 3), "fhat": fhat}


def _dims(dims):
    d = np.ones(3, dtype=np.int64)
    d[: len(dims)] = dims
    return d


def init_eq(name, K, dims, rho, u, nthreads=None):
    """f := f^eq_K(rho, u) everywhere.  rho [C], u [D, C] -> f [Q, C]."""
    lat = lattice(name)
    d = _dims(dims)
    C = int(np.prod(d))
    rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(C)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(lat["D"], C)
    f = np.zeros((lat["Q"], C))
    nt = default_threads() if nthreads is None else int(nthreads)
    rc = _load().orc_init_eq(_lat(name), int(K), d.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                             _dp(rho), _dp(u), _dp(f), nt)
    _check(rc, "init_eq")
    return f


def moments(name, dims, f):
    """(rho [C], u [D, C]) of distributions f [Q, C] (Eq. mme)."""
    lat = lattice(name)
    d = _dims(dims)
    C = int(np.prod(d))
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(lat["Q"], C)
    rho = np.zeros(C)
    u = np.zeros((lat["D"], C))
    rc = _load().orc_moments(_lat(name), d.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(f), _dp(rho), _dp(u))
    _check(rc, "moments")
    return rho, u


def default_threads():
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return max(1, os.cpu_count() or 1)


MODELS = {"filtered": 0, "bgk": 1}


def collide_bgk(name, K, tau, f):
    """One cell with the BGK operator (Eq. BGK) and the truncated f^eq."""
    Q = lattice(name)["Q"]
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(Q)
    _check(_load().orc_collide_bgk(_lat(name), int(K), float(tau), _dp(f), _dp(out)), "collide_bgk")
    return out


def fneq_hat_q(name, K, u, Qt):
    """Truncated energy-flux filtered part fhat^{neq,q} (Eq. pq series) at one cell."""
    Q = lattice(name)["Q"]
    out = np.zeros(Q)
    uu = _u3(u)
    T = np.zeros((3, 3, 3))
    Qt = np.asarray(Qt, dtype=np.float64)
    d = Qt.shape[0]
    T[:d, :d, :d] = Qt
    _check(_load().orc_fneq_hat_q(_lat(name), int(K), _dp(uu), _dp(T), _dp(out)), "fneq_hat_q")
    return out


def collide_theta(name, K, tau, theta, f):
    """One cell of the filtered collision with the energy-flux term: dict(fpost, Qt, fhatq)."""
    Q = lattice(name)["Q"]
    f = np.ascontiguousarray(f, dtype=np.float64)
    fpost, fhq = np.zeros(Q), np.zeros(Q)
    Qt = np.zeros(27)
    _check(_load().orc_collide_theta(_lat(name), int(K), float(tau), float(theta), _dp(f), _dp(fpost), _dp(Qt),
                                     _dp(fhq)), "collide_theta")
    return {"fpost": fpost, "Qt": Qt.reshape(3, 3, 3), "fhatq": fhq}


def run(name, K, tau, dims, f, nsteps, nthreads=None, model="filtered", theta=0.0):
    """Advance f [Q, C] by nsteps of collide + push (Eq. lbe-reg, optionally with the energy-flux
    term theta of Eq. pq, or Eq. BGK with model="bgk"; then Eq. lbe); returns a new array."""
    lat = lattice(name)
    d = _dims(dims)
    C = int(np.prod(d))
    out = np.array(f, dtype=np.float64, copy=True).reshape(lat["Q"], C)
    out = np.ascontiguousarray(out)
    nt = default_threads() if nthreads is None else int(nthreads)
    rc = _load().orc_run_model(_lat(name), int(K), float(tau), MODELS[model], float(theta),
                               d.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(out), int(nsteps), nt)
    _check(rc, "run")
    return out
