"""Helpers shared by the GPU parity tests: velocity-order mapping between the
library and the oracle, raw-storage encoding for checkpoints, error metrics.

Nothing here computes any step of the method; the expected values always come
from ``oracle``."""
import numpy as np

import oracle
from paper_2002_02503_gb300 import lbm

TOL_F32 = 1e-5   # max relative error of FP32 fields against the FP64 oracle after 100 steps
TOL_F64 = 1e-12
TOL_U16 = 1e-3   # relative error on u for shifted 16-bit storage: the accuracy target of the 16-bit forms
# Implementation parity of the 16-bit floating forms on short runs (tens of steps, white-noise or
# smooth seeded fields) against the FP64 oracle: a few units of the storage's own rounding of the
# scaled value h (2^-11 for FP16, 2^-8 for BF16, |h| up to ~0.3) over the decayed max|u|.  These
# check that the kernels compute the method; they are not the accuracy target, which the
# stated-size runs of test_gpu_storage_accuracy.py hold the storage forms to.
TOL_ROUND = {"f16": 2e-3, "bf16": 2e-2}

DIMS = {  # ragged sizes: several thread blocks per plane and a partial last block
    "D2Q9": (72, 44, 1),
    "D3Q15": (44, 22, 14),
    "D3Q19": (40, 26, 14),
    "D3Q27": (36, 22, 12),
    "D3Q39": (28, 18, 10),
}


def perm_lib_to_oracle(name):
    """perm[i_lib] = i_oracle with the same velocity vector."""
    g = lbm.lbm_lattice_info(name)["c"]
    o = [tuple(int(v) for v in c) for c in oracle.lattice(name)["c"]]
    return np.array([o.index(tuple(int(v) for v in c)) for c in g])


def to_lib_order(name, f_oracle):
    return f_oracle[perm_lib_to_oracle(name)]


def raw_from_f(name, dims, f_lib, storage, rho0=1.0):
    """Stored representation of pre-collision f (library order): g_i(y) = f_i(y + c_i), stored as
    (g_i - w_i rho0) / w_i in the storage type."""
    import torch

    info = lbm.lbm_lattice_info(name)
    nx, ny, nz = dims
    out = np.empty_like(f_lib)
    for i in range(info["Q"]):
        a = f_lib[i].reshape(nz, ny, nx)
        cx, cy, cz = info["c"][i]
        a = np.roll(a, (-cz, -cy, -cx), axis=(0, 1, 2))  # a'[y] = a[y + c]
        out[i] = a.reshape(-1) - info["w"][i] * rho0
    scaled = out / info["w"][:, None]  # every storage form holds (g - w rho0) / w
    if storage == "f64":
        return scaled.astype(np.float64)
    if storage == "f32":
        return scaled.astype(np.float32)
    if storage == "f16":
        return scaled.astype(np.float16)
    if storage == "bf16":
        return torch.from_numpy(scaled.astype(np.float32)).to(torch.bfloat16).view(torch.int16).numpy()
    raise ValueError(storage)


def rel_f(got, want):
    return float(np.max(np.abs(got - want) / np.abs(want)))


def rel_u(got, want):
    return float(np.max(np.abs(got - want)) / max(np.max(np.abs(want)), 1e-300))


def oracle_reference(name, K, tau, dims, rho, u, steps):
    f0 = oracle.init_eq(name, K, dims, rho, u)
    f = oracle.run(name, K, tau, dims, f0, steps)
    r, uu = oracle.moments(name, dims, f)
    return f, r, uu
