"""The C-ABI library loads, exports every entry point include/lbm.h declares, and
validates arguments on the host before any device work (no GPU needed).

No compute call is made here: only table queries and argument rejections."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2002_02503_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(lbm.LIB_PATH):
        from paper_2002_02503_gb300 import build
        build.build()
    return lbm.lib()


def test_every_declared_symbol_is_exported_and_bound(L):
    declared = _declared()
    assert len(declared) >= 18
    for name in declared:
        assert hasattr(L, name), name
    bound = {n for n, _, _ in lbm.SIGNATURES}
    assert declared <= bound, declared - bound


def test_lattice_tables_match_oracle_velocity_sets(L):
    for name in lbm.LATTICES:
        g = lbm.lbm_lattice_info(name)
        o = oracle.lattice(name)
        assert g["Q"] == o["Q"] and g["D"] == o["D"] and g["T0"] == o["T0"]
        gw = {tuple(c): w for c, w in zip(g["c"], g["w"])}
        ow = {tuple(int(v) for v in c): w for c, w in zip(o["c"], o["w"])}
        assert gw.keys() == ow.keys()
        for k in gw:
            assert abs(gw[k] - ow[k]) < 1e-16
        # pair order: rest first, then (+c, -c) adjacent
        assert not g["c"][0].any()
        for p in range((g["Q"] - 1) // 2):
            np.testing.assert_array_equal(g["c"][2 * p + 1], -g["c"][2 * p + 2])
    assert [lbm.lbm_lattice_info(n)["kmax"] for n in lbm.LATTICES] == [3, 3, 3, 5, 3]


def test_workspace_bytes(L):
    n = lbm.lbm_workspace_bytes("D3Q19", (256, 256, 256), "f32")
    assert n >= 2 * 19 * 256 ** 3 * 4
    assert n < 2 * 19 * 256 ** 3 * 4 + (1 << 20)
    assert lbm.lbm_workspace_bytes("D3Q19", (256, 256, 256), "f16") < n // 2 + (1 << 20)
    assert lbm.lbm_workspace_bytes("D2Q9", (64, 64, 2), "f32") == 0  # 2-D needs nz == 1
    assert lbm.lbm_workspace_bytes("D3Q39", (2, 8, 8), "f32") == 0   # dims >= max|c| = 3


def _create_status(lattice="D3Q19", dims=(8, 8, 8), tau=0.6, K=3, storage="f32", rho0=1.0, ws=4096 * 256,
                   nbytes=None):
    h = ctypes.c_void_p()
    if nbytes is None:
        nbytes = 1 << 40
    d = (ctypes.c_int64 * 3)(*dims)
    return lbm.lib().lbm_create(lbm.LATTICES[lattice], d, tau, K, lbm.STORAGES[storage], rho0,
                                ctypes.c_void_p(ws), nbytes, None, ctypes.byref(h)), h


def test_create_rejects_bad_arguments_before_device_work(L):
    assert _create_status(tau=0.5)[0] == lbm.LBM_ERR_INVALID_ARG
    assert _create_status(tau=float("nan"))[0] == lbm.LBM_ERR_INVALID_ARG
    assert _create_status(K=4)[0] == lbm.LBM_ERR_UNSUPPORTED        # D3Q19 supports K <= 3
    assert _create_status(K=1)[0] == lbm.LBM_ERR_UNSUPPORTED
    assert _create_status(lattice="D3Q39", K=6)[0] == lbm.LBM_ERR_UNSUPPORTED
    assert _create_status(ws=0)[0] == lbm.LBM_ERR_INVALID_ARG
    assert _create_status(ws=4096 * 256 + 8)[0] == lbm.LBM_ERR_INVALID_ARG  # misaligned
    assert _create_status(nbytes=1024)[0] == lbm.LBM_ERR_OUT_OF_MEMORY
    assert _create_status(lattice="D2Q9", dims=(8, 8, 2))[0] == lbm.LBM_ERR_INVALID_ARG
    assert _create_status(lattice="D3Q39", dims=(8, 2, 8), K=4)[0] == lbm.LBM_ERR_INVALID_ARG
    assert _create_status(rho0=0.0)[0] == lbm.LBM_ERR_INVALID_ARG
    st, h = _create_status(tau=0.4)
    assert h.value is None
    assert b"tau" in lbm.lib().lbm_last_error()


def test_null_solver_is_rejected(L):
    assert lbm.lib().lbm_step(None, 1) == lbm.LBM_ERR_INVALID_ARG
    assert lbm.lib().lbm_destroy(None) == lbm.LBM_OK
    assert lbm.lib().lbm_pool_set_kernel(None, 2, 128) == lbm.LBM_ERR_INVALID_ARG
    assert lbm.lib().lbm_pool_get_kernel(None, None, None) == lbm.LBM_ERR_INVALID_ARG
    assert lbm.lib().lbm_pool_cancel(None, 0) == lbm.LBM_ERR_INVALID_ARG
    assert lbm.lib().lbm_get_storage_range(None, None) == lbm.LBM_ERR_INVALID_ARG
    assert lbm.lib().lbm_pool_get_storage_range(None, None) == lbm.LBM_ERR_INVALID_ARG
    assert lbm.lib().lbm_pool_request_range(None, 0, None) == lbm.LBM_ERR_INVALID_ARG
    assert lbm.lib().lbm_set_storage_reference(None, None) == lbm.LBM_ERR_INVALID_ARG
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_step(None, 1)
    assert e.value.status == lbm.LBM_ERR_INVALID_ARG


def test_fixed_point_storage_host_checks(L):
    """The fixed-point form: two bytes per value, a range only it has, and the allocation-free
    reduction turns it away before any device work."""
    n16 = lbm.lbm_workspace_bytes("D3Q19", (64, 64, 64), "f16")
    assert lbm.lbm_workspace_bytes("D3Q19", (64, 64, 64), "q16") == n16
    assert lbm.lib().lbm_set_storage_range(None, 1.0) == lbm.LBM_ERR_INVALID_ARG
    assert lbm.lib().lbm_status_string(lbm.LBM_ERR_RANGE) == b"value outside the storage range"
    h = ctypes.c_void_p()
    st = lbm.lib().lbm_pool_create(lbm.LATTICES["D3Q19"], 3, lbm.STORAGES["q16"], None, 1 << 20, 4, None, None,
                                   ctypes.byref(h))
    assert st == lbm.LBM_ERR_INVALID_ARG and h.value is None  # pools take it; the NULL arena is refused
    assert lbm.lib().lbm_pool_set_storage_range(None, 1.0) == lbm.LBM_ERR_INVALID_ARG
    out = (ctypes.c_double * 4)()
    d = (ctypes.c_int64 * 3)(8, 8, 8)
    st = lbm.lib().lbm_conservation_noalloc(lbm.LATTICES["D3Q19"], lbm.STORAGES["q16"], d, 1.0,
                                            ctypes.c_void_p(256), out, lbm.MEM_HOST, None)
    assert st == lbm.LBM_ERR_UNSUPPORTED


def test_noalloc_dims_use_the_solver_limits(L):
    """The allocation-free sums reject, before any device work, every shape lbm_create rejects:
    a side above 2^24 (whose int conversion would wrap), a 2-D lattice with nz != 1, a side
    below the largest velocity component, and nz above its fixed scratch."""
    out = (ctypes.c_double * 4)()

    def status(lattice, dims):
        d = (ctypes.c_int64 * 3)(*dims)
        return lbm.lib().lbm_conservation_noalloc(lbm.LATTICES[lattice], lbm.STORAGES["f32"], d, 1.0,
                                                  ctypes.c_void_p(256), out, lbm.MEM_HOST, None)

    assert status("D3Q19", (1 << 31, 1, 1)) == lbm.LBM_ERR_INVALID_ARG
    assert status("D3Q19", (1 << 40, 1 << 40, 1)) == lbm.LBM_ERR_INVALID_ARG
    assert status("D2Q9", (8, 8, 2)) == lbm.LBM_ERR_INVALID_ARG
    assert status("D3Q39", (8, 2, 8)) == lbm.LBM_ERR_INVALID_ARG
    assert status("D3Q19", (4, 4, 4097)) == lbm.LBM_ERR_INVALID_ARG
    assert status("D3Q19", (0, 4, 4)) == lbm.LBM_ERR_INVALID_ARG
    assert b"dims" in lbm.lib().lbm_last_error() or b"4096" in lbm.lib().lbm_last_error()


def test_reference_velocity_forms_host_checks(L):
    """The forms with a per-cell reference velocity: Q + D planes of two bytes per buffer; pools
    and the allocation-free sums turn them away before any device work."""
    C = 64 ** 3
    n = lbm.lbm_workspace_bytes("D3Q19", (64, 64, 64), "f16r")
    n16 = lbm.lbm_workspace_bytes("D3Q19", (64, 64, 64), "f16")
    assert n - n16 == 2 * 3 * C * 2
    assert lbm.lbm_workspace_bytes("D2Q9", (64, 64, 1), "bf16r") - lbm.lbm_workspace_bytes(
        "D2Q9", (64, 64, 1), "bf16") == 2 * 2 * 64 * 64 * 2
    d = (ctypes.c_int64 * 3)(64, 64, 64)
    assert lbm.lib().lbm_pool_request_bytes(lbm.LATTICES["D3Q19"], d, lbm.STORAGES["f16r"]) == 0
    out = (ctypes.c_double * 4)()
    st = lbm.lib().lbm_conservation_noalloc(lbm.LATTICES["D3Q19"], lbm.STORAGES["f16r"], d, 1.0,
                                            ctypes.c_void_p(256), out, lbm.MEM_HOST, None)
    assert st == lbm.LBM_ERR_UNSUPPORTED


def test_bounds_walk_consistent_and_inconsistent_plane_sizes(L):
    """The guard's arithmetic on the host: for every cells-per-thread and a set of odd and
    degenerate sizes, no access of a register-pull launch falls outside a consistent plane
    (P = nx*ny*nz); with a dims/P pair that disagrees (one element short, or the nz of a bigger
    lattice) the walk counts the accesses the bounds-check build's kernels would skip."""
    cases = [("D3Q19", (1, 1, 1)), ("D3Q19", (5, 7, 9)), ("D3Q39", (3, 3, 3)), ("D3Q39", (12, 5, 3)),
             ("D2Q9", (3, 11, 1)), ("D3Q27", (8, 3, 1)), ("D3Q15", (16, 1, 5)), ("D3Q19", (72, 9, 4)),
             ("D3Q39", (4, 5, 3)), ("D3Q39", (8, 3, 3))]  # rows of one to four chunks (whole-chunk loads)
    for name, dims in cases:
        C = int(np.prod(dims))
        for V in (1, 2, 4, 8):
            if dims[0] % V:
                continue
            bad, n = lbm.lbm_bounds_walk(name, V, dims, C)
            assert bad == 0 and n > 0, (name, dims, V)
            bad, n = lbm.lbm_bounds_walk(name, V, dims, C - 1)
            assert bad > 0, (name, dims, V)  # the last cell's own store at least
            bigger = (dims[0], dims[1], dims[2] + 1) if name != "D2Q9" else (dims[0], dims[1] + 1, 1)
            bad, n = lbm.lbm_bounds_walk(name, V, bigger, C)
            assert bad > 0, (name, dims, V)
    assert lbm.lib().lbm_bounds_walk(lbm.LATTICES["D3Q19"], 3, (ctypes.c_int64 * 3)(8, 8, 8), 512, None) == -1
    assert lbm.lbm_bounds_checked() in (False, True)


def test_pool_request_bytes_use_the_padded_pitch(L):
    """A pool stores each request with its rows padded to a multiple of 4 cells (pad cells hold
    periodic images): two buffers of Q planes of px*ny*nz values, each 256-byte aligned, and a
    256-byte status word."""
    def align(v):
        return (v + 255) // 256 * 256

    for nx, ny, nz in [(33, 20, 7), (32, 32, 32), (1, 5, 6), (127, 3, 4)]:
        px = (nx + 3) // 4 * 4
        want = 2 * align(19 * px * ny * nz * 2) + 256
        assert lbm.lbm_pool_request_bytes("D3Q19", (nx, ny, nz), "f16") == want, (nx, ny, nz)
    assert lbm.lbm_pool_request_bytes("D3Q19", (33, 20, 7), "f32") == 2 * align(19 * 36 * 20 * 7 * 4) + 256
    # a plane within 2^31 - 1 cells whose padded rows would pass it: not admitted
    assert lbm.lbm_pool_request_bytes("D3Q19", (2 ** 24 - 1, 128, 1), "f16") == 0
    assert lbm.lbm_pool_request_bytes("D3Q19", (2 ** 24, 127, 1), "f16") == 2 * align(19 * 2 ** 24 * 127 * 2) + 256
