"""Accuracy of the storage forms at the stated sizes of the 16-bit Taylor-Green workloads.

D3Q19, u0 = 0.05, K = 2: 256^3 with tau = 0.55 for 1000 steps, and 512^3 with tau = 0.52 for
500 steps.  The oracle is too slow at these sizes, so each form is compared with the library's
own FP64 path on the same run, which the parity tests tie to the oracle within 1e-12 (and the
64^3 runs of test_gpu_physics.py compare each form with the oracle directly).  Error on u:
max|du| / max|u| (u crosses zero); on rho: per element.

Relative error on u, as measured on a GB300:
  256^3: FP32 1.2e-5, FP16 9.3e-3, BF16 9.6e-2, 16-bit fixed point (range 1/4) 1.3e-4,
         FP16 / BF16 with a per-cell reference velocity 2.7e-5 / 3.9e-4
  512^3: FP32 1.1e-5, FP16 7.8e-3, BF16 3.3e-2, 16-bit fixed point (range 1/4) 2.1e-4,
         FP16 / BF16 with a per-cell reference velocity 3.1e-5 / 4.6e-4
The fixed-point form and both reference-velocity forms meet the 1e-3 target on u at both
sizes.  FP16 and BF16 storage of the scaled shifted value itself miss it: the values that carry
the momentum (|h| ~ 0.15) round at ~6e-5 (FP16) or ~5e-4 (BF16) per step, and the errors
accumulate; with the reference velocity only the residual h_i - r_i (|.| ~ 0.006) is rounded.
The misses are recorded as expected failures of the target (strict: a form that starts
meeting it fails the record), and their measured size is held as a regression ceiling."""
import pytest

from paper_2002_02503_gb300 import fields, lbm

from _lbmtest import TOL_U16, rel_f, rel_u

pytestmark = pytest.mark.gpu

CONFIGS = {"256": ((256, 256, 256), 0.55, 1000), "512": ((512, 512, 512), 0.52, 500)}
# measured relative errors on u (see the module docstring) times 1.25: the regression ceilings
CEILING = {("256", "f16"): 1.25 * 9.3e-3, ("256", "bf16"): 1.25 * 9.6e-2,
           ("512", "f16"): 1.25 * 7.8e-3, ("512", "bf16"): 1.25 * 3.3e-2}
Q16_RANGE = 0.25

FORMS = ("f32", "f16", "bf16", "q16", "f16r", "bf16r")


@pytest.fixture(scope="module")
def errors():
    """{(key, storage): (rel_u, rel_rho)} of every storage form against the FP64 path, both sizes."""
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    out = {}
    for key, (dims, tau, steps) in CONFIGS.items():
        rho, u = fields.taylor_green_3d(dims, 0.05, 1.0 / 3.0)

        def run(st):
            s = lbm.Solver("D3Q19", dims, tau, 2, st, storage_range=Q16_RANGE if st == "q16" else None)
            s.set_fields(rho, u)
            s.step(steps)
            res = s.moments()
            s.close()
            del s
            torch.cuda.empty_cache()
            return res

        r_ref, u_ref = run("f64")
        for st in FORMS:
            r, uu = run(st)
            out[(key, st)] = (rel_u(uu, u_ref), rel_f(r, r_ref))
            print("D3Q19 %s^3 tau=%g %d steps, %s storage: rel u %.3e, rel rho %.3e (vs FP64 path)" % (
                key, tau, steps, st, out[(key, st)][0], out[(key, st)][1]))
            del r, uu
        del rho, u, r_ref, u_ref
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("key", ["256", "512"])
def test_fixed_point_storage_meets_u_bound(errors, key):
    eu, er = errors[(key, "q16")]
    assert eu < TOL_U16
    assert er < TOL_U16


@pytest.mark.parametrize("key", ["256", "512"])
@pytest.mark.parametrize("storage", ["f16r", "bf16r"])
def test_16bit_float_with_reference_velocity_meets_u_bound(errors, key, storage):
    """FP16 and BF16 storage of the residual after a per-cell reference velocity."""
    eu, er = errors[(key, storage)]
    assert eu < TOL_U16
    assert er < TOL_U16


@pytest.mark.parametrize("key", ["256", "512"])
def test_fp32_storage_at_stated_sizes(errors, key):
    """FP32 storage over the full runs (the 1e-5 bound is for 100 steps; over 500-1000 steps the
    FP32 error grows to ~1.2e-5, which is reported, not hidden)."""
    eu, er = errors[(key, "f32")]
    assert eu < 2e-5
    assert er < 1e-6


@pytest.mark.parametrize("key,storage", [("256", "f16"), ("256", "bf16"), ("512", "f16"), ("512", "bf16")])
@pytest.mark.xfail(strict=True, reason="FP16/BF16 storage of the scaled shifted value misses 1e-3 on u at the "
                                       "stated sizes (FP16 9.3e-3 / 7.8e-3, BF16 9.6e-2 / 3.3e-2)")
def test_16bit_float_storage_meets_u_bound(errors, key, storage):
    assert errors[(key, storage)][0] < TOL_U16


@pytest.mark.parametrize("key,storage", [("256", "f16"), ("256", "bf16"), ("512", "f16"), ("512", "bf16")])
def test_16bit_float_storage_error_regression(errors, key, storage):
    """The measured misses must not grow."""
    assert errors[(key, storage)][0] < CEILING[(key, storage)]
