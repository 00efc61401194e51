"""Shared helpers of the GPU tests (parity of the CUDA path with the oracle)."""
import numpy as np

# Parity bar of the gradient: relative L2 error <= 1e-5 against the FP64
# oracle.  Elementwise, every pair term is a unit vector scaled by a weight
# (rho_q, summing to 1, or 1/N), so the sum of absolute term values of A_i and
# of R_i is <= 1; FP32 pair arithmetic with row/block sums of <= 4096 terms
# folded into compensated or FP64 accumulators keeps each component within
# ~4096 * 2^-24 ~ 2.4e-4 in the worst case and ~sqrt(4096) * 2^-24 ~ 4e-6 in
# the typical case; 1e-5 absolute per component is the elementwise gate.
GRAD_REL_L2 = 1e-5
GRAD_ABS = 1e-5


def rel_l2(a, b) -> float:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def assert_grad_close(gpu, ref, what="G", rel=GRAD_REL_L2, atol=GRAD_ABS):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    e = rel_l2(gpu, ref)
    m = float(np.abs(gpu - ref).max())
    assert e <= rel, f"{what}: relative L2 error {e:.3e} > {rel:.1e}"
    assert m <= atol, f"{what}: max abs error {m:.3e} > {atol:.1e}"
    return e, m


# FP32 output of the FP64 projection (the default for every K dtype): the
# GPU's and the oracle's FP64 iterates agree to ~1e-11, so their FP32
# roundings differ by at most one ulp of |s| <= 1/2, i.e. 2^-24.
PROJ_F32_ROUND = 2.0 ** -24


def proj_tol_f32(ref, k) -> float:
    """Elementwise gate of the opt-in mixed-precision projection (FP32
    output, PROJECTION_MIXED).  The FP32 output
    rounds s (<= 2^-24 at |s| <= 1/2, doubled: 1.2e-7); the FP32 iteration
    of the mixed-precision form works on the displacement e = s - k and the
    duals, whose roundings (a few per iteration, accumulating over the
    iterations) stay within 128 * 2^-24 * max|e|."""
    e = np.abs(np.asarray(ref, np.float64) - np.asarray(k, np.float64)).max()
    return 1.2e-7 + 128 * 2.0 ** -24 * e
