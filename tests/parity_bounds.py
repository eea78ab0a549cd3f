"""Parity bounds shared by the GPU tests: the CUDA path against the FP64 oracle.

The force of Eq. (1) is a sum over simulations, F = sum_i c_i, of per-simulation
contributions c_i = weight_k * sum_n w_n s_i(n) (Sec. II; Sec. III A).  The tolerances:

FP64 mode
  * per simulation: |c_i(GPU) - c_i(oracle)| <= 1e-10 |c_i| + m u sqrt(T) max_j |c_j|;
  * the force:      |F(GPU) - F(oracle)|     <= 1e-10 |F|   + m u sqrt(T) sum_j |c_j|.
  The second terms are rounding floors.  Both sides run the same leapfrog in FP64 but
  round in a different order (fused multiply-adds, the order of the pixel sums, the
  reduction order).  One time step rounds each stored value at most m times (m = 16
  bounds the longest chain of rounded operations that produces one stored value in one
  step: the curl differences, the conductivity update, the CPML recursion, three Lorentz
  poles and the scaling by 1/eps), so a value carries a relative error of at most m u per
  step (u = 2^-53).  The leapfrog does not amplify errors (it conserves the discrete
  energy at sigma = 0 and damps it for sigma > 0), and the rounding errors of independent
  steps add like a random walk, so after T steps a field value differs between the two
  sides by about m u sqrt(T) times the field's magnitude.  A simulation's measured
  functional is a weighted sum of such values, so its error is bounded by m u sqrt(T)
  times the magnitude of the fields it samples -- not by its own value, which can be a
  small residual: a cross component (the x field of a y-directed source, non-zero only
  through reflections) is 1e-9 of the fields that carry its rounding, and a run of one
  step gives 9e-16 on the CPU where the GPU's order of summation gives exactly 0.  The
  largest contribution of the plan, max_j |c_j| (the self term of a source measured on
  its own face, a sum of terms of one sign), measures the magnitude of the sampled fields
  times the weights, since every simulation's source is an orthonormal harmonic.
  Summed over simulations, the force's floor is m u sqrt(T) sum_j |c_j|; on the closed
  contours of the piston sum_j |c_j| / |F| reaches 1e6-3e7, which no choice of summation
  can undo, because each c_i is itself only known to FP64 precision.
FP32 fields, FP64 accumulation
  * the force: |F(GPU) - F(oracle)| <= 1e-4 |F(oracle)| + m u sqrt(T) sum_j |c_j| (u = 2^-53:
    the rounding floor of the FP64 sums, which both sides form in FP64 as in FP64 mode; it
    matters only where the contributions cancel exactly, as in the first steps of a run
    whose sources have not yet reached an asymmetric object: there the oracle's force is 0.0
    and the GPU's a residual of order 1e-18 sum_j |c_j|);
  * per simulation: max_i |c_i(GPU) - c_i(oracle)| <= 2e-5 max_i |c_i(oracle)|, the same
    floor with u = 2^-24, m of about 5 and sqrt(T) of about 60 (T of a few thousand steps).
"""
import math

import numpy as np

U64 = 2.0 ** -53
M_OPS = 16


def fp64_sim_floor(parts, n_steps):
    """m u sqrt(T) max_j |c_j|: the rounding floor of one simulation in FP64 mode."""
    return M_OPS * U64 * math.sqrt(max(1, n_steps)) * float(np.max(np.abs(parts)))


def fp64_force_floor(parts, n_steps):
    """m u sqrt(T) sum_i |c_i|: the rounding floor of the force in FP64 mode."""
    return M_OPS * U64 * math.sqrt(max(1, n_steps)) * float(np.sum(np.abs(parts)))


def assert_parity(per, F_gpu, parts, F_oracle, n_steps, fp64, what=""):
    """Compare a GPU result (per-simulation contributions `per`, force component `F_gpu`)
    with the oracle's (`parts`, `F_oracle`) under the bounds above."""
    per = np.asarray(per, dtype=np.float64)
    parts = np.asarray(parts, dtype=np.float64)
    assert per.shape == parts.shape, (what, per.shape, parts.shape)
    dF = abs(F_gpu - F_oracle)
    frel = dF / abs(F_oracle) if F_oracle != 0 else float("inf") if dF else 0.0
    if fp64:
        d = np.abs(per - parts)
        lim = 1e-10 * np.abs(parts) + fp64_sim_floor(parts, n_steps)
        bad = d > lim
        worst = int(np.argmax(d / lim))
        assert not bad.any(), (f"{what}: {int(bad.sum())} of {len(parts)} simulations beyond their bound; "
                               f"worst sim {worst}: gpu {per[worst]!r} oracle {parts[worst]!r} bound {lim[worst]:.3e}")
        bound = 1e-10 * abs(F_oracle) + fp64_force_floor(parts, n_steps)
        assert dF <= bound, (f"{what}: force {F_gpu!r} vs oracle {F_oracle!r}: |dF| {dF:.3e} > bound {bound:.3e} "
                             f"(relative {frel:.3e})")
    else:
        dmax = float(np.max(np.abs(per - parts))) if len(parts) else 0.0
        assert dmax <= 2e-5 * float(np.max(np.abs(parts))), (
            f"{what}: per-simulation error {dmax:.3e} > 2e-5 of the largest {float(np.max(np.abs(parts))):.3e}")
        bound = 1e-4 * abs(F_oracle) + fp64_force_floor(parts, n_steps)
        assert dF <= bound, (f"{what}: force {F_gpu!r} vs oracle {F_oracle!r}: |dF| {dF:.3e} > bound {bound:.3e} "
                             f"(relative {frel:.3e})")
    return frel
