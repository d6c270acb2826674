"""Parity checks of GPU results against the FP64 oracle, shared by the tests.

Every comparison holds two bounds:
  * relative L2 error  ||x - ref|| / ||ref||  <= the form's bar (float32
    storage 1e-5, 16-bit storage 2e-3, 8-bit storage 0.8 times the format's
    unit roundoff: E4M3 (2^-4) 5e-2, E5M2 (2^-3) 1e-1);
  * element-wise error  max_n |x_n - ref_n| / max_n |ref_n|  <= a stated bound
    (by default the same number): no single voxel (or channel sample) may be
    wrong by more than that fraction of the image peak, which a norm over
    millions of values would not notice.
"""
import numpy as np

BAR = {"f32": 1e-5, "f16": 2e-3, "bf16": 2e-3, "e4m3": 5e-2, "e5m2": 1e-1}

# Element-wise bound of float32 results at the paper workload's scale: about
# 8000 contributing terms per voxel are summed in float32, and the rounding of
# a sum of T terms drifts by about sqrt(T) x 6e-8 of their magnitude
# (5e-6 at T = 8000); several standard deviations over 2 M voxels stay
# below 5e-5 of the peak.
ELEM_F32_PAPER = 5e-5


def rel_l2(a, b) -> float:
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def max_rel(a, b) -> float:
    """Largest element-wise error over the largest |b|."""
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def assert_parity(x, ref, l2: float, elem: "float | None" = None, what: str = "") -> tuple:
    """Both bounds; returns (relative L2, element-wise) for printing."""
    e2, em = rel_l2(x, ref), max_rel(x, ref)
    elem = l2 if elem is None else elem
    assert e2 <= l2 and em <= elem, (f"{what}: relative L2 {e2:.3e} (bar {l2:.1e}), "
                                     f"element-wise {em:.3e} of the peak (bound {elem:.1e})")
    return e2, em
