"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np


def rel_err(got, ref, scale=None):
    got = np.asarray(got)
    ref = np.asarray(ref)
    s = scale if scale is not None else max(1.0, float(np.abs(ref).max()))
    return float(np.abs(got - ref).max()) / s


def fp32_bound(abs_ref, eps_factor=64.0):
    """Error bound of an FP32 blocked sum: eps_factor * 2^-24 * sum |terms|."""
    return eps_factor * 2.0 ** -24 * np.asarray(abs_ref) + 1e-30
