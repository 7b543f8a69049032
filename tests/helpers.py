"""Shared comparison helpers for the parity tests (test code only)."""
import numpy as np


def masked_rel_err(got, ref, floor_frac):
    """max |got - ref| / ref over pixels with ref > floor_frac * max(ref)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    m = ref > floor_frac * ref.max()
    assert m.any()
    return float(np.max(np.abs(got[m] - ref[m]) / ref[m])), int(m.sum())


def rel_err_above(got, ref, floor_abs):
    """max |got - ref| / ref over pixels with ref > floor_abs (absolute)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    m = ref > floor_abs
    if not m.any():
        return 0.0, 0
    return float(np.max(np.abs(got[m] - ref[m]) / ref[m])), int(m.sum())


def abs_err_frac(got, ref):
    """max |got - ref| over all pixels, as a fraction of max(ref)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(got - ref)) / ref.max())


def gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False
