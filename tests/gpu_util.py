"""Helpers for the GPU parity tests (no method arithmetic here)."""
import numpy as np


def to_dev(*arrs):
    import torch
    return [torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda") for a in arrs]


def to_np(*ts):
    return [t.detach().cpu().numpy() for t in ts]


def eps_modes(a_re, a_im, b_re, b_im):
    """Eq. results:error per mode with the complex modulus: max|a - b| / max|b|."""
    a = np.asarray(a_re) + 1j * np.asarray(a_im)
    b = np.asarray(b_re) + 1j * np.asarray(b_im)
    den = np.max(np.abs(b), axis=-1)
    den = np.where(den > 0, den, 1.0)
    return np.max(np.abs(a - b), axis=-1) / den
