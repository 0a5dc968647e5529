"""Shared helpers of the parity tests (comparison rule only; no method arithmetic)."""
import numpy as np


def rel_err(got, ref, tau_frac: float = 1e-3) -> np.ndarray:
    """Per-output relative error |g - o| / max(|o|, tau), tau = tau_frac * rms(o) over the batch."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    tau = tau_frac * np.sqrt(np.mean(ref ** 2)) if ref.size else 0.0
    tau = max(tau, 1e-300)
    return np.abs(got - ref) / np.maximum(np.abs(ref), tau)
