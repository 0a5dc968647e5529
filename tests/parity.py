"""Shared helpers of the parity tests (comparison rule only; no method arithmetic).

Per-output relative error |g - o| / max(|o|, tau), tau = rms(o) over the
compared batch.  The floor is the batch rms because FP32 rounding of the 64
encoded inputs alone moves an output by about 6e-8 * sum_k |w_k h_k|; for an
output that is near zero by cancellation that is many times |o|, so no FP32
pipeline (and no 16-bit one) has a meaningful relative error there.  Above
the rms the measure is the plain relative error.  ``stats`` also reports the
error with the tighter floor 1e-3 * rms.
"""
import numpy as np


def rel_err(got, ref, tau_frac: float = 1.0) -> np.ndarray:
    """Per-output relative error floored at tau = tau_frac * rms(ref)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    tau = tau_frac * np.sqrt(np.mean(ref ** 2)) if ref.size else 0.0
    tau = max(tau, 1e-300)
    return np.abs(got - ref) / np.maximum(np.abs(ref), tau)


def stats(got, ref) -> dict:
    e1 = rel_err(got, ref, 1.0)
    e3 = rel_err(got, ref, 1e-3)
    return {"max": float(e1.max()), "p999_floor1e-3": float(np.quantile(e3, 0.999)),
            "max_floor1e-3": float(e3.max()), "median": float(np.median(e1))}
