"""Helpers shared by the GPU tests (no method arithmetic)."""
import numpy as np

NON_NEUTRAL = 4     # MSM_DEV_NON_NEUTRAL: warning bit of the device status word
NEUTRAL_TOL = 1e-5  # |sum q| > 1e-5 sum |q| counts as non-neutral


def expected_status(systems):
    """Status word expected after a clean forward: the non-neutral warning bit if
    some system with a periodic axis carries a net charge, else 0."""
    if not isinstance(systems, (list, tuple)):
        systems = [systems]
    for w in systems:
        q = np.asarray(w.q, np.float64)
        if any(w.pbc) and abs(q.sum()) > NEUTRAL_TOL * np.abs(q).sum():
            return NON_NEUTRAL
    return 0


def expected_for(pbc, q):
    """expected_status of one system given its periodicity and charges."""
    q = np.asarray(q, np.float64)
    return NON_NEUTRAL if any(pbc) and abs(q.sum()) > NEUTRAL_TOL * np.abs(q).sum() else 0
