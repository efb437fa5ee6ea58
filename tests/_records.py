"""Plain relative errors of the tendency parity checks, collected during the
run and printed in the terminal summary (tests/conftest.py)."""
import numpy as np

TENDENCY = []


def record_tendency(what, k, k_ref, S):
    """Per field: ||k - k_ref||_2 / ||k_ref||_2 (plain) and
    max|k - k_ref| / max S (the asserted measure)."""
    k = np.asarray(k).reshape(k_ref.shape)
    row = []
    for f in range(k_ref.shape[-2]):
        d = k[..., f, :] - k_ref[..., f, :]
        nref = np.linalg.norm(k_ref[..., f, :])
        row.append((float(np.linalg.norm(d) / nref) if nref > 0 else float("nan"),
                    float(np.abs(d).max() / S[..., f, :].max())))
    TENDENCY.append((what, row))
