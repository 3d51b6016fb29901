"""Ring statistics of the C network from the library's ring records
(System.rings): counts per size and replica, and the histogram of 6-ring
orientations (Sec. 3.3 plots both: the numbers of 5-, 6- and 7-membered
rings over time, and the orientations of the 6-membered rings on the
terrace). Binning of the records only; the rings themselves are found on
the GPU."""
from __future__ import annotations

import numpy as np


def counts(records: np.ndarray, n_replicas: int, max_size: int = 8) -> np.ndarray:
    """[n_replicas, max_size - 2] number of rings of each size 3..max_size."""
    out = np.zeros((n_replicas, max_size - 2), dtype=np.int64)
    np.add.at(out, (records["replica"], records["size"] - 3), 1)
    return out


def orientation_histogram(records: np.ndarray, bins: int = 60, replica: int | None = None,
                          zmin: float | None = None) -> np.ndarray:
    """Histogram of 6-ring orientations over [0, 60) degrees, optionally of
    one replica and of rings whose centre lies at z >= zmin (e.g. on the
    terrace)."""
    m = records["size"] == 6
    if replica is not None:
        m &= records["replica"] == replica
    if zmin is not None:
        m &= records["centre"][:, 2] >= zmin
    h, _ = np.histogram(records["orientation"][m], bins=bins, range=(0.0, 60.0))
    return h
