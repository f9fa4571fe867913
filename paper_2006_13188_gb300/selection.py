"""Fixed-budget component selection (Sec. 5 "Band-Limiting Revisited").

Host logic only: the energies come from the library (ext_filter_so2_energy,
FP64 on the device) and the sweep over the chosen components from
ext_corr_so2_subset.  Rule: G_0 is always kept (one real correlation, the
angle-independent mean); the remaining budget - 1 components are the k >= 1
of largest lattice energy, ties to the smaller k.
"""
from __future__ import annotations

import numpy as np

from . import _binding as b


def select(plan, F, budget):
    """Component list [0, k_1 < k_2 < ...] of length min(budget, K + 1)."""
    E = b.ext_filter_so2_energy(plan, F)
    K = len(E) - 1
    order = sorted(range(1, K + 1), key=lambda k: (-E[k], k))
    return [0] + sorted(order[:max(int(budget), 1) - 1])


def lowest(F, budget):
    """The band-limited alternative: components 0 .. budget - 1."""
    return list(range(min(int(budget), F.K + 1)))
