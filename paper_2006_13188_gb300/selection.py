"""Fixed-budget component selection (Sec. 5 "Band-Limiting Revisited").

The energies come from the library (ext_filter_so2_energy, FP64 on the
device), the rule from ext_select_components (G_0 always kept, then the
budget - 1 components k >= 1 of largest lattice energy, ties to the smaller
k), and the sweep over the chosen components from ext_corr_so2_subset.
"""
from __future__ import annotations

from . import _binding as b


def select(plan, F, budget):
    """Component list [0, k_1 < k_2 < ...] of length min(budget, K + 1)."""
    return b.ext_select_components(b.ext_filter_so2_energy(plan, F), budget)


def lowest(F, budget):
    """The band-limited alternative: components 0 .. budget - 1."""
    return list(range(min(int(budget), F.K + 1)))
