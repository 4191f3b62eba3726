"""The paper's cost accounting of the low-rank method (Sec. "Memory, computational complexity
and implementation"): a full-rank step costs O(n m) in time and memory, a low-rank step
O(r^2 (n + m)) in time and O(r (n + m)) in memory, with n cells, m = (N + 1)^2 moments and r
the rank averaged over the energy steps. Table 1 of the paper evaluates these with the mean
rank r_bar, as r_bar^2 (n + m) and r_bar (n + m)."""
from __future__ import annotations

import numpy as np


def costs(n: int, sh_degree: int, ranks) -> dict:
    """Full-rank and low-rank sizes for n cells, P_N degree sh_degree and the ranks of the
    energy steps (any sequence; their mean is the paper's average rank)."""
    m = (int(sh_degree) + 1) ** 2
    r = float(np.mean(np.asarray(ranks, dtype=np.float64)))
    full = float(n) * m
    comp = r * r * (n + m)
    size = r * (n + m)
    return dict(moments=m, mean_rank=r, full_rank=full, dlra_complexity=comp, dlra_system_size=size,
                complexity_percent=100.0 * comp / full, system_size_percent=100.0 * size / full)
