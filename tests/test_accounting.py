"""The paper's Table 1 cost figures from its formulas (paper_2508_04484_gb300/accounting.py)
against the printed values (tests/golden/table1_costs.json)."""
import json
import os

import pytest

from paper_2508_04484_gb300 import accounting as AC

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table1_costs.json")


@pytest.mark.parametrize("model", ["boltzmann", "fokker_planck"])
def test_table1_costs(model):
    g = json.load(open(GOLDEN))
    row = g[model]
    n = g["cells"]
    m = (row["sh_degree"] + 1) ** 2
    assert row["full_rank"] == n * m
    # the table prints the mean rank rounded to two digits; its system-size column fixes it
    r_bar = row["dlra_system_size"] / (n + m)
    assert abs(r_bar - row["mean_rank"]) < 5e-3
    c = AC.costs(n, row["sh_degree"], [r_bar])
    assert c["full_rank"] == row["full_rank"]
    assert abs(c["dlra_system_size"] / row["dlra_system_size"] - 1.0) < 1e-12
    # the complexity column is r_bar^2 (n + m) with that same mean rank
    assert abs(c["dlra_complexity"] / row["dlra_complexity"] - 1.0) < 1e-9
    assert abs(c["complexity_percent"] - row["complexity_percent"]) < 5e-5 * max(1.0, row["complexity_percent"])
    assert abs(c["system_size_percent"] - row["system_size_percent"]) < 5e-5 * max(1.0, row["system_size_percent"])


def test_mean_rank_is_averaged_over_the_steps():
    c = AC.costs(1000, 3, [2, 4, 6])
    assert c["moments"] == 16 and c["mean_rank"] == 4.0
    assert c["dlra_system_size"] == 4.0 * 1016 and c["dlra_complexity"] == 16.0 * 1016
