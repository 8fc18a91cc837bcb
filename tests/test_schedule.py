"""Host-only LPT schedule used by ragged batches (fwr_schedule_lpt), CPU."""

import os

import numpy as np
import pytest

from paper_1705_04298_gb300 import build_lib, fwr


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not os.path.exists(fwr.LIB_PATH):
        build_lib.build()
    return fwr.load()


@pytest.mark.parametrize("seed,n,ctas", [(0, 4096, 152), (1, 37, 8), (2, 5, 16), (3, 1000, 1)])
def test_lpt_is_a_partition_within_the_list_scheduling_bound(seed, n, ctas):
    rng = np.random.default_rng(seed)
    costs = np.where(rng.random(n) < 0.5, 1.0, 9.6) * (1 + 0.1 * rng.random(n))
    off, order = fwr.schedule_lpt(costs, ctas)
    assert off[0] == 0 and off[-1] == n and np.all(np.diff(off) >= 0)
    assert sorted(order.tolist()) == list(range(n))
    loads = np.array([costs[order[off[c]:off[c + 1]]].sum() for c in range(ctas)])
    # greedy list scheduling: makespan <= mean load + largest job; LPT <= 4/3 OPT
    assert loads.max() <= costs.sum() / ctas + costs.max() + 1e-9
    lower = max(costs.sum() / ctas, costs.max())
    assert loads.max() <= 4.0 / 3.0 * lower + 1e-9 or n <= ctas


def test_lpt_exact_small_case():
    # four jobs on two workers: 5 | 4, then 3 goes to the 4, then 2 to the 5
    off, order = fwr.schedule_lpt([2.0, 5.0, 3.0, 4.0], 2)
    assert off.tolist() == [0, 2, 4]
    assert order.tolist() == [1, 0, 3, 2]


def test_lpt_rejects_bad_input():
    with pytest.raises(fwr.FwrError):
        fwr.schedule_lpt([1.0, -1.0], 2)
    with pytest.raises(fwr.FwrError):
        fwr.schedule_lpt([1.0, float("nan")], 2)
    with pytest.raises(fwr.FwrError):
        fwr.schedule_lpt([1.0], 0)
