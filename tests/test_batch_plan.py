"""The host-only batch planner (dbm_batch_plan), i.e. the item table every
batched step launches, checked on the CPU: each simulation's strips x row
runs appear exactly once, padding and launch order follow the documented
layout, and the longest-first balance keeps the busiest CTA within the
list-scheduling bound and no worse than dealing the items round-robin."""
import numpy as np
import pytest

from paper_1308_0653_gb300 import dbm


def _expected(nr, nth, rows, width):
    out = set()
    for s, (n, t, L) in enumerate(zip(nr, nth, rows)):
        if n == 0:
            continue
        for j0 in range(0, n, width):
            for mb in range(0, t, L):
                out.add((s, j0, mb, min(mb + L, t)))
    return out


def _cost(item, nr, width):
    s, j0, mb, me = (int(x) for x in item)
    if s < 0:
        return 0.0
    return (me - mb + 2) * (0.3 + 0.7 * min(width, nr[s] - j0) / width)


def _busiest(items, nr, width, grid):
    c = [_cost(x, nr, width) for x in items]
    return max(sum(c[k::grid]) for k in range(grid)), c


@pytest.mark.parametrize("seed", range(5))
@pytest.mark.parametrize("width,grid", [(128, 304), (64, 296), (128, 7)])
def test_items_cover_each_simulation_once_and_balance(seed, width, grid):
    rng = np.random.default_rng(1000 + seed)
    nslots = 24
    nr = rng.integers(1, 1100, nslots)
    nr[rng.random(nslots) < 0.2] = 0                 # empty slots
    nth = rng.integers(1, 1100, nslots)
    rows = rng.choice([1, 7, 16, 32, 64, 5000], nslots)
    items = dbm.dbm_batch_plan(nr, nth, rows, width, grid, 1 << 21)
    real = [tuple(int(v) for v in x) for x in items if x[0] >= 0]
    assert len(real) == len(set(real))
    assert set(real) == _expected(nr, nth, rows, width)
    assert all(tuple(x) == (-1, 0, 0, 0) for x in items if x[0] < 0)
    if len(real) <= grid:
        assert len(items) == len(real)               # one wave: no padding
        return
    assert len(items) % grid == 0                    # CTA c runs c, c + grid, ...
    top, costs = _busiest(items, nr, width, grid)
    assert top <= sum(costs) / grid + max(costs) + 1e-9
    # dealing the interleaved items round-robin, without the balance
    rr = sorted(real, key=lambda x: (x[0], x[2], x[1]))
    rr_top, _ = _busiest(rr, nr, width, grid)
    assert top <= rr_top + 1e-9


def test_capacity_and_errors():
    # 3 x 5 + 1 x 3 = 18 items
    nr, nth, rows = [300, 0, 128], [72, 0, 40], [16, 16, 16]
    assert len(dbm.dbm_batch_plan(nr, nth, rows, 128, 304, 18)) == 18
    with pytest.raises(dbm.DbmError) as e:
        dbm.dbm_batch_plan(nr, nth, rows, 128, 304, 17)
    assert e.value.status == dbm.DBM_ENOMEM
    # balanced over 8 CTAs the table would need padding beyond 18 entries:
    # the interleaved order is kept instead
    items = dbm.dbm_batch_plan(nr, nth, rows, 128, 8, 18)
    assert len(items) == 18 and (items[:, 0] >= 0).all()
    assert [tuple(x) for x in items[:3]] == [(0, 0, 0, 16), (2, 0, 0, 16), (0, 128, 0, 16)]
    assert len(dbm.dbm_batch_plan(nr, nth, rows, 128, 8, 1000)) % 8 == 0
    assert len(dbm.dbm_batch_plan([0, 0], [0, 0], [1, 1], 128, 304, 10)) == 0
    for bad in [([5], [5], [0], 128, 8), ([5], [0], [1], 128, 8), ([-1], [5], [1], 128, 8),
                ([5], [5], [1], 0, 8), ([5], [5], [1], 128, 0)]:
        with pytest.raises(dbm.DbmError) as e:
            dbm.dbm_batch_plan(*bad, 100)
        assert e.value.status == dbm.DBM_EINVAL
