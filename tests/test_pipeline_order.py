"""The encoder pipeline's ticket order (host logic, no GPU): every wave item
waits only for items with smaller tickets, so a launch in which every warp is
resident always progresses.

A wave item (t, s) encodes rows 32s..32s+31 of slice t in the raster order of
Alg. 3.  From the method, its waits are:
  * the strip above (row 32s-1 of slice t, a raster predecessor);
  * slice t-1 under its faces and its 3-D Lorenzo stencil (Alg. 4 and
    Sec. VI: rows i-1 and i for row i), i.e. strips s-1 and s of slice t-1;
  * with prediction units (SL, MoP, learned; Sec. VI-A/B), the footprint of
    the units covering its rows: slice t-1 down to row 32s+31+R (R the
    back-trace reach), whose last strip enqueues them.
The tests derive these waits independently of the key formula the library
uses and check them against the library's order, for single fields and for
merged batches (where each field must also keep its own order)."""
import itertools

import numpy as np
import pytest

from paper_2510_25143_gb300 import cpt


def _waits(t, s, H, R, units):
    nstrips = (H + 31) // 32
    w = []
    if s >= 1:
        w.append((t, s - 1))
    if t >= 1:
        w += [(t - 1, x) for x in (s - 1, s) if x >= 0]
        if units:
            last = min(nstrips - 1, (32 * s + 31 + R) // 32)
            w += [(t - 1, x) for x in range(s + 1, last + 1)]
    return w


def _check(fields, schedule=None):
    order = cpt.pipeline_order(fields, schedule)
    n_items = sum(T * ((H + 31) // 32) for T, H, _, _ in fields)
    assert order.shape == (n_items, 3)
    pos = {tuple(int(v) for v in row): x for x, row in enumerate(order)}
    assert len(pos) == n_items  # every item exactly once
    for f, (T, H, R, units) in enumerate(fields):
        for t in range(T):
            for s in range((H + 31) // 32):
                me = pos[(f, t, s)]
                for (tw, sw) in _waits(t, s, H, R, units):
                    assert pos[(f, tw, sw)] < me, ((T, H, R, units), schedule, (t, s), (tw, sw))
    return order


@pytest.mark.parametrize("schedule", [None, (0, 0, 1, 0, 0), (0, 0, 8, 0, 0), (0, 0, 32, 0, 0),
                                      (30, 0, 0, 32, 3), (60, 0, 0, 128, 0), (0, 0, 0, 1, 0)])
def test_single_field_waits_for_smaller_tickets(schedule):
    for T, H in itertools.product([1, 2, 5], [1, 31, 32, 33, 100, 512]):
        _check([(T, H, 0, 0)], schedule)
        for R in (1, 5, 31, 32, 33, 70):
            _check([(T, H, R, 1)], schedule)


def test_batch_merge_keeps_each_field_order():
    rng = np.random.default_rng(5)
    fields = []
    for _ in range(12):
        units = int(rng.integers(0, 2))
        fields.append((int(rng.integers(1, 9)), int(rng.integers(1, 300)), int(rng.integers(1, 60)) * units, units))
    for schedule in (None, (45, 0, 0, 64, 0), (0, 0, 3, 96, 0)):
        order = _check(fields, schedule)
        for f, fld in enumerate(fields):
            alone = cpt.pipeline_order([fld], schedule)
            mine = order[order[:, 0] == f]
            assert (mine[:, 1:] == alone[:, 1:]).all()


def test_arguments():
    with pytest.raises(cpt.CptError):
        cpt.pipeline_order([(0, 10, 0, 0)])
    with pytest.raises(cpt.CptError):
        cpt.pipeline_order([(3, 10, -1, 1)])
    assert cpt.pipeline_order([(2, 33, 0, 0)]).shape == (4, 3)
