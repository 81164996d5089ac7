"""Oracle runs for the full-size parity tests, executed in worker processes
(started with the spawn method) while the GPU side of the tests runs.  Only
the oracle and the seeded input generators are imported here: a worker
never touches the GPU.  Each job returns the oracle's arrays for the
comparison, so the expected values come from the oracle alone."""
from __future__ import annotations

import numpy as np

KEEP = ("q", "qhat", "xi", "qxi", "modes", "mask", "qd", "bytes", "stats")


def _slim(r):
    return {k: r[k] for k in KEEP if k in r}


def whole_field(workload, eb, pred):
    """The oracle over a whole named workload at relative bound eb."""
    import oracle
    from paper_2510_25143_gb300 import synth
    uv, _ = synth.workload(workload)
    return _slim(oracle.compress(uv, eb, pred=pred))


def leading_slices(uv_head, eps, pred, t_end, model=None):
    """The oracle on the first t_end + 1 slices of a field, with the field's
    absolute bound eps.  Alg. 3 bounds and encodes slice t from slices t-1,
    t and t+1 only (the incident faces of a vertex and the predictors reach
    no further), so slices 0 .. t_end-1 of this run equal those of a run
    over the whole field whenever the fixed-point scale is the same (the
    caller checks that premise)."""
    import oracle
    return _slim(oracle.compress(uv_head, eps, eb_mode="abs", pred=pred, t_end=t_end, model=model))


def stream_of(uv, eb, pred):
    """The oracle's stream of one field (no debug arrays)."""
    import oracle
    return oracle.compress(np.ascontiguousarray(uv), eb, pred=pred, debug=False)["bytes"]
