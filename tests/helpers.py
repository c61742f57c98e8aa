"""Test-side glue between the seeded workloads and the CPU oracle."""
import numpy as np

import oracle
from paper_1608_01966_gb300 import masks_to_dense


def oracle_params(case):
    return oracle.params(case.C, case.S, case.n_in, case.thr, case.inc, case.dec,
                         case.min_overlap, case.k, case.inhibition, case.gw, case.gh,
                         case.radius)


def oracle_run(case, frames_u8, learn, perm=None, want_ov=False):
    """Run the oracle over frames from `perm` (default: the case's initial
    permanences, copied).  Returns (active [n][C] u8, perm, ov or None)."""
    p = (case.perm if perm is None else perm).copy()
    r = oracle.run(oracle_params(case), case.idx, p, case.boost, frames_u8, learn,
                   want_ov=want_ov)
    if want_ov:
        act, ov = r
        return act, p, ov
    return r, p, None


def dense(masks, C):
    return masks_to_dense(masks, C)


def first_diff(a, b):
    d = np.argwhere(np.asarray(a) != np.asarray(b))
    return None if d.size == 0 else tuple(d[0])
