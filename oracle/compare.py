"""The error rule of the parity checks, applied to engine results against an
oracle result.  TEST INFRASTRUCTURE ONLY (tests, smoke check, the benchmark's
accuracy and CPU-baseline legs).

Per aggregate cell: counts must be bit-exact; a sum g with oracle value r and
oracle scale A = SUM(|value|) must satisfy
    |g - r| <= 1e-6 * max(|r|, 1e-3 * A),
a relative error of 1e-6 wherever the sum is not a cancellation of terms 1000x
larger than itself.

Small inputs: the engine multiplies in 24-bit precision (FP32 products, or the
three-way bf16 split), so one product carries a relative error up to 2^-24 and
a sum of products an error up to about 2^-24 * A.  With few rows the rule above
can be tighter than that (its floor 1e-9 * A only dominates the statistical
2^-24 * sqrt(sum v^2) once the sum has ~10^4 terms), so checks on small or
ragged sizes may also accept |g - r| <= ARITH_FLOOR * A.  Checks on the
benchmark configurations use the rule alone (arith_floor=0).
"""
from __future__ import annotations

import numpy as np

REL_TOL = 1e-6
COND_FLOOR = 1e-3
ARITH_FLOOR = 2.0 ** -21


def compare(got, want, arith_floor=0.0):
    """Return (failures, stats).  `want` is an oracle.OracleResult."""
    fails = []
    max_rel = 0.0
    max_ratio = 0.0
    for a, (g, r) in enumerate(zip(got, want.values)):
        g = np.asarray(g)
        if want.kinds[a] == 'count':
            if g.shape != r.shape or not np.array_equal(g.astype(np.int64), r):
                bad = np.nonzero(g != r)[0][:5] if g.shape == r.shape else 'shape'
                fails.append((a, 'count', bad))
            continue
        A = want.abs[a]
        err = np.abs(g - r)
        allow = np.maximum(REL_TOL * np.maximum(np.abs(r), COND_FLOOR * A), arith_floor * A)
        with np.errstate(divide='ignore', invalid='ignore'):
            rel = np.where(np.abs(r) > 0, err / np.abs(r), np.where(err > 0, np.inf, 0.0))
            ratio = np.where(allow > 0, err / allow, np.where(err > 0, np.inf, 0.0))
        if rel.size:
            max_rel = max(max_rel, float(np.max(rel[np.isfinite(rel)], initial=0.0)))
            max_ratio = max(max_ratio, float(np.max(ratio)))
        if np.any(err > allow):
            i = int(np.argmax(err - allow))
            fails.append((a, 'sum', dict(cell=i, got=float(g[i]), want=float(r[i]), A=float(A[i]))))
    return fails, {'max_raw_rel_err': max_rel, 'max_err_over_allowed': max_ratio}


def result_kind(agg) -> str:
    """Which part of the engine produces an aggregate: 'count' (COUNT, possibly
    grouped: exact integers), 'gram' (an ungrouped SUM of a degree <= 2
    monomial: the covar matrix), 'grouped' (a grouped SUM) or 'filtered' (a
    SUM under threshold indicators)."""
    kinds = [f[1] for f in agg.factors]
    if any(k in ('le', 'gt') for k in kinds):
        return 'filtered' if any(k == 'pow' for k in kinds) else 'count'
    if not kinds:
        return 'count'
    return 'grouped' if agg.group_by else 'gram'


def compare_by_kind(batch, got, want) -> dict:
    """The error statistics of compare() for each result kind of the batch
    (result_kind), with the number of aggregates and failures of each."""
    out = {}
    for kind in ('gram', 'grouped', 'filtered', 'count'):
        idx = [i for i, a in enumerate(batch) if result_kind(a) == kind]
        if not idx:
            continue
        sub = type(want)([want.kinds[i] for i in idx], [want.shapes[i] for i in idx], [want.values[i] for i in idx],
                         [want.abs[i] for i in idx], want.join_size)
        fails, stats = compare([got[i] for i in idx], sub)
        out[kind] = {'aggregates': len(idx), 'failures': len(fails), **stats}
    return out
