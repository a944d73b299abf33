"""Pins for the CPU oracle that do not use the oracle: the natural join by
brute force, a join on more than one shared attribute, and an ill-conditioned
sum whose exact value is known.

`pin_battery(lib, evaluate)` runs all of them against an oracle library
handle and front-end and raises AssertionError on the first that fails;
tests/test_oracle_pins.py runs them on the oracle itself,
tests/test_oracle_mutants.py on copies of the oracle with one planted mistake
each.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from oracle import oracle
from workloads import Agg, Column, Relation, Schema, covar_batch, tiny_schema


def brute_force(schema, batch):
    """Cartesian product of all relations; keep the tuples that agree on
    every attribute name two relations share (the natural join, Sec. 1.1) and
    evaluate each aggregate literally.  Returns (values, join size, SUM|value|):
    int64 counts for products of indicators, fsum-exact float64 sums else."""
    rels = schema.relations
    cells = []
    out = []
    for agg in batch:
        dom = [_domain(schema, g) for g in agg.group_by]
        n = int(np.prod(dom)) if dom else 1
        is_count = all(f[1] != 'pow' for f in agg.factors)
        cells.append((dom, is_count))
        out.append([0] * n if is_count else [[] for _ in range(n)])
    size = 0
    for combo in itertools.product(*[range(r.nrows) for r in rels]):
        vals = {}
        ok = True
        for r, row in zip(rels, combo):
            for c in r.columns:
                v = c.data[row].item()
                if c.name in vals and vals[c.name] != v:
                    ok = False
                    break
                vals[c.name] = v
            if not ok:
                break
        if not ok:
            continue
        size += 1
        for a, agg in enumerate(batch):
            v = 1.0
            for attr, kind, p in agg.factors:
                x = vals[attr]
                if kind == 'pow':
                    v *= x ** int(p)
                elif kind == 'le':
                    v *= 1.0 if x <= p else 0.0
                else:
                    v *= 1.0 if x > p else 0.0
            dom, is_count = cells[a]
            cell = 0
            for g, d in zip(agg.group_by, dom):
                cell = cell * d + int(vals[g])
            if is_count:
                out[a][cell] += int(v)
            else:
                out[a][cell].append(v)
    res, absv = [], []
    for a in range(len(batch)):
        if cells[a][1]:
            res.append(np.array(out[a], np.int64))
            absv.append(None)
        else:
            res.append(np.array([math.fsum(c) for c in out[a]], np.float64))
            absv.append(np.array([math.fsum(abs(x) for x in c) for c in out[a]], np.float64))
    return res, size, absv


def _domain(schema, attr):
    for r in schema.relations:
        for c in r.columns:
            if c.name == attr:
                return c.cat_domain
    raise KeyError(attr)


def assert_close(got, want, rel=1e-12, absolute=1e-12):
    np.testing.assert_allclose(got, want, rtol=rel, atol=absolute)


def check_against_brute_force(schema, batch, nthreads=1, lib=None, evaluate=None):
    """The oracle's values, SUM(|value|) and join size equal the brute force's."""
    res = (evaluate or oracle.evaluate)(schema, batch, nthreads=nthreads, lib=lib)
    want, size, want_abs = brute_force(schema, batch)
    assert res.join_size == size, (res.join_size, size)
    for a in range(len(batch)):
        if res.kinds[a] == 'count':
            assert np.array_equal(res.values[a], want[a]), (a, batch[a])
        else:
            assert_close(res.values[a], want[a])
            assert_close(res.abs[a], want_abs[a])


# ----------------------------------------------------------------------------
def shared_attribute_schema(seed: int):
    """R(a, b, x) joined to S(a, b, u, y) joined to U(u, z): R and S share two
    attributes, so the natural join also requires R.b = S.b (Sec. 3.1 joins a
    child to its parent on every attribute the two have in common)."""
    rng = np.random.Generator(np.random.Philox(seed))
    nr, ns, nu = 9, 8, 4
    R = Relation('R', [
        Column('a', 'key', rng.integers(0, 3, nr).astype(np.int32)),
        Column('b', 'cat', rng.integers(0, 3, nr).astype(np.int32), 3),
        Column('x', 'cont', (rng.integers(-3, 4, nr) + rng.random(nr).round(2)).astype(np.float64))])
    S = Relation('S', [
        Column('a', 'key', rng.integers(0, 3, ns).astype(np.int32)),
        Column('b', 'cat', rng.integers(0, 3, ns).astype(np.int32), 3),
        Column('u', 'key', rng.integers(0, 3, ns).astype(np.int32)),
        Column('y', 'cont', (rng.integers(-3, 4, ns) + rng.random(ns).round(2)).astype(np.float64))])
    U = Relation('U', [
        Column('u', 'key', rng.integers(0, 3, nu).astype(np.int32)),
        Column('z', 'cont', (rng.integers(-3, 4, nu) + rng.random(nu).round(2)).astype(np.float64))])
    sch = Schema([R, S, U], [('R', 'S', 'a'), ('S', 'U', 'u')], 'R')
    batch = covar_batch(['x', 'y', 'z']) + [Agg(group_by=('b',)),
                                            Agg(group_by=('b',), factors=(('y', 'pow', 1),))]
    return sch, batch


def ill_conditioned_schema():
    """One relation whose column sums to 4 through terms of size 1e16: a plain
    double sum returns a multiple of 2 that is wrong, a compensated sum the
    exact 4 (the oracle keeps its sums with Neumaier compensation)."""
    x = np.array([1e16, 1.0, -1e16, 1.0, 1e16, 1.0, -1e16, 1.0], np.float64)
    sch = Schema([Relation('R', [Column('x', 'cont', x)])], [], 'R')
    return sch, [Agg(factors=(('x', 'pow', 1),))], math.fsum(x.tolist())


def check_compensated_sum(lib=None, nthreads=1, evaluate=None):
    sch, batch, want = ill_conditioned_schema()
    res = (evaluate or oracle.evaluate)(sch, batch, nthreads=nthreads, lib=lib)
    assert want == 4.0
    assert res.values[0][0] == want, res.values[0][0]


# ----------------------------------------------------------------------------
TINY_SEEDS = list(range(1000, 1040))


def pin_battery(lib=None, evaluate=None):
    """Every pin of this module, against one oracle library and front-end."""
    check_compensated_sum(lib, nthreads=1, evaluate=evaluate)
    check_compensated_sum(lib, nthreads=3, evaluate=evaluate)
    for seed in range(3):
        sch, batch = shared_attribute_schema(seed)
        check_against_brute_force(sch, batch, 1 + seed % 2, lib, evaluate)
    for seed in TINY_SEEDS:
        sch, batch = tiny_schema(seed, unique_keys=(seed % 4 == 3))
        check_against_brute_force(sch, batch, 1 + seed % 3, lib, evaluate)
    for seed in TINY_SEEDS[:12]:
        sch, batch = tiny_schema(seed, feat_dtype=np.float32)
        check_against_brute_force(sch, batch, 1 + seed % 2, lib, evaluate)
