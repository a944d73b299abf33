"""The oracle's pins catch plausible mistakes in the oracle.

Each case below copies the oracle's C source (or its Python front-end),
plants one slip in the copy (a comparison off by one, a dropped term, a
transposed index, a lost compensation, ...), builds it on the CPU and runs the
pin battery of oracle_pinlib against it: every planted mistake must make some
pin fail (or the oracle report an error).  The unchanged copies pass the same battery, so the failures come
from the slips.
"""
import os
import types

import pytest

from oracle import oracle
from oracle_pinlib import pin_battery

# (what the slip is, text in the oracle, text it is replaced with)
MUTANTS = [
    ('power loop runs once too often',
     'for (int e = 0; e < g->f_pow[f]; ++e) p *= x;',
     'for (int e = 0; e <= g->f_pow[f]; ++e) p *= x;'),
    ('1[x <= t] read as 1[x < t]',
     'if (!(x <= g->f_thr[f])) zero = 1;',
     'if (!(x < g->f_thr[f])) zero = 1;'),
    ('1[x > t] read as 1[x >= t]',
     'if (!(x > g->f_thr[f])) zero = 1;',
     'if (!(x >= g->f_thr[f])) zero = 1;'),
    ('indicator ignored',
     'if (!(x > g->f_thr[f])) zero = 1;',
     '(void)x;'),
    ('group cells in column-major order',
     'cell = cell * g->gb_dom[k] + iv;',
     'cell += iv * (k ? g->gb_dom[k - 1] : 1);'),
    ('binary search skips the first match',
     'if (ix->keys[mid] < v) lo = mid + 1;',
     'if (ix->keys[mid] <= v) lo = mid + 1;'),
    ('only the first matching child row joins',
     '    extend(P, pos + 1, cur, A);\n  }',
     '    extend(P, pos + 1, cur, A);\n    break;\n  }'),
    ('child rows with a larger key join too',
     'i < ix->n && ix->keys[i] == key;',
     'i < ix->n && ix->keys[i] >= key;'),
    ('second shared attribute not compared',
     'for (int q = 1; q < e->n_eq && ok; ++q)',
     'for (int q = 1; q < 1 && ok; ++q)'),
    ('FP32 column read as int32',
     'case ORC_F32: return (double)((const float*)rel->data[col])[row];',
     'case ORC_F32: return (double)((const int32_t*)rel->data[col])[row];'),
    ('compensation with the wrong sign',
     'if (fabs(*s) >= fabs(v)) *c += (*s - t) + v;',
     'if (fabs(*s) >= fabs(v)) *c -= (*s - t) + v;'),
    ('compensation dropped at the end',
     'out_sum[i] = s + c;',
     'out_sum[i] = s;'),
    ('per-thread compensation not combined',
     'neumaier_add(&s, &c, acc[t].comp[i]);',
     ''),
    ('SUM(|value|) keeps the sign',
     'A->abs[g->offset + cell] += fabs(v);',
     'A->abs[g->offset + cell] += v;'),
    ('last root rows of a thread dropped',
     'e = root_begin + total * (t + 1) / nt;',
     'e = root_begin + total / nt * (t + 1);'),
]


# the same for the Python front-end that marshals schemas and batches
FRONT_END_MUTANTS = [
    ('only the declared key compared between parent and child',
     "shared = [key] + [n for n in pr.names() if n in cr.names() and n != key]",
     "shared = [key]"),
    ('thresholds truncated to integers',
     "[float(f[2]) if f[1] != 'pow' else 0.0 for f in agg.factors]",
     "[float(int(f[2])) if f[1] != 'pow' else 0.0 for f in agg.factors]"),
    ('every power taken as 1',
     "_i32([int(f[2]) if f[1] == 'pow' else 0 for f in agg.factors])",
     "_i32([1 if f[1] == 'pow' else 0 for f in agg.factors])"),
    ('last root row left out',
     "b, e = (0, rels[root].nrows) if root_range is None else root_range",
     "b, e = (0, rels[root].nrows - 1) if root_range is None else root_range"),
    ('group-by domains reversed',
     "dom = [int(col.cat_domain) for _, _, col in gb]",
     "dom = [int(col.cat_domain) for _, _, col in gb][::-1]"),
]


def _front_end(text):
    mod = types.ModuleType('oracle_front_end_copy')
    mod.__file__ = oracle.__file__
    exec(compile(text, oracle.__file__, 'exec'), mod.__dict__)
    return mod


def _build(tmp_path, name, text):
    src = os.path.join(tmp_path, f'{name}.c')
    with open(src, 'w') as f:
        f.write(text)
    return oracle.load_library(oracle.build(force=True, src=src,
                                            out=os.path.join(tmp_path, f'lib{name}.so')))


def _source():
    with open(oracle.SRC) as f:
        return f.read()


def test_unchanged_copy_passes(tmp_path):
    pin_battery(_build(str(tmp_path), 'control', _source()))


@pytest.mark.parametrize('what,old,new', MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, what, old, new):
    text = _source()
    assert text.count(old) == 1, f'mutation site not unique or missing: {what}'
    lib = _build(str(tmp_path), 'mutant', text.replace(old, new))
    with pytest.raises((AssertionError, RuntimeError)):
        pin_battery(lib)


def _front_end_source():
    with open(oracle.__file__) as f:
        return f.read()


def test_unchanged_front_end_copy_passes():
    pin_battery(evaluate=_front_end(_front_end_source()).evaluate)


@pytest.mark.parametrize('what,old,new', FRONT_END_MUTANTS, ids=[m[0] for m in FRONT_END_MUTANTS])
def test_planted_front_end_mistake_is_caught(what, old, new):
    text = _front_end_source()
    assert text.count(old) == 1, f'mutation site not unique or missing: {what}'
    with pytest.raises((AssertionError, RuntimeError)):
        pin_battery(evaluate=_front_end(text.replace(old, new)).evaluate)
