"""Python front-end of the CPU oracle (lmf_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg; the GPU library never imports it.

`evaluate(schema, batch)` returns, for every aggregate of the batch, its exact
value over the natural join (Sec. 1.1): an int64 array for counts (products of
indicators only) or a float64 array of sums with the matching SUM(|value|)
array, each of shape (n_groups,) with groups in row-major order of the
group-by attributes' values.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, 'lmf_oracle.c')
LIB = os.path.join(HERE, '_build', 'liblmf_oracle.so')

_lock = threading.Lock()
_lib = None

I32, F32, F64 = 0, 1, 2
POW, LE, GT = 0, 1, 2
_KIND = {'pow': POW, 'le': LE, 'gt': GT}


def build(force: bool = False, src: str = SRC, out: str = LIB) -> str:
    """Compile the oracle with the host C compiler (OpenMP when available).
    `src`/`out` default to this package's source and library; the tests that
    plant mistakes in a copy of the source build that copy the same way."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    tmp = out + f'.{os.getpid()}.tmp'
    base = ['gcc', '-O2', '-std=c11', '-fPIC', '-shared', src, '-o', tmp, '-lm']
    try:
        subprocess.run(base[:1] + ['-fopenmp'] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, out)
    return out


class _Rel(ctypes.Structure):
    _fields_ = [('nrows', ctypes.c_int64), ('ncols', ctypes.c_int32),
                ('dtypes', ctypes.POINTER(ctypes.c_int32)),
                ('data', ctypes.POINTER(ctypes.c_void_p))]


class _Edge(ctypes.Structure):
    _fields_ = [('parent', ctypes.c_int32), ('child', ctypes.c_int32), ('n_eq', ctypes.c_int32),
                ('parent_cols', ctypes.POINTER(ctypes.c_int32)),
                ('child_cols', ctypes.POINTER(ctypes.c_int32))]


class _Agg(ctypes.Structure):
    _fields_ = [('n_group_by', ctypes.c_int32),
                ('gb_rel', ctypes.POINTER(ctypes.c_int32)),
                ('gb_col', ctypes.POINTER(ctypes.c_int32)),
                ('gb_dom', ctypes.POINTER(ctypes.c_int32)),
                ('n_factors', ctypes.c_int32),
                ('f_rel', ctypes.POINTER(ctypes.c_int32)),
                ('f_col', ctypes.POINTER(ctypes.c_int32)),
                ('f_kind', ctypes.POINTER(ctypes.c_int32)),
                ('f_pow', ctypes.POINTER(ctypes.c_int32)),
                ('f_thr', ctypes.POINTER(ctypes.c_double)),
                ('is_count', ctypes.c_int32),
                ('offset', ctypes.c_int64)]


def load_library(path: str):
    """ctypes handle of a compiled oracle library with its signatures set."""
    lib = ctypes.CDLL(path)
    lib.orc_evaluate.restype = ctypes.c_int
    lib.orc_evaluate.argtypes = [
        ctypes.c_int, ctypes.POINTER(_Rel), ctypes.c_int, ctypes.c_int,
        ctypes.POINTER(_Edge), ctypes.c_int, ctypes.POINTER(_Agg),
        ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
        ctypes.POINTER(ctypes.c_int64)]
    lib.orc_max_threads.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
    return _lib


def max_threads(lib=None) -> int:
    return int((lib if lib is not None else _load()).orc_max_threads())


def _i32(seq) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(seq, dtype=np.int32))


class OracleResult:
    def __init__(self, kinds, shapes, values, abs_values, join_size):
        self.kinds: List[str] = kinds          # 'count' or 'sum' per aggregate
        self.shapes: List[tuple] = shapes      # group-by domain sizes per aggregate
        self.values: List[np.ndarray] = values
        self.abs: List[Optional[np.ndarray]] = abs_values
        self.join_size: int = join_size


def evaluate(schema, batch: Sequence, root_range=None, nthreads: Optional[int] = None,
             lib=None) -> OracleResult:
    """`lib`: a handle from load_library() to evaluate with instead of this
    package's library."""
    lib = lib if lib is not None else _load()
    rels = schema.relations
    rindex = {r.name: i for i, r in enumerate(rels)}
    keep = []   # keep every buffer alive across the call

    c_rels = (_Rel * len(rels))()
    for i, r in enumerate(rels):
        dts, ptrs = [], []
        for c in r.columns:
            a = np.ascontiguousarray(c.data)
            if a.dtype == np.int32:
                dts.append(I32)
            elif a.dtype == np.float32:
                dts.append(F32)
            elif a.dtype == np.float64:
                dts.append(F64)
            else:
                raise TypeError(f'{r.name}.{c.name}: dtype {a.dtype}')
            keep.append(a)
            ptrs.append(a.ctypes.data if a.size else 0)
        dt = _i32(dts)
        pa = (ctypes.c_void_p * max(1, len(ptrs)))(*ptrs)
        keep += [dt, pa]
        c_rels[i].nrows = r.nrows
        c_rels[i].ncols = len(r.columns)
        c_rels[i].dtypes = dt.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        c_rels[i].data = ctypes.cast(pa, ctypes.POINTER(ctypes.c_void_p))

    c_edges = (_Edge * max(1, len(schema.edges)))()
    for e, (p, c, key) in enumerate(schema.edges):
        pr, cr = rels[rindex[p]], rels[rindex[c]]
        shared = [key] + [n for n in pr.names() if n in cr.names() and n != key]
        pc = _i32([pr.names().index(n) for n in shared])
        cc = _i32([cr.names().index(n) for n in shared])
        keep += [pc, cc]
        c_edges[e].parent = rindex[p]
        c_edges[e].child = rindex[c]
        c_edges[e].n_eq = len(shared)
        c_edges[e].parent_cols = pc.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        c_edges[e].child_cols = cc.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))

    def locate(attr):
        for i, r in enumerate(rels):
            if attr in r.names():
                return i, r.names().index(attr), r.col(attr)
        raise KeyError(attr)

    c_aggs = (_Agg * max(1, len(batch)))()
    kinds, shapes = [], []
    n_sum = n_cnt = 0
    offsets = []
    for a, agg in enumerate(batch):
        gb = [locate(g) for g in agg.group_by]
        dom = [int(col.cat_domain) for _, _, col in gb]
        fr = [locate(f[0]) for f in agg.factors]
        is_count = all(f[1] != 'pow' for f in agg.factors)
        ncell = int(np.prod(dom)) if dom else 1
        arrs = [_i32([g[0] for g in gb]), _i32([g[1] for g in gb]), _i32(dom),
                _i32([f[0] for f in fr]), _i32([f[1] for f in fr]),
                _i32([_KIND[f[1]] for f in agg.factors]),
                _i32([int(f[2]) if f[1] == 'pow' else 0 for f in agg.factors]),
                np.ascontiguousarray(np.asarray(
                    [float(f[2]) if f[1] != 'pow' else 0.0 for f in agg.factors], np.float64))]
        keep += arrs
        P = lambda x: x.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))  # noqa: E731
        c_aggs[a].n_group_by = len(gb)
        c_aggs[a].gb_rel, c_aggs[a].gb_col, c_aggs[a].gb_dom = P(arrs[0]), P(arrs[1]), P(arrs[2])
        c_aggs[a].n_factors = len(agg.factors)
        c_aggs[a].f_rel, c_aggs[a].f_col, c_aggs[a].f_kind = P(arrs[3]), P(arrs[4]), P(arrs[5])
        c_aggs[a].f_pow = P(arrs[6])
        c_aggs[a].f_thr = arrs[7].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        c_aggs[a].is_count = int(is_count)
        if is_count:
            c_aggs[a].offset = n_cnt
            offsets.append(n_cnt)
            n_cnt += ncell
        else:
            c_aggs[a].offset = n_sum
            offsets.append(n_sum)
            n_sum += ncell
        kinds.append('count' if is_count else 'sum')
        shapes.append(tuple(dom))

    out_sum = np.zeros(max(1, n_sum), np.float64)
    out_abs = np.zeros(max(1, n_sum), np.float64)
    out_cnt = np.zeros(max(1, n_cnt), np.int64)
    js = ctypes.c_int64(0)
    root = rindex[schema.root]
    b, e = (0, rels[root].nrows) if root_range is None else root_range
    nt = max_threads(lib) if nthreads is None else int(nthreads)
    rc = lib.orc_evaluate(len(rels), c_rels, root, len(schema.edges), c_edges, len(batch),
                          c_aggs, n_sum, n_cnt, int(b), int(e), nt,
                          out_sum.ctypes.data, out_abs.ctypes.data, out_cnt.ctypes.data,
                          ctypes.byref(js))
    if rc != 0:
        raise RuntimeError(f'oracle failed with status {rc}')
    values, absv = [], []
    for a in range(len(batch)):
        n = int(np.prod(shapes[a])) if shapes[a] else 1
        o = offsets[a]
        if kinds[a] == 'count':
            values.append(out_cnt[o:o + n].copy())
            absv.append(None)
        else:
            values.append(out_sum[o:o + n].copy())
            absv.append(out_abs[o:o + n].copy())
    return OracleResult(kinds, shapes, values, absv, int(js.value))
