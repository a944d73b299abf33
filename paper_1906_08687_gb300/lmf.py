"""Thin ctypes binding of the C ABI in include/lmf.h (argument marshalling only).

Every computation runs in liblmf.so's CUDA kernels.  Loading fails loudly
when the library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import build as _build

# status codes and enums (include/lmf.h)
LMF_OK = 0
LMF_ERR_ARG, LMF_ERR_NOT_TREE, LMF_ERR_DTYPE, LMF_ERR_KEY = -1, -2, -3, -4
LMF_ERR_OOM, LMF_ERR_CUDA, LMF_ERR_TIMEOUT, LMF_ERR_OVERFLOW = -5, -6, -7, -8
LMF_ERR_STATE, LMF_ERR_UNSUPPORTED = -9, -10
LMF_I32, LMF_F32, LMF_F64, LMF_I64 = 0, 1, 2, 3
LMF_KEY, LMF_CONT, LMF_CAT = 0, 1, 2
LMF_POW, LMF_LE, LMF_GT = 0, 1, 2
LMF_PREC_PLAIN_FP32, LMF_PREC_SPLIT_BF16 = 0, 1
LMF_BATCH_SINGLE, LMF_BATCH_GRAPH = 0, 1
LMF_ROOT_DECLARED, LMF_ROOT_EXPLICIT, LMF_ROOT_HEURISTIC, LMF_ROOT_PER_QUERY = 0, 1, 2, 3
LMF_MAX_GROUP_BY = 3
LMF_STAGES = 5
LMF_PLAN_FEATURES = 26
LMF_PLAN_NO_JIT = 1
LMF_PLAN_ROW_GRAM = 2
LMF_DEVICE, LMF_HOST_COPY, LMF_HOST_MAPPED = 0, 1, 2
STAGE_NAMES = ['input', 'views', 'root_scan', 'tree', 'finalize']

_ROLE = {'key': LMF_KEY, 'cont': LMF_CONT, 'cat': LMF_CAT}
_KIND = {'pow': LMF_POW, 'le': LMF_LE, 'gt': LMF_GT}


class lmf_column(ctypes.Structure):
    _fields_ = [('name', ctypes.c_char_p), ('dtype', ctypes.c_int32), ('role', ctypes.c_int32),
                ('data', ctypes.c_void_p), ('cat_domain', ctypes.c_int32),
                ('on_host', ctypes.c_int32)]


class lmf_factor(ctypes.Structure):
    _fields_ = [('attr', ctypes.c_char_p), ('kind', ctypes.c_int32), ('power', ctypes.c_int32),
                ('threshold', ctypes.c_double)]


class lmf_agg_spec(ctypes.Structure):
    _fields_ = [('n_group_by', ctypes.c_int32), ('group_by', ctypes.c_char_p * LMF_MAX_GROUP_BY),
                ('n_factors', ctypes.c_int32), ('factors', ctypes.POINTER(lmf_factor))]


class lmf_plan_opts(ctypes.Structure):
    _fields_ = [('precision', ctypes.c_int32), ('batching', ctypes.c_int32),
                ('tile_rows', ctypes.c_int32), ('ctas_per_sm', ctypes.c_int32),
                ('root_mode', ctypes.c_int32), ('root_rel', ctypes.c_int32),
                ('no_merge', ctypes.c_int32), ('flags', ctypes.c_int32)]


class lmf_plan_stats(ctypes.Structure):
    _fields_ = [('n_views', ctypes.c_int32), ('n_probe_groups', ctypes.c_int32),
                ('z_len', ctypes.c_int32), ('n_gram_aggs', ctypes.c_int32),
                ('n_grouped_aggs', ctypes.c_int32), ('n_filtered_aggs', ctypes.c_int32),
                ('n_kernels_per_run', ctypes.c_int32), ('unique_keys', ctypes.c_int32),
                ('root_grid', ctypes.c_int32), ('precision', ctypes.c_int32),
                ('root_rel', ctypes.c_int32), ('merged', ctypes.c_int32),
                ('tree_nodes', ctypes.c_int32), ('tree_groups', ctypes.c_int32),
                ('tree_slices', ctypes.c_int32), ('tree_split_w', ctypes.c_int32),
                ('tree_node_w', ctypes.c_int32), ('tree_ctas_per_sm', ctypes.c_int32),
                ('tree_chunk', ctypes.c_int32),
                ('root_rows', ctypes.c_int64), ('scratch_bytes', ctypes.c_int64),
                ('resident_group', ctypes.c_int32), ('resident_cells', ctypes.c_int32),
                ('jit', ctypes.c_int32), ('key_level', ctypes.c_int32), ('n_roots', ctypes.c_int32)]


class lmf_mi_pair(ctypes.Structure):
    _fields_ = [('beta', ctypes.c_void_p), ('gamma', ctypes.c_void_p), ('delta', ctypes.c_void_p),
                ('dom_i', ctypes.c_int32), ('dom_j', ctypes.c_int32)]


# every symbol include/lmf.h declares, with its ctypes signature
_P = ctypes.c_void_p
_I = ctypes.c_int
_SIGNATURES = {
    'lmf_create': (_I, [_I, ctypes.POINTER(_P)]),
    'lmf_destroy': (_I, [_P]),
    'lmf_register_relation': (_I, [_P, ctypes.c_char_p, ctypes.c_int64, ctypes.POINTER(lmf_column),
                                   _I, ctypes.POINTER(_I)]),
    'lmf_declare_join': (_I, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I),
                              ctypes.POINTER(ctypes.c_char_p)]),
    'lmf_declare_batch': (_I, [_P, ctypes.POINTER(lmf_agg_spec), _I, ctypes.POINTER(_I)]),
    'lmf_plan': (_I, [_P, _I, ctypes.POINTER(lmf_plan_opts)]),
    'lmf_plan_info': (_I, [_P, _I, ctypes.POINTER(lmf_plan_stats)]),
    'lmf_run': (_I, [_P, _I, _P]),
    'lmf_sync': (_I, [_P, _I]),
    'lmf_run_profiled': (_I, [_P, _I, _P, ctypes.POINTER(ctypes.c_float)]),
    'lmf_result_info': (_I, [_P, _I, _I, ctypes.POINTER(ctypes.c_int64),
                             ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)]),
    'lmf_result_sizes': (_I, [_P, _I, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    'lmf_read_results': (_I, [_P, _I, _P, _P, _I, _P]),
    'lmf_read_result': (_I, [_P, _I, _I, _P]),
    'lmf_plan_candidates': (_I, [_P, _I, ctypes.POINTER(lmf_plan_opts), ctypes.POINTER(lmf_plan_opts), _I,
                                 ctypes.POINTER(_I)]),
    'lmf_plan_features': (_I, [_P, _I, ctypes.POINTER(ctypes.c_float), _I]),
    'lmf_plan_learned': (_I, [_P, _I, _P, ctypes.POINTER(lmf_plan_opts), ctypes.POINTER(lmf_plan_opts)]),
    'lmf_plan_precompile': (_I, [_P, _I, ctypes.POINTER(lmf_plan_opts), _I, ctypes.POINTER(_I)]),
    'lmf_mlp_create': (_I, [_I, _I, _I, ctypes.c_uint64, ctypes.POINTER(_P)]),
    'lmf_mlp_destroy': (_I, [_P]),
    'lmf_mlp_num_params': (_I, [_P, ctypes.POINTER(ctypes.c_int64)]),
    'lmf_mlp_get_params': (_I, [_P, ctypes.POINTER(ctypes.c_float), ctypes.c_int64]),
    'lmf_mlp_set_params': (_I, [_P, ctypes.POINTER(ctypes.c_float), ctypes.c_int64]),
    'lmf_mlp_set_norm': (_I, [_P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                              ctypes.c_float, ctypes.c_float]),
    'lmf_mlp_forward': (_I, [_P, _P, _I, _P]),
    'lmf_mlp_grad': (_I, [_P, _P, _P, _I, _P, ctypes.POINTER(ctypes.c_float)]),
    'lmf_mlp_train_step': (_I, [_P, _P, _P, _I, ctypes.c_float, ctypes.POINTER(ctypes.c_float)]),
    'lmf_gram_noalloc': (_I, [ctypes.POINTER(ctypes.c_void_p), _I, ctypes.c_int64, _P, _P]),
    'lmf_ridge_bgd': (_I, [_P, _I, ctypes.c_double, ctypes.c_double, _I, ctypes.c_double, _P, _P, _P]),
    'lmf_mutual_information': (_I, [_P, _I, ctypes.c_int64, _P, _P]),
    'lmf_chow_liu': (_I, [_P, _I, _P, _P, _P]),
    'lmf_wait_selftest': (_I, [_P]),
    'lmf_status_string': (ctypes.c_char_p, [_I]),
    'lmf_error_message': (ctypes.c_char_p, [_P]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Load liblmf.so; raise if it has not been built (no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise ImportError(f'liblmf.so is not built ({_build.LIB}); run '
                              'paper_1906_08687_gb300.build.build() first')
        lib = ctypes.CDLL(_build.LIB)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class LmfError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ''):
        self.status = status
        msg = load().lmf_status_string(status).decode()
        super().__init__(f'{what}: {msg} ({status}){": " + detail if detail else ""}')


class Engine:
    """One lmf_ctx on one CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = load()
        h = ctypes.c_void_p()
        self._check(self.lib.lmf_create(device, ctypes.byref(h)), 'lmf_create', ctx=False)
        self.ctx = h
        self._keep = []
        self.rel_ids = {}

    # -- helpers --------------------------------------------------------------
    def _check(self, st: int, what: str, ctx: bool = True):
        if st != LMF_OK:
            detail = self.lib.lmf_error_message(self.ctx).decode() if ctx and self.ctx else ''
            raise LmfError(st, what, detail)

    def close(self):
        if getattr(self, 'ctx', None):
            self.lib.lmf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C ABI ------------------------------------------------------------------
    def register_relation(self, name: str, nrows: int, columns: Sequence[dict]) -> int:
        """columns: dicts with name, dtype (LMF_*), role, data (pointer int),
        cat_domain, on_host."""
        arr = (lmf_column * max(1, len(columns)))()
        for i, c in enumerate(columns):
            nm = c['name'].encode()
            self._keep.append(nm)
            arr[i].name = nm
            arr[i].dtype = c['dtype']
            arr[i].role = c['role']
            arr[i].data = c['data']
            arr[i].cat_domain = c.get('cat_domain', 0)
            arr[i].on_host = c.get('on_host', 0)
        rid = ctypes.c_int()
        self._check(self.lib.lmf_register_relation(self.ctx, name.encode(), nrows, arr, len(columns),
                                                   ctypes.byref(rid)), 'lmf_register_relation')
        self.rel_ids[name] = rid.value
        return rid.value

    def declare_join(self, edges: Sequence[Tuple[int, int, str]]):
        n = len(edges)
        par = (ctypes.c_int * max(1, n))(*[e[0] for e in edges])
        chi = (ctypes.c_int * max(1, n))(*[e[1] for e in edges])
        keys = [e[2].encode() for e in edges]
        ka = (ctypes.c_char_p * max(1, n))(*keys)
        self._check(self.lib.lmf_declare_join(self.ctx, n, par, chi, ka), 'lmf_declare_join')

    def declare_batch(self, aggs: Sequence) -> int:
        """aggs: objects with .group_by (names) and .factors ((attr, 'pow'|'le'|'gt', p_or_t))."""
        arr = (lmf_agg_spec * max(1, len(aggs)))()
        for i, a in enumerate(aggs):
            arr[i].n_group_by = len(a.group_by)
            for q, g in enumerate(a.group_by):
                b = g.encode()
                self._keep.append(b)
                arr[i].group_by[q] = b
            fs = (lmf_factor * max(1, len(a.factors)))()
            for q, (attr, kind, val) in enumerate(a.factors):
                b = attr.encode()
                self._keep.append(b)
                fs[q].attr = b
                fs[q].kind = _KIND[kind]
                fs[q].power = int(val) if kind == 'pow' else 0
                fs[q].threshold = float(val) if kind != 'pow' else 0.0
            self._keep.append(fs)
            arr[i].n_factors = len(a.factors)
            arr[i].factors = fs
        bid = ctypes.c_int()
        self._check(self.lib.lmf_declare_batch(self.ctx, arr, len(aggs), ctypes.byref(bid)),
                    'lmf_declare_batch')
        return bid.value

    def plan(self, batch: int, precision: int = LMF_PREC_SPLIT_BF16, batching: int = LMF_BATCH_GRAPH,
             tile_rows: int = 0, ctas_per_sm: int = 0, root_mode: int = 0, root_rel: int = 0,
             no_merge: int = 0, jit: bool = True, key_level: bool = True):
        flags = (0 if jit else LMF_PLAN_NO_JIT) | (0 if key_level else LMF_PLAN_ROW_GRAM)
        o = lmf_plan_opts(precision, batching, tile_rows, ctas_per_sm, root_mode, root_rel, no_merge, flags)
        self._check(self.lib.lmf_plan(self.ctx, batch, ctypes.byref(o)), 'lmf_plan')

    def plan_info(self, batch: int) -> dict:
        s = lmf_plan_stats()
        self._check(self.lib.lmf_plan_info(self.ctx, batch, ctypes.byref(s)), 'lmf_plan_info')
        return {f: getattr(s, f) for f, _ in s._fields_}

    def run(self, batch: int, stream: int = 0):
        self._check(self.lib.lmf_run(self.ctx, batch, ctypes.c_void_p(stream)), 'lmf_run')

    def run_profiled(self, batch: int, stream: int = 0) -> List[float]:
        ms = (ctypes.c_float * LMF_STAGES)()
        self._check(self.lib.lmf_run_profiled(self.ctx, batch, ctypes.c_void_p(stream), ms),
                    'lmf_run_profiled')
        return list(ms)

    def sync(self, batch: int):
        self._check(self.lib.lmf_sync(self.ctx, batch), 'lmf_sync')

    def result_layout(self, batch: int, n_aggs: int) -> List[Tuple[int, int, int]]:
        out = []
        n, dt, off = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64()
        for a in range(n_aggs):
            self._check(self.lib.lmf_result_info(self.ctx, batch, a, ctypes.byref(n), ctypes.byref(dt),
                                                 ctypes.byref(off)), 'lmf_result_info')
            out.append((n.value, dt.value, off.value))
        return out

    def result_sizes(self, batch: int) -> Tuple[int, int]:
        a, b = ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.lmf_result_sizes(self.ctx, batch, ctypes.byref(a), ctypes.byref(b)),
                    'lmf_result_sizes')
        return a.value, b.value

    def read_results(self, batch: int, dst_i64: int, dst_f64: int, dst_is_device: bool,
                     stream: int = 0):
        self._check(self.lib.lmf_read_results(self.ctx, batch, ctypes.c_void_p(dst_i64),
                                              ctypes.c_void_p(dst_f64), int(dst_is_device),
                                              ctypes.c_void_p(stream)), 'lmf_read_results')

    def read_result(self, batch: int, agg: int, dst: int):
        self._check(self.lib.lmf_read_result(self.ctx, batch, agg, ctypes.c_void_p(dst)),
                    'lmf_read_result')

    def wait_selftest(self) -> int:
        """Status of lmf_wait_selftest: LMF_ERR_TIMEOUT when the bounded device
        wait gave up and reported it (expected)."""
        return int(self.lib.lmf_wait_selftest(self.ctx))

    def plan_opts(self, batch: int, opts: 'lmf_plan_opts'):
        self._check(self.lib.lmf_plan(self.ctx, batch, ctypes.byref(opts)), 'lmf_plan')

    def plan_candidates(self, batch: int, base: Optional['lmf_plan_opts'] = None) -> List['lmf_plan_opts']:
        b = base or lmf_plan_opts(LMF_PREC_SPLIT_BF16, LMF_BATCH_GRAPH, 0, 0, 0, 0, 0, 0)
        n = ctypes.c_int()
        self._check(self.lib.lmf_plan_candidates(self.ctx, batch, ctypes.byref(b), None, 0, ctypes.byref(n)),
                    'lmf_plan_candidates')
        arr = (lmf_plan_opts * max(1, n.value))()
        self._check(self.lib.lmf_plan_candidates(self.ctx, batch, ctypes.byref(b), arr, n.value, ctypes.byref(n)),
                    'lmf_plan_candidates')
        return [arr[i] for i in range(n.value)]

    def plan_features(self, batch: int) -> np.ndarray:
        f = np.zeros(LMF_PLAN_FEATURES, np.float32)
        self._check(self.lib.lmf_plan_features(self.ctx, batch, f.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                               LMF_PLAN_FEATURES), 'lmf_plan_features')
        return f

    def plan_precompile(self, batch: int, base: Optional['lmf_plan_opts'] = None, threads: int = 0) -> int:
        b = base or lmf_plan_opts(LMF_PREC_SPLIT_BF16, LMF_BATCH_GRAPH, 0, 0, 0, 0, 0, 0)
        n = ctypes.c_int()
        self._check(self.lib.lmf_plan_precompile(self.ctx, batch, ctypes.byref(b), threads, ctypes.byref(n)),
                    'lmf_plan_precompile')
        return n.value

    def plan_learned(self, batch: int, model: Optional['Mlp'], base: Optional['lmf_plan_opts'] = None
                     ) -> 'lmf_plan_opts':
        b = base or lmf_plan_opts(LMF_PREC_SPLIT_BF16, LMF_BATCH_GRAPH, 0, 0, 0, 0, 0, 0)
        out = lmf_plan_opts()
        self._check(self.lib.lmf_plan_learned(self.ctx, batch, model.h if model else None, ctypes.byref(b),
                                              ctypes.byref(out)), 'lmf_plan_learned')
        return out

    # -- convenience: all results as numpy arrays ------------------------------
    def results(self, batch: int, n_aggs: int) -> List[np.ndarray]:
        n_i64, n_f64 = self.result_sizes(batch)
        i64 = np.zeros(max(1, n_i64), np.int64)
        f64 = np.zeros(max(1, n_f64), np.float64)
        self.read_results(batch, i64.ctypes.data, f64.ctypes.data, False)
        out = []
        for n, dt, off in self.result_layout(batch, n_aggs):
            out.append((i64 if dt == LMF_I64 else f64)[off:off + n].copy())
        return out


class Mlp:
    """The planner's cost model (lmf_mlp): FP32 MLP with hand-written GPU kernels."""

    def __init__(self, in_dim: int = 24, hidden: int = 128, seed: int = 0, device: int = 0):
        self.lib = load()
        h = ctypes.c_void_p()
        st = self.lib.lmf_mlp_create(device, in_dim, hidden, seed, ctypes.byref(h))
        if st != LMF_OK:
            raise LmfError(st, 'lmf_mlp_create')
        self.h = h
        self.in_dim, self.hidden = in_dim, hidden
        n = ctypes.c_int64()
        self.lib.lmf_mlp_num_params(h, ctypes.byref(n))
        self.n_params = n.value

    def close(self):
        if getattr(self, 'h', None):
            self.lib.lmf_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, st, what):
        if st != LMF_OK:
            raise LmfError(st, what)

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.n_params, np.float32)
        self._ck(self.lib.lmf_mlp_get_params(self.h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                             self.n_params), 'lmf_mlp_get_params')
        return p

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, np.float32)
        self._ck(self.lib.lmf_mlp_set_params(self.h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                             self.n_params), 'lmf_mlp_set_params')

    def set_norm(self, mean, std, y_mean: float, y_std: float):
        m = np.ascontiguousarray(mean, np.float32)
        s = np.ascontiguousarray(std, np.float32)
        self._ck(self.lib.lmf_mlp_set_norm(self.h, m.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                           s.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                           float(y_mean), float(y_std)), 'lmf_mlp_set_norm')

    def forward(self, x_dev: int, batch: int, y_dev: int):
        self._ck(self.lib.lmf_mlp_forward(self.h, ctypes.c_void_p(x_dev), batch, ctypes.c_void_p(y_dev)),
                 'lmf_mlp_forward')

    def grad(self, x_dev: int, y_dev: int, batch: int, grad_dev: int) -> float:
        loss = ctypes.c_float()
        self._ck(self.lib.lmf_mlp_grad(self.h, ctypes.c_void_p(x_dev), ctypes.c_void_p(y_dev), batch,
                                       ctypes.c_void_p(grad_dev), ctypes.byref(loss)), 'lmf_mlp_grad')
        return loss.value

    def train_step(self, x_dev: int, y_dev: int, batch: int, lr: float) -> float:
        loss = ctypes.c_float()
        self._ck(self.lib.lmf_mlp_train_step(self.h, ctypes.c_void_p(x_dev), ctypes.c_void_p(y_dev), batch,
                                             float(lr), ctypes.byref(loss)), 'lmf_mlp_train_step')
        return loss.value


def column_dtype(arr) -> int:
    """LMF dtype of a numpy array or torch tensor."""
    s = str(arr.dtype)
    if s.endswith('int32'):
        return LMF_I32
    if s.endswith('float32'):
        return LMF_F32
    if s.endswith('float64'):
        return LMF_F64
    raise TypeError(f'unsupported column dtype {s}')


def register_schema(engine: Engine, schema, tensors: dict, on_host=False) -> None:
    """Register every relation of `schema` and its join tree.

    schema: object with .relations (each .name, .columns with .name, .role
    ('key'|'cont'|'cat'), .cat_domain), .edges ((parent, child, key)) and
    .root.  tensors[(relation, column)] is the buffer holding that column
    (device tensor, or pinned host tensor when on_host); its .data_ptr() is
    passed to the C ABI.  on_host: one LMF_DEVICE / LMF_HOST_COPY /
    LMF_HOST_MAPPED mode (a bool means device / copy) or a dict relation name
    -> mode.
    """
    for r in schema.relations:
        mode = on_host.get(r.name, LMF_DEVICE) if isinstance(on_host, dict) else int(on_host)
        cols = []
        for c in r.columns:
            t = tensors[(r.name, c.name)]
            cols.append(dict(name=c.name, dtype=column_dtype(t), role=_ROLE[c.role], data=t.data_ptr(),
                             cat_domain=int(c.cat_domain), on_host=mode))
        engine.register_relation(r.name, int(r.nrows), cols)
    ids = engine.rel_ids
    engine.declare_join([(ids[p], ids[c], k) for p, c, k in schema.edges])


# -- consumers of a batch (Sec. 2): thin wrappers over the C ABI, device pointers in and out
def ridge_bgd(sigma_ptr: int, m: int, count: float, lam: float, theta_ptr: int, iters_ptr: int,
              max_iter: int = 10_000, tol: float = 1e-13, stream: int = 0) -> None:
    """lmf_ridge_bgd: theta (m - 1 doubles) from the m x m covar matrix."""
    st = load().lmf_ridge_bgd(sigma_ptr, m, count, lam, max_iter, tol, theta_ptr, iters_ptr, stream or None)
    if st != LMF_OK:
        raise LmfError(st, 'lmf_ridge_bgd')


def mutual_information(pairs_ptr: int, n_pairs: int, alpha: int, out_ptr: int, stream: int = 0) -> None:
    """lmf_mutual_information over a device array of lmf_mi_pair."""
    st = load().lmf_mutual_information(pairs_ptr, n_pairs, alpha, out_ptr, stream or None)
    if st != LMF_OK:
        raise LmfError(st, 'lmf_mutual_information')


def chow_liu(mi_ptr: int, n: int, edges_ptr: int, n_edges_ptr: int, stream: int = 0) -> None:
    """lmf_chow_liu: the tree's edges from an n x n MI matrix."""
    st = load().lmf_chow_liu(mi_ptr, n, edges_ptr, n_edges_ptr, stream or None)
    if st != LMF_OK:
        raise LmfError(st, 'lmf_chow_liu')
