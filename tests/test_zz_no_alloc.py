"""lmf_gram_noalloc: the Gram of one relation from a kernel whose scratch is a
fixed array inside the library, for callers that cannot allocate device
memory (a pool or custom allocator that forbids outside allocations, code that
must avoid an allocation's implicit synchronisation).  Its result must match
the regular entry point's (register, plan, run) within the tests' error rule,
on two calls in a row; oversized inputs are refused."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _columns(n=300_007, k=7, seed=42):
    rng = np.random.default_rng(seed)
    cols = [rng.standard_normal(n).astype(np.float32) for _ in range(k)]
    if k > 1:
        cols[1] = (np.abs(cols[1]) * 40 + 3).astype(np.float32)   # a positive, large column
    return cols


def _regular_gram(cols):
    """The same Gram through the regular entry points (plain precision)."""
    from workloads import Column, Relation, Schema, covar_batch
    from lmf_testlib import run_engine
    names = [f'c{i}' for i in range(len(cols))]
    sch = Schema([Relation('R', [Column(nm, 'cont', c) for nm, c in zip(names, cols)])], [], 'R')
    batch = covar_batch(names)
    got, info, eng = run_engine(sch, batch, precision=0, batching=0)
    eng.close()
    m = len(cols) + 1
    G = np.zeros((m, m))
    k = 1
    G[0, 0] = got[0][0]
    for i in range(len(cols)):
        G[0, i + 1] = G[i + 1, 0] = got[k][0]
        k += 1
    for i in range(len(cols)):
        for j in range(i, len(cols)):
            G[i + 1, j + 1] = G[j + 1, i + 1] = got[k][0]
            k += 1
    return G


def _noalloc(lib, dev_cols, n, out, stream=0):
    arr = (ctypes.c_void_p * len(dev_cols))(*[c.data_ptr() for c in dev_cols])
    return lib.lmf_gram_noalloc(arr, len(dev_cols), n, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))


def test_noalloc_matches_regular_entry_point_twice():
    import torch
    from paper_1906_08687_gb300 import lmf
    lib = lmf.load()
    cols = _columns()
    n, m = len(cols[0]), len(cols) + 1
    want = _regular_gram(cols)
    dev = [torch.from_numpy(c).cuda() for c in cols]
    A = np.abs(np.stack([np.ones(n)] + [c.astype(np.float64) for c in cols]))
    scale = A @ A.T                                   # sum of |z_i z_j| per entry (m x m)
    for call in range(2):
        out = torch.full((m, m), float('nan'), dtype=torch.float64, device='cuda')
        assert _noalloc(lib, dev, n, out) == lmf.LMF_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        err = np.abs(got - want)
        allow = 1e-6 * np.maximum(np.abs(want), 1e-3 * scale)
        assert np.all(err <= allow), (call, float(np.max(err / allow)))
        assert got[0, 0] == n


@pytest.mark.parametrize('n,k', [(0, 3), (100, 1), (257, 31), (300_007, 0)])
def test_noalloc_edge_shapes(n, k):
    """No rows, one column, the full 31-column block with a ragged tile, no
    columns; on a stream of its own.  Against NumPy's FP64 Gram of the same
    FP32 columns (plus the small-input arithmetic floor 2^-21 * sum|v|), and
    G[0][0] exactly the row count."""
    import torch
    from paper_1906_08687_gb300 import lmf
    lib = lmf.load()
    cols = _columns(n, k, seed=7 + n + k) if k else []
    m = k + 1
    Z = np.stack([np.ones(n)] + [c.astype(np.float64) for c in cols]) if n else np.zeros((m, 0))
    want = Z @ Z.T
    scale = np.abs(Z) @ np.abs(Z).T
    dev = [torch.from_numpy(c).cuda() for c in cols]
    stream = torch.cuda.Stream()
    out = torch.full((m, m), float('nan'), dtype=torch.float64, device='cuda')
    arr = (ctypes.c_void_p * k)(*[c.data_ptr() for c in dev]) if k else None
    with torch.cuda.stream(stream):
        assert lib.lmf_gram_noalloc(arr, k, n, ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(stream.cuda_stream)) == lmf.LMF_OK
    stream.synchronize()
    got = out.cpu().numpy()
    allow = np.maximum(1e-6 * np.maximum(np.abs(want), 1e-3 * scale), 2.0 ** -21 * scale)
    assert np.all(np.abs(got - want) <= allow), float(np.max(np.abs(got - want) - allow))
    assert got[0, 0] == n


def test_noalloc_refuses_oversized_and_null():
    import torch
    from paper_1906_08687_gb300 import lmf
    lib = lmf.load()
    cols = [torch.zeros(10, dtype=torch.float32, device='cuda') for _ in range(32)]
    out = torch.zeros((33, 33), dtype=torch.float64, device='cuda')
    assert _noalloc(lib, cols, 10, out) == lmf.LMF_ERR_ARG           # 32 > 31 columns
    arr = (ctypes.c_void_p * 1)(None)
    assert lib.lmf_gram_noalloc(arr, 1, 10, ctypes.c_void_p(out.data_ptr()), None) == lmf.LMF_ERR_ARG
