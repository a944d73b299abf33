"""The consumers of a batch on the GPU (lmf_ridge_bgd, lmf_mutual_information,
lmf_chow_liu) against their FP64 oracle (oracle/consumers.py): ridge BGD over
the covar matrix of the star join, MI of every categorical pair and the
Chow-Liu tree of the Chow-Liu/cube batch, from the engine's own results."""
import ctypes

import numpy as np
import pytest

from oracle import consumers, oracle
from workloads import config1, config4

from lmf_testlib import run_engine

pytestmark = pytest.mark.gpu


def _covar_values(batch, values):
    out = {}
    for a, agg in enumerate(batch):
        names = tuple(sorted([f[0] for f in agg.factors for _ in range(int(f[2]))]))
        out[names] = float(np.asarray(values[a]).reshape(-1)[0])
    return out


def _gpu_ridge(S, count, lam, max_iter=10_000, tol=1e-13):
    import torch
    from paper_1906_08687_gb300 import lmf
    lib = lmf.load()
    m = S.shape[0]
    sig = torch.from_numpy(np.ascontiguousarray(S, np.float64)).cuda()
    theta = torch.full((m - 1,), float('nan'), dtype=torch.float64, device='cuda')
    iters = torch.full((1,), -1, dtype=torch.int32, device='cuda')
    st = lib.lmf_ridge_bgd(ctypes.c_void_p(sig.data_ptr()), m, count, lam, max_iter, tol,
                           ctypes.c_void_p(theta.data_ptr()), ctypes.c_void_p(iters.data_ptr()), None)
    assert st == lmf.LMF_OK
    torch.cuda.synchronize()
    return theta.cpu().numpy(), int(iters.cpu()[0])


@pytest.mark.parametrize('lam', [0.0, 0.01, 1.0])
def test_ridge_bgd_same_covar_matches_oracle(lam):
    """The same covar matrix (the oracle's, of a 200k-row star join) through the
    device BGD and the FP64 reference BGD: the same iterates up to rounding."""
    sch, batch = config1(200_000)
    res = oracle.evaluate(sch, batch)
    feats = [f for f in sch.meta['features'] if f != 'r0']
    count = float(res.values[0][0])
    S = consumers.covar_matrix(_covar_values(batch, res.values), feats, 'r0', count)
    want, it_ref = consumers.ridge_bgd(S, count, lam)
    got, it = _gpu_ridge(S, count, lam)
    assert 0 < it < 10_000 and 0 < it_ref < 10_000      # both converged (their paths differ by rounding)
    np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-11)
    # the device's answer is a stationary point of J
    g = consumers.ridge_gradient(got, S, count, lam)
    g0 = consumers.ridge_gradient(np.zeros_like(got), S, count, lam)
    assert np.linalg.norm(g) <= 1e-10 * max(1.0, np.linalg.norm(g0))


def test_ridge_bgd_from_engine_covar():
    """The covar batch evaluated by the engine on the GPU, then BGD on the GPU,
    against BGD over the oracle's covar: the model agrees to the accuracy the
    covar carries (1e-6 relative entries, a well-conditioned star join)."""
    sch, batch = config1(200_000)
    got_vals, info, eng = run_engine(sch, batch, precision=0, batching=1)
    eng.close()
    res = oracle.evaluate(sch, batch)
    feats = [f for f in sch.meta['features'] if f != 'r0']
    S_gpu = consumers.covar_matrix(_covar_values(batch, got_vals), feats, 'r0', float(got_vals[0][0]))
    S_ref = consumers.covar_matrix(_covar_values(batch, res.values), feats, 'r0', float(res.values[0][0]))
    lam = 0.01
    theta, _ = _gpu_ridge(S_gpu, float(got_vals[0][0]), lam)
    want, _ = consumers.ridge_bgd(S_ref, float(res.values[0][0]), lam)
    np.testing.assert_allclose(theta, want, rtol=1e-5, atol=1e-7)


def test_ridge_bgd_refuses_bad_arguments():
    import torch
    from paper_1906_08687_gb300 import lmf
    lib = lmf.load()
    sig = torch.zeros((97, 97), dtype=torch.float64, device='cuda')
    th = torch.zeros(96, dtype=torch.float64, device='cuda')
    it = torch.zeros(1, dtype=torch.int32, device='cuda')
    p = [ctypes.c_void_p(t.data_ptr()) for t in (sig, th, it)]
    assert lib.lmf_ridge_bgd(p[0], 97, 1.0, 0.0, 10, 1e-12, p[1], p[2], None) == lmf.LMF_ERR_ARG   # m > 96
    assert lib.lmf_ridge_bgd(p[0], 5, 0.0, 0.0, 10, 1e-12, p[1], p[2], None) == lmf.LMF_ERR_ARG   # count 0
    assert lib.lmf_ridge_bgd(None, 5, 1.0, 0.0, 10, 1e-12, p[1], p[2], None) == lmf.LMF_ERR_ARG


def _mi_inputs(batch, values, cats):
    """alpha, marginals per attribute, joint tables per pair (i < j) from a
    Chow-Liu batch's results, keyed like the batch."""
    marg, joint = {}, {}
    for a, agg in enumerate(batch):
        if len(agg.group_by) == 1:
            marg[agg.group_by[0]] = np.asarray(values[a], np.int64)
        elif len(agg.group_by) == 2 and not agg.factors:
            joint[agg.group_by] = np.asarray(values[a], np.int64)
    alpha = int(marg[cats[0]].sum())
    return alpha, marg, joint


@pytest.mark.parametrize('order', ['sorted', 'random'])
def test_mutual_information_and_chow_liu(order):
    """All 435 pair MIs of the Chow-Liu batch and the tree over the 30
    attributes, from the engine's counts on the GPU, against the FP64 oracle on
    the oracle's counts (the counts are bit-identical, so the MIs agree to
    rounding and the trees are equal)."""
    import torch
    from paper_1906_08687_gb300 import lmf
    lib = lmf.load()
    sch, batch = config4(500_000, fact_order=order)
    cats = sch.meta['cats']
    got_vals, info, eng = run_engine(sch, batch, precision=0, batching=1)
    eng.close()
    res = oracle.evaluate(sch, batch)
    alpha_g, marg_g, joint_g = _mi_inputs(batch, got_vals, cats)
    alpha_r, marg_r, joint_r = _mi_inputs(batch, res.values, cats)
    assert alpha_g == alpha_r == 500_000
    dom = {c: len(marg_g[c]) for c in cats}
    keep = []
    pairs = []
    for (a, b), t in joint_g.items():
        bt = torch.from_numpy(marg_g[a]).cuda()
        gt = torch.from_numpy(marg_g[b]).cuda()
        dt = torch.from_numpy(t).cuda()
        keep += [bt, gt, dt]
        pairs.append(lmf.lmf_mi_pair(bt.data_ptr(), gt.data_ptr(), dt.data_ptr(), dom[a], dom[b]))
    arr = (lmf.lmf_mi_pair * len(pairs))(*pairs)
    dev_pairs = torch.empty(ctypes.sizeof(arr), dtype=torch.uint8, device='cuda')
    dev_pairs.copy_(torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8))
    mi = torch.full((len(pairs),), float('nan'), dtype=torch.float64, device='cuda')
    assert lib.lmf_mutual_information(ctypes.c_void_p(dev_pairs.data_ptr()), len(pairs), alpha_g,
                                      ctypes.c_void_p(mi.data_ptr()), None) == lmf.LMF_OK
    torch.cuda.synchronize()
    mi = mi.cpu().numpy()
    n = len(cats)
    M = np.zeros((n, n))
    want = {}
    for k, ((a, b), _) in enumerate(joint_g.items()):
        ref = consumers.mutual_information(alpha_r, marg_r[a], marg_r[b], joint_r[(a, b)])
        assert abs(mi[k] - ref) <= 1e-12 * max(1.0, abs(ref)), (a, b, mi[k], ref)
        i, j = cats.index(a), cats.index(b)
        M[min(i, j), max(i, j)] = mi[k]
        want[(min(i, j), max(i, j))] = ref
    dM = torch.from_numpy(M).cuda()
    edges = torch.full((2 * (n - 1),), -1, dtype=torch.int32, device='cuda')
    ne = torch.zeros(1, dtype=torch.int32, device='cuda')
    assert lib.lmf_chow_liu(ctypes.c_void_p(dM.data_ptr()), n, ctypes.c_void_p(edges.data_ptr()),
                            ctypes.c_void_p(ne.data_ptr()), None) == lmf.LMF_OK
    torch.cuda.synchronize()
    got_edges = [tuple(e) for e in edges.cpu().numpy().reshape(-1, 2)[:int(ne.cpu()[0])]]
    assert got_edges == consumers.chow_liu_tree(n, want)
    assert len(got_edges) == n - 1


def test_chow_liu_ties_and_small_sizes():
    """Equal weights go to the first pair in row-major order; one attribute has
    no edge; two attributes one edge."""
    import torch
    from paper_1906_08687_gb300 import lmf
    lib = lmf.load()
    for n, M in [(1, np.zeros((1, 1))), (2, np.array([[0, 0.5], [0, 0]])), (4, np.ones((4, 4)))]:
        dM = torch.from_numpy(np.ascontiguousarray(M, np.float64)).cuda()
        edges = torch.full((max(2, 2 * (n - 1)),), -1, dtype=torch.int32, device='cuda')
        ne = torch.zeros(1, dtype=torch.int32, device='cuda')
        assert lib.lmf_chow_liu(ctypes.c_void_p(dM.data_ptr()), n, ctypes.c_void_p(edges.data_ptr()),
                                ctypes.c_void_p(ne.data_ptr()), None) == lmf.LMF_OK
        torch.cuda.synchronize()
        got = [tuple(e) for e in edges.cpu().numpy().reshape(-1, 2)[:int(ne.cpu()[0])]]
        want = consumers.chow_liu_tree(n, {(i, j): float(M[i, j]) for i in range(n) for j in range(i + 1, n)})
        assert got == want
