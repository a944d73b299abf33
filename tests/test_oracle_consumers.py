"""Pins for the FP64 reference of the batch's consumers (oracle/consumers.py):
ridge regression by BGD against the closed-form solution computed from the
materialised data, the objective and gradient against their per-row
definitions, mutual information against a hand-worked table, closed forms
and an independent library implementation, the Chow-Liu tree against a
library maximum spanning tree and against recovery of a known tree."""
import math

import numpy as np
import pytest

from oracle import consumers, oracle
from workloads import Agg, config1, config4, pair_count_batch


# ----------------------------------------------------------------------------
def _data(seed, n=500, d=4):
    rng = np.random.default_rng(seed)
    X = np.hstack([np.ones((n, 1)), rng.standard_normal((n, d)) * [1, 3, 0.5, 2][:d] + 1])
    y = X @ rng.standard_normal(d + 1) + 0.3 * rng.standard_normal(n)
    Z = np.hstack([X, y[:, None]])
    return X, y, Z.T @ Z


@pytest.mark.parametrize('lam', [0.0, 0.1])
def test_objective_and_gradient_match_per_row_definitions(lam):
    X, y, S = _data(1)
    n = len(y)
    theta = np.random.default_rng(2).standard_normal(X.shape[1])
    per_row = 0.5 / n * float(np.sum((X @ theta - y) ** 2)) + 0.5 * lam * float(theta @ theta)
    assert abs(consumers.ridge_objective(theta, S, n, lam) - per_row) <= 1e-12 * per_row
    eps = 1e-6
    num = np.zeros_like(theta)
    for k in range(len(theta)):
        e = np.zeros_like(theta)
        e[k] = eps
        fp = 0.5 / n * np.sum((X @ (theta + e) - y) ** 2) + 0.5 * lam * (theta + e) @ (theta + e)
        fm = 0.5 / n * np.sum((X @ (theta - e) - y) ** 2) + 0.5 * lam * (theta - e) @ (theta - e)
        num[k] = (fp - fm) / (2 * eps)
    np.testing.assert_allclose(consumers.ridge_gradient(theta, S, n, lam), num, rtol=1e-6, atol=1e-8)


@pytest.mark.parametrize('lam', [0.0, 1e-3, 0.5])
def test_bgd_reaches_the_closed_form_ridge_solution(lam):
    X, y, S = _data(3)
    n = len(y)
    want = np.linalg.solve(X.T @ X / n + lam * np.eye(X.shape[1]), X.T @ y / n)
    if lam == 0.0:
        np.testing.assert_allclose(want, np.linalg.lstsq(X, y, rcond=None)[0], rtol=1e-10)
    theta, iters = consumers.ridge_bgd(S, n, lam)
    assert 0 < iters < 10_000
    np.testing.assert_allclose(theta, want, rtol=1e-7, atol=1e-9)


def test_ridge_over_the_oracle_covar_of_a_join():
    """Covar batch over the star join (config 1) -> BGD equals ridge regression
    solved on the materialised join."""
    sch, batch = config1(3000)
    res = oracle.evaluate(sch, batch)
    values = {}
    for a, agg in enumerate(batch):
        names = tuple(sorted([f[0] for f in agg.factors for _ in range(int(f[2]))]))
        values[names] = float(res.values[a][0])
    feats = [f for f in sch.meta['features'] if f != 'r0']
    count = float(res.values[0][0])
    S = consumers.covar_matrix(values, feats, 'r0', count)
    R, Sd, T = sch.rel('R'), sch.rel('S'), sch.rel('T')
    k1, k2 = R.col('k1').data, R.col('k2').data
    cols = []
    for f in feats:
        if f.startswith('r'):
            cols.append(R.col(f).data)
        elif f.startswith('s'):
            cols.append(Sd.col(f).data[k1])
        else:
            cols.append(T.col(f).data[k2])
    X = np.column_stack([np.ones(len(k1))] + cols)
    y = R.col('r0').data
    lam = 0.01
    want = np.linalg.solve(X.T @ X / len(y) + lam * np.eye(X.shape[1]), X.T @ y / len(y))
    theta, _ = consumers.ridge_bgd(S, count, lam)
    np.testing.assert_allclose(theta, want, rtol=1e-6, atol=1e-9)


# ----------------------------------------------------------------------------
def test_mi_hand_worked_table():
    """counts [[3, 1], [1, 3]]: alpha 8, beta = gamma = (4, 4):
    2 * 3/8 log(8*3/16) + 2 * 1/8 log(8*1/16)."""
    mi = consumers.mutual_information(8, np.array([4, 4]), np.array([4, 4]), np.array([[3, 1], [1, 3]]))
    assert abs(mi - (0.75 * math.log(1.5) + 0.25 * math.log(0.5))) < 1e-15


def test_mi_closed_forms():
    u, v = np.array([2, 6, 1]), np.array([3, 1, 4, 2])
    alpha = u.sum() * v.sum()
    delta = np.outer(u, v)                               # independent: MI = 0
    assert consumers.mutual_information(alpha, u * v.sum(), v * u.sum(), delta) == 0.0
    c = np.array([5, 1, 7, 3])                           # X_j = X_i: MI = entropy of X_i
    p = c / c.sum()
    H = -float(np.sum(p * np.log(p)))
    mi = consumers.mutual_information(c.sum(), c, c, np.diag(c))
    assert abs(mi - H) < 1e-14


def test_mi_symmetric_and_nonnegative():
    rng = np.random.default_rng(4)
    for _ in range(20):
        d = rng.integers(0, 6, size=(rng.integers(1, 5), rng.integers(1, 5)))
        d[0, 0] += 1
        a, b, g = d.sum(), d.sum(axis=1), d.sum(axis=0)
        keep_b, keep_g = b > 0, g > 0
        d = d[keep_b][:, keep_g]
        m1 = consumers.mutual_information(a, b[keep_b], g[keep_g], d)
        m2 = consumers.mutual_information(a, g[keep_g], b[keep_b], d.T)
        assert m1 >= -1e-15 and abs(m1 - m2) < 1e-14


def test_mi_from_oracle_counts_matches_library_on_the_join():
    """MI of two categories from the oracle's four count queries (Eq. mi) over
    the Chow-Liu star join equals an independent library's MI of the two
    columns of the materialised join."""
    metrics = pytest.importorskip('sklearn.metrics')
    sch, _ = config4(4000)
    cats = sch.meta['cats']
    a_name, b_name = cats[0], cats[9]          # one in D1, one in D2
    batch = [Agg(), Agg(group_by=(a_name,)), Agg(group_by=(b_name,)), Agg(group_by=(a_name, b_name))]
    r = oracle.evaluate(sch, batch)
    beta, gamma = r.values[1], r.values[2]
    delta = r.values[3].reshape(r.shapes[3])
    kb, kg = beta > 0, gamma > 0
    mi = consumers.mutual_information(float(r.values[0][0]), beta[kb], gamma[kg], delta[kb][:, kg])
    F = sch.rel('F')
    xa = sch.rel('D1').col(a_name).data[F.col('k1').data]
    xb = sch.rel('D2').col(b_name).data[F.col('k2').data]
    assert abs(mi - metrics.mutual_info_score(xa, xb)) < 1e-12


# ----------------------------------------------------------------------------
def test_chow_liu_is_a_maximum_spanning_tree():
    nx = pytest.importorskip('networkx')
    rng = np.random.default_rng(5)
    for n in (2, 3, 6, 12):
        mi = {(i, j): float(rng.random()) for i in range(n) for j in range(i + 1, n)}
        edges = consumers.chow_liu_tree(n, mi)
        assert len(edges) == n - 1
        G = nx.Graph()
        G.add_weighted_edges_from((i, j, w) for (i, j), w in mi.items())
        T = nx.maximum_spanning_tree(G)
        assert sorted(tuple(sorted(e)) for e in T.edges()) == sorted(edges)
        assert nx.is_tree(nx.Graph(edges))


def test_chow_liu_recovers_a_generating_tree():
    """Samples of a tree-structured distribution (each variable a noisy copy of
    its parent): the tree over empirical MI is the generating tree."""
    rng = np.random.default_rng(6)
    parent = [-1, 0, 0, 1, 1, 2, 5]
    n, N, dom = len(parent), 50_000, 4
    X = np.zeros((N, n), np.int64)
    X[:, 0] = rng.integers(0, dom, N)
    for v in range(1, n):
        keep = rng.random(N) < 0.7
        X[:, v] = np.where(keep, X[:, parent[v]], rng.integers(0, dom, N))
    mi = {}
    for i in range(n):
        for j in range(i + 1, n):
            d = np.zeros((dom, dom))
            np.add.at(d, (X[:, i], X[:, j]), 1)
            mi[(i, j)] = consumers.mutual_information(N, d.sum(1), d.sum(0), d)
    want = sorted((min(v, parent[v]), max(v, parent[v])) for v in range(1, n))
    assert sorted(consumers.chow_liu_tree(n, mi)) == want


def test_pair_count_batch_feeds_every_mi_pair():
    """Sec. 2: MI over all pairs of the 30 categories needs the pair counts,
    the marginals and COUNT, all in the Chow-Liu batch of config 4."""
    sch, batch = config4(10)
    cats = sch.meta['cats']
    have = {a.group_by for a in batch}
    assert all((a, b) in have for a, b in [p.group_by for p in pair_count_batch(cats)])
    assert all((c,) in have for c in cats) and () in have


# ----------------------------------------------------------------------------
MUTANTS = [
    ('MI log argument inverted',
     'math.log(alpha * d / (float(beta[a]) * float(gamma[b])))',
     'math.log((float(beta[a]) * float(gamma[b])) / (alpha * d))'),
    ('MI weight delta instead of delta/alpha', 'terms.append(d / alpha * math.log(', 'terms.append(d * math.log('),
    ('penalty dropped from the gradient', 'return (sigma[:n, :] @ t) / count + lam * np.asarray(theta, np.float64)',
     'return (sigma[:n, :] @ t) / count'),
    ('gradient not divided by |D|', 'return (sigma[:n, :] @ t) / count + lam',
     'return (sigma[:n, :] @ t) + lam'),
    ('label parameter +1', "t = np.append(np.asarray(theta, np.float64), -1.0)\n    n = len(theta)",
     "t = np.append(np.asarray(theta, np.float64), 1.0)\n    n = len(theta)"),
    ('Chow-Liu takes the smallest MI first', 'key=lambda e: (-mi[e], e))', 'key=lambda e: (mi[e], e))'),
    ('Chow-Liu keeps cycle-closing edges', '        if ri == rj:\n            continue\n', ''),
    ('covar entry of the constant read as a sum', 'S[i, j] = values[k] if k else count',
     'S[i, j] = values[k] if k else 1.0'),
]


@pytest.mark.parametrize('what,old,new', MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(what, old, new):
    import types
    with open(consumers.__file__) as f:
        text = f.read()
    assert text.count(old) == 1, what
    mod = types.ModuleType('consumers_copy')
    exec(compile(text.replace(old, new), consumers.__file__, 'exec'), mod.__dict__)
    saved = {k: getattr(consumers, k) for k in ('ridge_objective', 'ridge_gradient', 'ridge_bgd',
                                                'covar_matrix', 'mutual_information', 'chow_liu_tree')}
    failed = False
    try:
        for k in saved:
            setattr(consumers, k, getattr(mod, k))
        for test in (lambda: test_objective_and_gradient_match_per_row_definitions(0.1),
                     lambda: test_bgd_reaches_the_closed_form_ridge_solution(0.1),
                     test_ridge_over_the_oracle_covar_of_a_join, test_mi_hand_worked_table,
                     test_mi_closed_forms, test_chow_liu_is_a_maximum_spanning_tree,
                     test_chow_liu_recovers_a_generating_tree):
            try:
                test()
            except (AssertionError, np.linalg.LinAlgError):
                failed = True
                break
    finally:
        for k, v in saved.items():
            setattr(consumers, k, v)
    assert failed, what


def test_chow_liu_over_the_oracle_batch_of_config4():
    """The whole Chow-Liu application of Sec. 2 on a small config-4 instance:
    MI of all 435 category pairs from the oracle's count batch, then the tree;
    the same tree as from a library MI of the materialised join's columns and
    a library maximum spanning tree."""
    metrics = pytest.importorskip('sklearn.metrics')
    nx = pytest.importorskip('networkx')
    sch, batch = config4(5000)
    cats = sch.meta['cats']
    res = oracle.evaluate(sch, batch)
    by_gb = {agg.group_by: (res.values[i], res.shapes[i]) for i, agg in enumerate(batch)}
    alpha = float(sch.rel('F').nrows)
    mi = {}
    for i in range(len(cats)):
        for j in range(i + 1, len(cats)):
            beta, gamma = by_gb[(cats[i],)][0], by_gb[(cats[j],)][0]
            vals, shape = by_gb[(cats[i], cats[j])]
            delta = vals.reshape(shape)
            kb, kg = beta > 0, gamma > 0
            mi[(i, j)] = consumers.mutual_information(alpha, beta[kb], gamma[kg], delta[kb][:, kg])
    tree = consumers.chow_liu_tree(len(cats), mi)
    F = sch.rel('F')
    cols = []
    for c in cats:
        d = next(r for r in sch.relations if c in r.names())
        key = d.columns[0].name
        cols.append(d.col(c).data[F.col(key).data])
    G = nx.Graph()
    for (i, j) in mi:
        w = metrics.mutual_info_score(cols[i], cols[j])
        assert abs(w - mi[(i, j)]) < 1e-12
        G.add_edge(i, j, weight=w)
    want = sorted(tuple(sorted(e)) for e in nx.maximum_spanning_tree(G).edges())
    assert sorted(tree) == want
