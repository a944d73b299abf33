"""FP64 reference of the applications that consume an aggregate batch (Sec. 2):
ridge linear regression trained by batch gradient descent over the covar
matrix, the mutual information of two categorical attributes from the four
count queries of Eq. mi, the Chow-Liu tree over those values, and the split
choice of a classification tree (CART) from the class counts of Eq.
classification-tree.

TEST INFRASTRUCTURE ONLY (imported by tests; the engine never imports it).

Readings where the paper leaves a choice:
* Ridge regression (Sec. 2, objective J and its BGD update): the features
  X_1..X_n include the constant 1 as X_1 (the intercept), the label is X_{n+1}
  with its parameter fixed at -1, and the penalty covers theta_1..theta_n.  The
  step size follows the paper's experimental setup (Sec. 4): a Barzilai-Borwein
  step, shortened by Armijo backtracking until the objective decreases enough.
* Mutual information (Sec. 2, Eq. mi and the aggregate function f): natural
  logarithm; cells with delta = 0 contribute 0 (the limit of d log d).
* Chow-Liu (Sec. 2): the edges chosen round by round are those of a maximum
  spanning tree of the complete graph weighted by mutual information (an edge
  that would close a cycle is skipped); ties go to the pair (i, j), i < j,
  that comes first in row-major order.
* Classification trees (Sec. 2, decision trees): the cost of a split of the
  fragment D_i into the rows with X_j <= t and the rest is the entropy or Gini
  index of each side weighted by the side's share of D_i (the CART cost of a
  split; the paper gives the index of one fragment); entropy with the natural
  logarithm (the chosen split does not depend on the base); a split that
  leaves a side empty is not a split; ties go to the first candidate in the
  order given (features in batch order, thresholds ascending).
"""
from __future__ import annotations

import math
from typing import Dict, List, Sequence, Tuple

import numpy as np


# ----------------------------------------------------------------------------
# ridge linear regression over the covar matrix
# ----------------------------------------------------------------------------
def ridge_objective(theta: np.ndarray, sigma: np.ndarray, count: float, lam: float) -> float:
    """J(theta) = 1/(2|D|) sum_X (sum_{j in [n+1]} theta_j X_j)^2 + lam/2 ||theta||^2,
    written with the covar matrix sigma = sum_X X X^T over (X_1..X_n, X_{n+1})
    and the label's parameter theta_{n+1} = -1."""
    t = np.append(np.asarray(theta, np.float64), -1.0)
    return float(t @ sigma @ t) / (2.0 * count) + 0.5 * lam * float(theta @ theta)


def ridge_gradient(theta: np.ndarray, sigma: np.ndarray, count: float, lam: float) -> np.ndarray:
    """grad_k J = 1/|D| sum_{j in [n+1]} theta_j sigma[j, k] + lam theta_k, k in [n]."""
    t = np.append(np.asarray(theta, np.float64), -1.0)
    n = len(theta)
    return (sigma[:n, :] @ t) / count + lam * np.asarray(theta, np.float64)


def ridge_bgd(sigma: np.ndarray, count: float, lam: float, max_iter: int = 10_000,
              tol: float = 1e-13) -> Tuple[np.ndarray, int]:
    """Batch gradient descent over the covar matrix (the matrix does not depend
    on theta, so every iteration reads only it).  Returns (theta, iterations).

    sigma: (n+1) x (n+1) covar matrix, the last row/column the label.
    Each iteration: gradient g; trial step s (the Barzilai-Borwein step
    <d theta, d theta> / <d theta, d g> after the first iteration, 1 before);
    halve s until J(theta - s g) <= J(theta) - s/2 ||g||^2 (Armijo); update.
    Stops when ||g|| <= tol * max(1, ||g_0||).

    J is quadratic in theta, so the change J(theta - s g) - J(theta) equals
    -s ||g||^2 + s^2/2 g^T H g with H = sigma[:n, :n]/|D| + lam I; the Armijo
    test evaluates it in that form, because the difference of two nearly
    equal objective values loses its digits close to the optimum."""
    sigma = np.asarray(sigma, np.float64)
    n = sigma.shape[0] - 1
    H = sigma[:n, :n] / count + lam * np.eye(n)
    theta = np.zeros(n)
    g = ridge_gradient(theta, sigma, count, lam)
    g0 = float(np.linalg.norm(g))
    s = 1.0
    prev_theta, prev_g = None, None
    for it in range(1, max_iter + 1):
        if float(np.linalg.norm(g)) <= tol * max(1.0, g0):
            return theta, it - 1
        if prev_theta is not None:
            dt, dg = theta - prev_theta, g - prev_g
            den = float(dt @ dg)
            if den > 0:
                s = float(dt @ dt) / den
        gg = float(g @ g)
        gHg = float(g @ H @ g)
        while -s * gg + 0.5 * s * s * gHg > -0.5 * s * gg:
            s *= 0.5
        prev_theta, prev_g = theta, g
        theta = theta - s * g
        g = ridge_gradient(theta, sigma, count, lam)
    return theta, max_iter


def covar_matrix(values: Dict[Tuple[str, ...], float], features: Sequence[str], label: str,
                 count: float) -> np.ndarray:
    """Assemble the (n+1) x (n+1) covar matrix over (1, features..., label) from
    aggregate values keyed by the sorted tuple of attribute names of each
    monomial (() for COUNT, (a,) for SUM(a), (a, a) for SUM(a^2), (a, b) for
    SUM(a*b))."""
    names = ['1'] + list(features) + [label]
    m = len(names)
    S = np.empty((m, m))
    for i in range(m):
        for j in range(m):
            k = tuple(sorted(x for x in (names[i], names[j]) if x != '1'))
            S[i, j] = values[k] if k else count
    return S


# ----------------------------------------------------------------------------
# mutual information and the Chow-Liu tree
# ----------------------------------------------------------------------------
def mutual_information(alpha: float, beta: np.ndarray, gamma: np.ndarray,
                       delta: np.ndarray) -> float:
    """MI = sum over (a, b) of f(alpha, beta_a, gamma_b, delta_ab) with
    f = delta/alpha * log(alpha delta / (beta gamma)) (Sec. 2, Eq. mi):
    alpha = COUNT, beta = COUNT by X_i, gamma = COUNT by X_j, delta = COUNT by
    (X_i, X_j) as a beta.size x gamma.size table."""
    delta = np.asarray(delta, np.float64).reshape(len(beta), len(gamma))
    terms = []
    for a in range(len(beta)):
        for b in range(len(gamma)):
            d = delta[a, b]
            if d == 0:
                continue
            terms.append(d / alpha * math.log(alpha * d / (float(beta[a]) * float(gamma[b]))))
    return math.fsum(terms)


def chow_liu_tree(n: int, mi: Dict[Tuple[int, int], float]) -> List[Tuple[int, int]]:
    """Edges (i, j), i < j, of the Chow-Liu tree over attributes 0..n-1: pairs
    taken in decreasing mutual information, skipping those that would close a
    cycle (a maximum spanning tree, Kruskal's order)."""
    parent = list(range(n))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    order = sorted(((i, j) for i in range(n) for j in range(i + 1, n)),
                   key=lambda e: (-mi[e], e))
    edges = []
    for i, j in order:
        ri, rj = find(i), find(j)
        if ri == rj:
            continue
        parent[ri] = rj
        edges.append((i, j))
        if len(edges) == n - 1:
            break
    return edges


# ----------------------------------------------------------------------------
# classification trees
# ----------------------------------------------------------------------------
def impurity(counts: Sequence[float], criterion: str = 'gini') -> float:
    """Entropy -sum_k pi_k log pi_k or Gini index 1 - sum_k pi_k^2 of a fragment
    with the given class counts, pi_k = count_k / |D_i| (Sec. 2); 0 for an
    empty fragment."""
    c = np.asarray(counts, np.float64)
    n = float(c.sum())
    if n <= 0:
        return 0.0
    pi = c / n
    if criterion == 'gini':
        return 1.0 - math.fsum(float(p) * float(p) for p in pi)
    if criterion == 'entropy':
        return -math.fsum(float(p) * math.log(float(p)) for p in pi if p > 0)
    raise ValueError(criterion)


def split_cost(left: Sequence[float], total: Sequence[float], criterion: str = 'gini') -> float:
    """Cost of splitting a fragment with class counts `total` into `left` (the
    rows with X_j <= t) and total - left: each side's impurity weighted by its
    share of the fragment."""
    lft = np.asarray(left, np.float64)
    tot = np.asarray(total, np.float64)
    rgt = tot - lft
    n = float(tot.sum())
    return (float(lft.sum()) / n) * impurity(lft, criterion) + (float(rgt.sum()) / n) * impurity(rgt, criterion)


def best_split(total: Sequence[float], left: Sequence[Tuple[object, Sequence[float]]],
               criterion: str = 'gini'):
    """The candidate of least cost among `left`, a sequence of (condition,
    class counts of the rows that satisfy it) in candidate order; returns
    (condition, cost), or None when no candidate leaves both sides non-empty."""
    n = float(np.asarray(total, np.float64).sum())
    best = None
    for cond, counts in left:
        nl = float(np.asarray(counts, np.float64).sum())
        if nl <= 0 or nl >= n:
            continue
        cost = split_cost(counts, total, criterion)
        if best is None or cost < best[1]:
            best = (cond, cost)
    return best


def classification_level_splits(batch, values, nodes, features, thresholds, n_classes: int,
                                criterion: str = 'gini'):
    """The CART step for one tree level from the results of a classification
    level batch (the layout of workloads.config3_classification): per node, the
    class counts of the node, of every candidate f <= t, and the best split.
    Returns, per node, (node class counts, best (f, t) or None, its cost)."""
    out = []
    a = 0
    for node in nodes:
        total = np.asarray(values[a], np.int64).reshape(n_classes)
        assert int(values[a + 1][0]) == int(total.sum()) and batch[a].factors == tuple(node)
        a += 2
        cands = []
        for f in features:
            for t in thresholds[f]:
                assert batch[a].factors == tuple(node) + ((f, 'le', float(t)),)
                counts = np.asarray(values[a], np.int64).reshape(n_classes)
                assert int(values[a + 1][0]) == int(counts.sum())
                cands.append(((f, float(t)), counts))
                a += 2
        b = best_split(total, cands, criterion)
        out.append((total, None if b is None else b[0], None if b is None else b[1]))
    assert a == len(batch)
    return out


def cart_children(node, split) -> List[tuple]:
    """The two children of a node split on (f, t): the node's conditions with
    f <= t, and with f > t."""
    f, t = split
    return [tuple(node) + ((f, 'le', float(t)),), tuple(node) + ((f, 'gt', float(t)),)]
