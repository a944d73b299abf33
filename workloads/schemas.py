"""Seeded synthetic schemas and aggregate batches.

Everything here is *input*: relations as columnar numpy arrays, a join tree
(parent, child, key) and a batch of aggregates written in the query form of
Sec. 2 (Eq. query): group-by attributes and a product of factors, each factor a
power of an attribute or a threshold indicator (Sec. 1.1).  The shapes follow
the paper's workloads (star / snowflake schemas with a large fact table and
small dimensions, Sec. 4 and App. A); the paper's datasets are not available,
so seeded stand-ins of the same structure are generated.

Random streams come from numpy's Philox counter-based generator, one stream per
config, seeded with ``SEED_BASE + config index``.
"""
from __future__ import annotations

import dataclasses
import itertools
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

SEED_BASE = 1906086870


# ----------------------------------------------------------------------------
# containers
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Column:
    name: str
    role: str                  # 'key' | 'cont' | 'cat'
    data: np.ndarray           # int32 for key/cat, float32 or float64 for cont
    cat_domain: int = 0        # values of a 'cat' column lie in [0, cat_domain)


@dataclasses.dataclass
class Relation:
    name: str
    columns: List[Column]

    @property
    def nrows(self) -> int:
        return int(len(self.columns[0].data)) if self.columns else 0

    def col(self, name: str) -> Column:
        for c in self.columns:
            if c.name == name:
                return c
        raise KeyError(name)

    def names(self) -> List[str]:
        return [c.name for c in self.columns]


@dataclasses.dataclass
class Schema:
    relations: List[Relation]
    edges: List[Tuple[str, str, str]]          # (parent, child, key attribute)
    root: str
    meta: Dict = dataclasses.field(default_factory=dict)

    def rel(self, name: str) -> Relation:
        for r in self.relations:
            if r.name == name:
                return r
        raise KeyError(name)

    def owner(self, attr: str) -> Relation:
        """Relation that holds a non-key attribute (attribute names are unique)."""
        for r in self.relations:
            for c in r.columns:
                if c.name == attr and c.role != 'key':
                    return r
        raise KeyError(attr)


@dataclasses.dataclass(frozen=True)
class Agg:
    """One aggregate Q(group_by; prod(factors)).

    factors: tuples (attr, 'pow', p) with p in {1, 2}, or (attr, 'le', t) /
    (attr, 'gt', t) for the indicators 1[attr <= t] / 1[attr > t].  An empty
    product is COUNT (SUM(1)).
    """
    group_by: Tuple[str, ...] = ()
    factors: Tuple[Tuple[str, str, float], ...] = ()


# ----------------------------------------------------------------------------
# samplers
# ----------------------------------------------------------------------------
def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def sort_by_join_attributes(rel: Relation, keys: Sequence[str]) -> Relation:
    """The relation with its rows in the scan order of Sec. 3.5: sorted on its
    join attributes, the attribute with the fewest distinct values first (ties
    keep the given order).  The paper's experiments get every relation sorted
    by its join attributes (App. B).  Same rows, so every aggregate keeps its
    value; only the row order changes."""
    if rel.nrows == 0 or not keys:
        return rel
    ndist = [len(np.unique(rel.col(k).data)) for k in keys]
    order = [k for _, _, k in sorted(zip(ndist, range(len(keys)), keys))]
    perm = np.lexsort([rel.col(k).data for k in reversed(order)])
    return Relation(rel.name, [dataclasses.replace(c, data=np.ascontiguousarray(c.data[perm]))
                               for c in rel.columns])


def zipf_keys(rng: np.random.Generator, n: int, k: int, s: float) -> np.ndarray:
    """n draws over key ids 0..k-1 with P(rank i) ~ i^-s (i = 1..k); ranks are
    mapped to key ids by a seeded random permutation.  s = 0 is uniform."""
    if k <= 0:
        return np.zeros(n, dtype=np.int32)
    if s == 0.0:
        return rng.integers(0, k, size=n, dtype=np.int64).astype(np.int32)
    w = np.arange(1, k + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    perm = rng.permutation(k).astype(np.int32)
    out = np.empty(n, dtype=np.int32)
    chunk = 1 << 22
    for b in range(0, n, chunk):
        u = rng.random(min(chunk, n - b))
        r = np.searchsorted(cdf, u, side='right')
        np.minimum(r, k - 1, out=r)
        out[b:b + len(r)] = perm[r]
    return out


def _feature(rng: np.random.Generator, n: int, gidx: int, dtype) -> np.ndarray:
    """Continuous feature number gidx: even -> N(0,1); odd -> the mixture
    0.7 LogNormal(0, 0.5) + 0.3 LogNormal(1.5, 1.0)."""
    if gidx % 2 == 0:
        v = rng.standard_normal(n)
    else:
        pick = rng.random(n) < 0.7
        a = rng.lognormal(0.0, 0.5, n)
        b = rng.lognormal(1.5, 1.0, n)
        v = np.where(pick, a, b)
    return v.astype(dtype)


def _log_uniform_int(rng: np.random.Generator, lo: int, hi: int) -> int:
    return int(round(float(np.exp(rng.uniform(np.log(lo), np.log(hi))))))


# ----------------------------------------------------------------------------
# aggregate batches (Sec. 2)
# ----------------------------------------------------------------------------
def covar_batch(features: Sequence[str]) -> List[Agg]:
    """COUNT, SUM(x_i) and SUM(x_i x_j), i <= j: the covar matrix of ridge
    linear regression (Sec. 2, Eq. lr-sigma); (n+1)(n+2)/2 aggregates."""
    out = [Agg()]
    out += [Agg(factors=((f, 'pow', 1),)) for f in features]
    for i, a in enumerate(features):
        for b in features[i:]:
            if a == b:
                out.append(Agg(factors=((a, 'pow', 2),)))
            else:
                out.append(Agg(factors=((a, 'pow', 1), (b, 'pow', 1))))
    return out


def grouped_batch(cats: Sequence[str], features: Sequence[str]) -> List[Agg]:
    """Covar entries with one categorical attribute, one-hot encoded as a
    group-by (Sec. 2, Covar(X_j; X_k)): COUNT and SUM(x_i) grouped by each cat."""
    out = []
    for c in cats:
        out.append(Agg(group_by=(c,)))
        out += [Agg(group_by=(c,), factors=((f, 'pow', 1),)) for f in features]
    return out


def pair_count_batch(cats: Sequence[str]) -> List[Agg]:
    """COUNT grouped by each pair of categorical attributes (Sec. 2,
    Covar(X_j, X_k; 1) and the Q_{i,j} counts of Eq. mi)."""
    return [Agg(group_by=(a, b)) for a, b in itertools.combinations(cats, 2)]


def cube_batch(dims: Sequence[str]) -> List[Agg]:
    """A data cube with COUNT measure: one aggregate per subset of the
    dimensions (Sec. 2, Eq. data-cube), 2^d aggregates."""
    out = []
    for r in range(len(dims) + 1):
        for sub in itertools.combinations(dims, r):
            out.append(Agg(group_by=tuple(sub)))
    return out


# ----------------------------------------------------------------------------
# config 1: star schema, 66 aggregates
# ----------------------------------------------------------------------------
def _check_order(fact_order: str) -> None:
    if fact_order not in ('sorted', 'random'):
        raise ValueError(f"fact_order must be 'sorted' or 'random', not {fact_order!r}")


def config1(n_fact: int = 200_000, seed: Optional[int] = None,
            fact_order: str = 'sorted') -> Tuple[Schema, List[Agg]]:
    _check_order(fact_order)
    rng = _rng(SEED_BASE + 1 if seed is None else seed)
    ks, kt = 1000, 500
    R = Relation('R', [
        Column('k1', 'key', zipf_keys(rng, n_fact, ks, 0.0)),
        Column('k2', 'key', zipf_keys(rng, n_fact, kt, 0.0)),
    ] + [Column(f'r{i}', 'cont', rng.standard_normal(n_fact)) for i in range(3)])
    if fact_order == 'sorted':
        R = sort_by_join_attributes(R, ['k1', 'k2'])
    S = Relation('S', [Column('k1', 'key', np.arange(ks, dtype=np.int32))] +
                 [Column(f's{i}', 'cont', rng.standard_normal(ks)) for i in range(4)])
    T = Relation('T', [Column('k2', 'key', np.arange(kt, dtype=np.int32))] +
                 [Column(f't{i}', 'cont', rng.standard_normal(kt)) for i in range(3)])
    sch = Schema([R, S, T], [('R', 'S', 'k1'), ('R', 'T', 'k2')], 'R',
                 meta={'name': 'star-200k', 'features': [f'r{i}' for i in range(3)] +
                       [f's{i}' for i in range(4)] + [f't{i}' for i in range(3)]})
    return sch, covar_batch(sch.meta['features'])


# ----------------------------------------------------------------------------
# config 2 / 3: snowflake  F -> D1 -> Sub1 -> Sub2, F -> D2, F -> D3, F -> D4
# (D3 and D4 share the fact key k3, like two dimensions keyed on one date)
# ----------------------------------------------------------------------------
_SNOW = [  # relation, key, K, parent, fk-on-parent
    ('D1', 'k1', 100_000, 'F'),
    ('Sub1', 's1', 5_000, 'D1'),
    ('Sub2', 's2', 500, 'Sub1'),
    ('D2', 'k2', 10_000, 'F'),
    ('D3', 'k3', 1_000, 'F'),
    ('D4', 'k3', 1_000, 'F'),
]


def _snowflake(rng, n_fact, n_fact_feat, dim_feat, dim_cat, fk_s, cat_s, cat_lo,
               cat_hi, label=False, feat_dtype=np.float32, fact_order='sorted'):
    _check_order(fact_order)
    feats: List[str] = []
    cats: List[str] = []
    gidx = 0
    fact_cols = []
    for rel, key, K, parent in _SNOW:
        if parent == 'F' and key not in [c.name for c in fact_cols]:
            fact_cols.append(Column(key, 'key', zipf_keys(rng, n_fact, K, fk_s)))
    for i in range(n_fact_feat):
        fact_cols.append(Column(f'x{i}', 'cont', _feature(rng, n_fact, gidx, feat_dtype)))
        feats.append(f'x{i}')
        gidx += 1
    if label:
        fact_cols.append(Column('y', 'cont', _feature(rng, n_fact, 0, feat_dtype)))
    rels = {'F': Relation('F', fact_cols)}
    if fact_order == 'sorted':
        rels['F'] = sort_by_join_attributes(rels['F'], [c.name for c in fact_cols if c.role == 'key'])
    edges = []
    for rel, key, K, parent in _SNOW:
        cols = [Column(key, 'key', np.arange(K, dtype=np.int32))]
        for child_rel, ckey, cK, cparent in _SNOW:
            if cparent == rel:
                cols.append(Column(ckey, 'key', zipf_keys(rng, K, cK, fk_s)))
        low = rel.lower()
        for i in range(dim_feat[rel]):
            cols.append(Column(f'{low}_x{i}', 'cont', _feature(rng, K, gidx, feat_dtype)))
            feats.append(f'{low}_x{i}')
            gidx += 1
        for i in range(dim_cat.get(rel, 0)):
            dom = _log_uniform_int(rng, cat_lo, cat_hi)
            cols.append(Column(f'{low}_c{i}', 'cat', zipf_keys(rng, K, dom, cat_s), dom))
            cats.append(f'{low}_c{i}')
        rels[rel] = Relation(rel, cols)
        edges.append((parent, rel, key))
    order = ['F'] + [r for r, *_ in _SNOW]
    return Schema([rels[r] for r in order], edges, 'F'), feats, cats


def config2(n_fact: int = 20_000_000, seed: Optional[int] = None,
            fact_order: str = 'sorted') -> Tuple[Schema, List[Agg]]:
    rng = _rng(SEED_BASE + 2 if seed is None else seed)
    sch, feats, cats = _snowflake(
        rng, n_fact, 8,
        dim_feat={'D1': 6, 'Sub1': 4, 'Sub2': 2, 'D2': 5, 'D3': 3, 'D4': 2},
        dim_cat={'D1': 2, 'Sub1': 1, 'Sub2': 1, 'D2': 3, 'D3': 2, 'D4': 1},
        fk_s=0.8, cat_s=1.1, cat_lo=5, cat_hi=1000, fact_order=fact_order)
    sch.meta.update(name=f'snowflake-{n_fact}', features=feats, cats=cats)
    batch = covar_batch(feats) + grouped_batch(cats, feats) + pair_count_batch(cats)
    return sch, batch


# ----------------------------------------------------------------------------
# config 3: regression-tree level batch
# ----------------------------------------------------------------------------
def _joined_sample(sch: Schema, attr: str, rows: np.ndarray) -> np.ndarray:
    """Values of attribute `attr` for the given fact rows, followed through the
    (unique, dense) dimension keys.  Used only to place quantile thresholds."""
    path = []
    rel = sch.owner(attr).name
    while rel != sch.root:
        parent, key = next((p, k) for p, c, k in sch.edges if c == rel)
        path.append((parent, key))
        rel = parent
    idx = rows
    for parent, key in reversed(path):
        idx = sch.rel(parent).col(key).data[idx]
    return sch.owner(attr).col(attr).data[idx]


def _tree_level(sch: Schema, feats: Sequence[str], rng: np.random.Generator, n_fact: int,
                n_nodes_depth: int, n_thresholds: int, sample_rows: int):
    """Thresholds per feature at the empirical j/(T+1) quantiles of a sample of
    joined rows, and the leaves of a random complete tree of the given depth
    (each internal node a (feature, one of its thresholds) condition)."""
    rows = rng.integers(0, n_fact, size=min(sample_rows, n_fact))
    thr = {}
    for f in feats:
        v = _joined_sample(sch, f, rows).astype(np.float64)
        q = np.quantile(v, np.arange(1, n_thresholds + 1) / (n_thresholds + 1))
        thr[f] = np.unique(q.astype(np.float32)).astype(np.float64)
    leaves: List[Tuple[Tuple[str, str, float], ...]] = [()]
    for _ in range(n_nodes_depth):
        nxt = []
        for path in leaves:
            f = feats[int(rng.integers(0, len(feats)))]
            t = float(thr[f][int(rng.integers(0, len(thr[f])))])
            nxt.append(path + ((f, 'le', t),))
            nxt.append(path + ((f, 'gt', t),))
        leaves = nxt
    return thr, leaves


def config3(n_fact: int = 10_000_000, seed: Optional[int] = None, n_nodes_depth: int = 6,
            n_thresholds: int = 32, sample_rows: int = 1_000_000,
            fact_order: str = 'sorted') -> Tuple[Schema, List[Agg]]:
    rng = _rng(SEED_BASE + 3 if seed is None else seed)
    sch, feats, _ = _snowflake(
        rng, n_fact, 6,
        dim_feat={'D1': 4, 'Sub1': 2, 'Sub2': 1, 'D2': 3, 'D3': 2, 'D4': 2},
        dim_cat={}, fk_s=0.8, cat_s=1.1, cat_lo=5, cat_hi=1000, label=True, fact_order=fact_order)
    thr, leaves = _tree_level(sch, feats, rng, n_fact, n_nodes_depth, n_thresholds, sample_rows)
    batch = []
    for node in leaves:
        for f in feats:
            for t in thr[f]:
                for p in (0, 1, 2):
                    lab = () if p == 0 else (('y', 'pow', p),)
                    batch.append(Agg(factors=node + ((f, 'le', float(t)),) + lab))
    sch.meta.update(name=f'tree-level-{n_fact}', features=feats, thresholds=thr,
                    nodes=leaves, label='y')
    return sch, batch


def config3_classification(n_fact: int = 1_000_000, n_classes: int = 4, seed: Optional[int] = None,
                           n_nodes_depth: int = 6, n_thresholds: int = 32, sample_rows: int = 1_000_000,
                           fact_order: str = 'sorted') -> Tuple[Schema, List[Agg]]:
    """A classification-tree level (Sec. 2, decision trees): config 3's
    snowflake and tree with a categorical label `cls` on the fact relation
    instead of the continuous y.  The class is a noisy quantile bin of
    x0 + d1_x0 + 0.5 d2_x0, so splits on those features lower the impurity.

    Per leaf node nu, feature f and threshold t the two queries of Eq.
    classification-tree and its total: COUNT grouped by cls and COUNT, both
    under alpha = nu and f <= t; per node the same two under nu alone (the
    counts the other side of every split is the difference from).  Order:
    for each node, [CT(cls; nu), CT(nu)], then for each f, t:
    [CT(cls; nu, f <= t), CT(nu, f <= t)]."""
    rng = _rng(SEED_BASE + 31 if seed is None else seed)
    sch, feats, _ = _snowflake(
        rng, n_fact, 6,
        dim_feat={'D1': 4, 'Sub1': 2, 'Sub2': 1, 'D2': 3, 'D3': 2, 'D4': 2},
        dim_cat={}, fk_s=0.8, cat_s=1.1, cat_lo=5, cat_hi=1000, label=False, fact_order=fact_order)
    rows = np.arange(n_fact)
    score = (_joined_sample(sch, 'x0', rows).astype(np.float64)
             + _joined_sample(sch, 'd1_x0', rows).astype(np.float64)
             + 0.5 * _joined_sample(sch, 'd2_x0', rows).astype(np.float64))
    score = score + 0.5 * np.std(score) * rng.standard_normal(n_fact)
    edges = np.quantile(score, np.arange(1, n_classes) / n_classes)
    cls = np.searchsorted(edges, score, side='right').astype(np.int32)
    fact = sch.rel('F')
    fact.columns.append(Column('cls', 'cat', cls, n_classes))
    thr, leaves = _tree_level(sch, feats, rng, n_fact, n_nodes_depth, n_thresholds, sample_rows)
    batch = []
    for node in leaves:
        batch.append(Agg(group_by=('cls',), factors=node))
        batch.append(Agg(factors=node))
        for f in feats:
            for t in thr[f]:
                alpha = node + ((f, 'le', float(t)),)
                batch.append(Agg(group_by=('cls',), factors=alpha))
                batch.append(Agg(factors=alpha))
    sch.meta.update(name=f'classification-tree-level-{n_fact}', features=feats, thresholds=thr,
                    nodes=leaves, label='cls', n_classes=n_classes)
    return sch, batch


# ----------------------------------------------------------------------------
# config 4: Chow-Liu pair counts + data cube
# ----------------------------------------------------------------------------
def config4(n_fact: int = 50_000_000, seed: Optional[int] = None,
            fact_order: str = 'sorted') -> Tuple[Schema, List[Agg]]:
    _check_order(fact_order)
    rng = _rng(SEED_BASE + 4 if seed is None else seed)
    Ks = [200, 1000, 5000, 20000]
    ncat = [7, 7, 8, 8]
    cube_dom = {0: 50, 1: 20, 2: 10}
    fact = Relation('F', [Column(f'k{j + 1}', 'key', zipf_keys(rng, n_fact, Ks[j], 1.0))
                          for j in range(4)])
    if fact_order == 'sorted':
        fact = sort_by_join_attributes(fact, [f'k{j + 1}' for j in range(4)])
    rels = [fact]
    edges = []
    cats: List[str] = []
    cube: List[str] = []
    for j in range(4):
        name = f'D{j + 1}'
        cols = [Column(f'k{j + 1}', 'key', np.arange(Ks[j], dtype=np.int32))]
        for i in range(ncat[j]):
            dom = cube_dom[j] if (i == 0 and j in cube_dom) else _log_uniform_int(rng, 2, 1000)
            cname = f'd{j + 1}_c{i}'
            cols.append(Column(cname, 'cat', zipf_keys(rng, Ks[j], dom, 1.0), dom))
            cats.append(cname)
            if i == 0 and j in cube_dom:
                cube.append(cname)
        rels.append(Relation(name, cols))
        edges.append(('F', name, f'k{j + 1}'))
    sch = Schema(rels, edges, 'F', meta={'name': f'chowliu-{n_fact}', 'cats': cats, 'cube': cube})
    batch = pair_count_batch(cats) + [Agg(group_by=(c,)) for c in cats] + cube_batch(cube)
    return sch, batch


# ----------------------------------------------------------------------------
# config 5: random acyclic schemas for plan selection
# ----------------------------------------------------------------------------
def config5_schema(index: int, n_scale: float = 1.0, seed: Optional[int] = None,
                   fact_order: str = 'mixed') -> Tuple[Schema, List[Agg]]:
    """Schema number `index` of the plan-selection corpus: 3-8 relations on a
    random tree, fact 1M-50M rows (times n_scale), 5-40 features, key skew
    s in [0, 1.2], 10-2000 monomial / grouped aggregates.  fact_order 'mixed'
    sorts the fact table on its join attributes (Sec. 3.5 order) for even
    indices and keeps generation order for odd ones, so the corpus holds both
    input orders; 'sorted' / 'random' fix one."""
    if fact_order != 'mixed':
        _check_order(fact_order)
    rng = _rng((SEED_BASE + 5 if seed is None else seed) * 1000 + index)
    nrel = int(rng.integers(3, 9))
    n_fact = max(1000, int(float(np.exp(rng.uniform(np.log(1e6), np.log(5e7)))) * n_scale))
    skew = float(rng.uniform(0.0, 1.2))
    nfeat = int(rng.integers(5, 41))
    parents = [-1] + [int(rng.integers(0, i)) for i in range(1, nrel)]
    sizes = [n_fact] + [int(float(np.exp(rng.uniform(np.log(100), np.log(200_000)))))
                        for _ in range(1, nrel)]
    feat_owner = rng.integers(0, nrel, size=nfeat)
    rels = []
    edges = []
    feats = []
    cats = []
    for r in range(nrel):
        name = 'F' if r == 0 else f'R{r}'
        cols = []
        if r > 0:
            cols.append(Column(f'k{r}', 'key', np.arange(sizes[r], dtype=np.int32)))
            edges.append(('F' if parents[r] == 0 else f'R{parents[r]}', name, f'k{r}'))
        for c in range(1, nrel):
            if parents[c] == r:
                cols.append(Column(f'k{c}', 'key', zipf_keys(rng, sizes[r], sizes[c], skew)))
        for i in np.nonzero(feat_owner == r)[0]:
            cols.append(Column(f'f{i}', 'cont', _feature(rng, sizes[r], int(i), np.float32)))
            feats.append(f'f{i}')
        if r > 0 and rng.random() < 0.5:
            dom = _log_uniform_int(rng, 2, 200)
            cols.append(Column(f'c{r}', 'cat', zipf_keys(rng, sizes[r], dom, 1.0), dom))
            cats.append(f'c{r}')
        if not cols:
            cols.append(Column(f'f_pad{r}', 'cont', np.zeros(sizes[r], np.float32)))
            feats.append(f'f_pad{r}')
        rels.append(Relation(name, cols))
    batch = covar_batch(feats)
    n_target = int(rng.integers(10, 2001))
    if len(batch) > n_target:
        keep = np.sort(rng.choice(len(batch), size=n_target, replace=False))
        batch = [batch[i] for i in keep]
    if cats:
        batch += grouped_batch(cats, feats[: max(1, min(len(feats), (n_target // 10) + 1))])
    if fact_order == 'sorted' or (fact_order == 'mixed' and index % 2 == 0):
        fks = [f'k{c}' for c in range(1, nrel) if parents[c] == 0]
        if fks:
            rels[0] = sort_by_join_attributes(rels[0], fks)
    sch = Schema(rels, edges, 'F', meta={'name': f'random-{index}', 'features': feats,
                                          'cats': cats, 'skew': skew})
    return sch, batch


def spread_keys(sch: Schema, mult: int = 1_000_003, offset: int = 7) -> Schema:
    """The same database with every join-key value k >= 0 replaced by
    k * mult + offset (negative values kept): an injective relabelling, so
    every aggregate keeps its value, but keys far too sparse to index an array
    directly (int32 range permitting)."""
    keys = {k for _, _, k in sch.edges}
    rels = []
    for r in sch.relations:
        cols = []
        for c in r.columns:
            if c.name in keys:
                v = c.data.astype(np.int64)
                v = np.where(v >= 0, v * mult + offset, v)
                if v.size and v.max() > np.iinfo(np.int32).max:
                    raise ValueError(f'{r.name}.{c.name}: spread keys overflow int32')
                c = dataclasses.replace(c, data=v.astype(np.int32))
            cols.append(c)
        rels.append(Relation(r.name, cols))
    return Schema(rels, list(sch.edges), sch.root, meta=dict(sch.meta))


# ----------------------------------------------------------------------------
# tiny schemas for brute-force tests
# ----------------------------------------------------------------------------
def tiny_schema(seed: int, max_rel: int = 4, max_rows: int = 9, unique_keys: bool = False,
                allow_empty: bool = True, feat_dtype=np.float64) -> Tuple[Schema, List[Agg]]:
    """A random tree of 1..max_rel relations with few rows.  Unless
    unique_keys, child keys repeat and some foreign keys dangle (values with no
    matching row), so joins fan out and drop rows.  Features are small integers
    plus a random fraction so products are exact-ish but not trivial."""
    rng = _rng(seed)
    nrel = int(rng.integers(1, max_rel + 1))
    parents = [-1] + [int(rng.integers(0, i)) for i in range(1, nrel)]
    rows = []
    for r in range(nrel):
        lo = 0 if (allow_empty and r > 0) else 1
        rows.append(int(rng.integers(lo, max_rows + 1)))
    dom = [int(rng.integers(2, 5)) for _ in range(nrel)]     # key domains
    rels, edges, feats, cats = [], [], [], []
    for r in range(nrel):
        name = f'T{r}'
        cols = []
        if r > 0:
            if unique_keys:
                n = min(rows[r], dom[r])
                keys = rng.permutation(dom[r])[:n].astype(np.int32)
                rows[r] = n
            else:
                keys = rng.integers(0, dom[r], size=rows[r]).astype(np.int32)
            cols.append(Column(f'k{r}', 'key', keys))
            edges.append((f'T{parents[r]}', name, f'k{r}'))
        for c in range(1, nrel):
            if parents[c] == r:
                # one past the child's domain: some foreign keys dangle
                cols.append(Column(f'k{c}', 'key',
                                   rng.integers(0, dom[c] + 1, size=rows[r]).astype(np.int32)))
        for i in range(int(rng.integers(1, 3))):
            v = rng.integers(-3, 4, size=rows[r]) + rng.random(rows[r]).round(3)
            cols.append(Column(f'{name.lower()}_x{i}', 'cont', v.astype(feat_dtype)))
            feats.append(f'{name.lower()}_x{i}')
        if rng.random() < 0.7:
            d = int(rng.integers(2, 4))
            cols.append(Column(f'{name.lower()}_c', 'cat',
                               rng.integers(0, d, size=rows[r]).astype(np.int32), d))
            cats.append(f'{name.lower()}_c')
        rels.append(Relation(name, cols))
    sch = Schema(rels, edges, 'T0', meta={'name': f'tiny-{seed}', 'features': feats,
                                          'cats': cats})
    batch = covar_batch(feats) + grouped_batch(cats, feats) + pair_count_batch(cats)
    if feats:
        f0 = feats[0]
        col = sch.owner(f0).col(f0).data
        t = float(np.median(col)) if len(col) else 0.0
        batch.append(Agg(factors=((f0, 'le', t),)))
        batch.append(Agg(factors=((f0, 'gt', t), (feats[-1], 'pow', 2))))
    return sch, batch


def chain_schema(n: int, size: int, dom: int, seed: int, group_copies: bool = False) -> Schema:
    """The chain join S_1(X_1,X_2), ..., S_{n-1}(X_{n-1},X_n) of Sec. 3.3 with
    `size` random tuples per relation over a domain of `dom` values.  The
    tree is rooted at S_1; S_k is joined to S_{k+1} on X_{k+1}.  group_copies:
    S_k (k >= 2) also carries G{k}, a categorical copy of its join attribute
    X_k, so that Q_k(X_k; COUNT) can be declared as COUNT grouped by G{k}."""
    rng = _rng(seed)
    rels = []
    edges = []
    for k in range(1, n):
        a = rng.integers(0, dom, size=size).astype(np.int32)
        b = rng.integers(0, dom, size=size).astype(np.int32)
        cols = []
        # S_k's left attribute is the join key towards S_{k-1}
        cols.append(Column(f'X{k}', 'key' if k > 1 else 'cat', a, dom))
        cols.append(Column(f'X{k + 1}', 'key' if k < n - 1 else 'cat', b, dom))
        if group_copies and k > 1:
            cols.append(Column(f'G{k}', 'cat', a.copy(), dom))
        rels.append(Relation(f'S{k}', cols))
        if k > 1:
            edges.append((f'S{k - 1}', f'S{k}', f'X{k}'))
    return Schema(rels, edges, 'S1', meta={'name': f'chain-{n}'})


# ----------------------------------------------------------------------------
# a many-to-many join much larger than its inputs (Sec. 4, the Yelp shape)
# ----------------------------------------------------------------------------
def many_to_many(n_review: int = 1_000_000, n_user: int = 50_000, n_business: int = 20_000,
                 max_categories: int = 8, max_attributes: int = 12, seed: Optional[int] = None,
                 fact_order: str = 'sorted') -> Tuple[Schema, List[Agg]]:
    """Review(user_id, business_id, stars, useful) as the root; User(user_id;
    fans, review_count) and Business(business_id; bstars, lat) with unique
    keys; Category(business_id; cat, cat_w) and Attribute(business_id;
    attr_val) with 1..max_categories and 0..max_attributes rows per business,
    so that a review joins with |Category(b)| x |Attribute(b)| tuples and the
    join is some tens of times larger than its inputs (the shape of the Yelp
    dataset of Sec. 4, where a business has many categories and attributes);
    a business without attributes drops its reviews from the join.  Foreign
    keys Zipf 0.8; categories Zipf 1.0 over 40 values.

    Batch: the covar batch over the eight features (COUNT, SUM(x_i),
    SUM(x_i x_j): every product of two features of the fanning-out relations
    sums over their cross product per business) and COUNT grouped by cat."""
    _check_order(fact_order)
    rng = _rng(SEED_BASE + 41 if seed is None else seed)
    users = zipf_keys(rng, n_review, n_user, 0.8)
    biz = zipf_keys(rng, n_review, n_business, 0.8)
    review = Relation('Review', [Column('user_id', 'key', users), Column('business_id', 'key', biz),
                                 Column('stars', 'cont', rng.integers(1, 6, n_review).astype(np.float32)),
                                 Column('useful', 'cont', _feature(rng, n_review, 1, np.float32))])
    if fact_order == 'sorted':
        review = sort_by_join_attributes(review, ['user_id', 'business_id'])
    user = Relation('User', [Column('user_id', 'key', np.arange(n_user, dtype=np.int32)),
                             Column('fans', 'cont', _feature(rng, n_user, 1, np.float32)),
                             Column('review_count', 'cont', _feature(rng, n_user, 3, np.float32))])
    business = Relation('Business', [Column('business_id', 'key', np.arange(n_business, dtype=np.int32)),
                                     Column('bstars', 'cont', _feature(rng, n_business, 0, np.float32)),
                                     Column('lat', 'cont', _feature(rng, n_business, 2, np.float32))])
    nc = rng.integers(1, max_categories + 1, n_business)
    cb = np.repeat(np.arange(n_business, dtype=np.int32), nc)
    category = Relation('Category', [Column('business_id', 'key', cb),
                                     Column('cat', 'cat', zipf_keys(rng, len(cb), 40, 1.0), 40),
                                     Column('cat_w', 'cont', _feature(rng, len(cb), 0, np.float32))])
    na = rng.integers(0, max_attributes + 1, n_business)
    ab = np.repeat(np.arange(n_business, dtype=np.int32), na)
    attribute = Relation('Attribute', [Column('business_id', 'key', ab),
                                       Column('attr_val', 'cont', _feature(rng, len(ab), 2, np.float32))])
    sch = Schema([review, user, business, category, attribute],
                 [('Review', 'User', 'user_id'), ('Review', 'Business', 'business_id'),
                  ('Business', 'Category', 'business_id'), ('Business', 'Attribute', 'business_id')],
                 'Review')
    feats = ['stars', 'useful', 'fans', 'review_count', 'bstars', 'lat', 'cat_w', 'attr_val']
    sch.meta.update(name=f'many-to-many-{n_review}', features=feats, cats=['cat'])
    return sch, covar_batch(feats) + [Agg(group_by=('cat',))]
