"""Host-side pieces of the learned plan choice that need no GPU: the shipped
checkpoint's shape, the feature normalisation and the regret bookkeeping."""
import json
import os

import numpy as np

from oracle import mlp as ref_mlp
from paper_1906_08687_gb300 import costmodel, lmf

HERE = os.path.dirname(os.path.abspath(costmodel.__file__))


def test_shipped_checkpoint_is_complete():
    with open(os.path.join(HERE, 'costmodel_gb300.json')) as f:
        meta = json.load(f)
    assert meta['in_dim'] == lmf.LMF_PLAN_FEATURES and meta['hidden'] == 128
    assert len(meta['mean']) == len(meta['std']) == meta['in_dim']
    assert all(s > 0 for s in meta['std']) and meta['y_std'] > 0
    p = np.fromfile(os.path.join(HERE, 'costmodel_gb300.bin'), dtype=np.float32)
    assert p.size == ref_mlp.n_params(meta['in_dim'], meta['hidden'])
    assert np.all(np.isfinite(p))
    # the study the checkpoint was trained in: training and held-out schemas of
    # the config-5 corpus, at a stated fact-table scale
    assert meta['train']['schemas'] >= 80 and meta['test']['schemas'] >= 20 and meta['scale'] > 0
    assert meta['test']['learned_regret_mean'] <= meta['test']['heuristic_regret_mean']
    # its FP64 forward pass at the normalisation centre is finite
    y, _ = ref_mlp.forward(p, np.array([meta['mean']]), np.array(meta['mean']),
                           np.array(meta['std']), meta['in_dim'], meta['hidden'])
    assert np.all(np.isfinite(y))


def test_fit_norm_guards_constant_features():
    X = np.array([[1.0, 5.0], [3.0, 5.0], [5.0, 5.0]])
    y = np.array([0.0, 1.0, 2.0])
    mean, std, ym, ys = costmodel.fit_norm(X, y)
    assert np.allclose(mean, [3.0, 5.0]) and std[1] == 1.0 and abs(std[0] - np.std([1, 3, 5])) < 1e-6
    assert ym == 1.0 and abs(ys - np.std(y)) < 1e-12


def test_regret_of_the_root_rule():
    """evaluate() without a model reports the rule's regret t(rule)/t(best) - 1."""
    recs = [{'ms': np.array([2.0, 1.0, 4.0]), 'heur_ms': 2.0, 'feat': None},
            {'ms': np.array([3.0, 3.0]), 'heur_ms': 3.0, 'feat': None}]
    out = costmodel.evaluate(None, recs)
    assert out['schemas'] == 2
    assert abs(out['heuristic_regret_mean'] - 0.5) < 1e-15
    assert abs(out['heuristic_regret_median'] - 0.5) < 1e-15
    assert 'learned_regret_mean' not in out
