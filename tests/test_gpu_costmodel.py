"""The learned plan choice end to end: candidates are compiled and timed on the
GPU, the cost model is trained by the engine's kernels, and its choices are
compared with the exhaustive best and the root rule (Sec. 3.3) on schemas it
was not trained on."""
import json

import numpy as np
import pytest

from workloads import config5_schema

pytestmark = pytest.mark.gpu


def test_small_study_learns_and_plans():
    """A small corpus: the loss falls, and the C planner's learned choice is the
    argmin of the model's predictions over the candidates."""
    from paper_1906_08687_gb300 import costmodel, Engine, register_schema
    from workloads import to_device
    schemas = [config5_schema(i, n_scale=0.003) for i in range(12)]
    recs = costmodel.collect(schemas, runs=3)
    assert all(len(r['ms']) >= 2 for r in recs)
    model, losses = costmodel.train(recs[:9], steps=600, lr=2e-3)
    assert np.mean(losses[-30:]) < 0.5 * np.mean(losses[:10])
    sch, batch = schemas[10]
    eng = Engine(0)
    tens = to_device(sch)
    register_schema(eng, sch, tens)
    bid = eng.declare_batch(batch)
    chosen = eng.plan_learned(bid, model)
    i = int(np.argmin(costmodel.predict(model, recs[10]['feat'])))
    assert costmodel._opts_tuple(chosen) == recs[10]['cand'][i]
    eng.run(bid)              # the chosen plan is compiled and runs
    eng.sync(bid)
    eng.close()


def test_shipped_checkpoint_beats_rule_on_held_out():
    """The shipped checkpoint against the root rule on corpus schemas beyond
    its training split (indices from 'train.schemas' on), at the study's fact
    scale: the learned choice's mean regret against the exhaustive best is no
    larger than the rule's."""
    from paper_1906_08687_gb300 import costmodel
    model, origin = costmodel.load_shipped(0)
    assert model is not None, origin
    with open(costmodel.SHIPPED + '.json') as f:
        meta = json.load(f)
    first = meta['train']['schemas']
    scale = meta['scale']
    held = [config5_schema(first + i, n_scale=scale) for i in range(6)]
    recs = costmodel.collect(held, runs=3)
    res = costmodel.evaluate(model, recs)
    print(origin, res)
    assert res['learned_regret_mean'] <= res['heuristic_regret_mean'] + 1e-9, res
