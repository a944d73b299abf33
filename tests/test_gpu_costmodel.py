"""The learned plan choice end to end on a small corpus: candidates are timed
on the GPU, the cost model is trained by the engine's kernels, and its choices
are compared with the exhaustive best and the root rule (Sec. 3.3)."""
import numpy as np
import pytest

from workloads import config5_schema

pytestmark = pytest.mark.gpu


def test_small_study_learns_and_plans():
    from paper_1906_08687_gb300 import costmodel, Engine, register_schema
    from lmf_testlib import to_device
    schemas = [config5_schema(i, n_scale=0.003) for i in range(14)]
    recs = costmodel.collect(schemas, runs=3)
    assert all(len(r['ms']) >= 4 for r in recs)
    model, losses = costmodel.train(recs[:10], steps=600, lr=2e-3)
    assert np.mean(losses[-30:]) < 0.5 * np.mean(losses[:10])
    tr = costmodel.evaluate(model, recs[:10])
    te = costmodel.evaluate(model, recs[10:])
    print('train', tr, 'test', te)
    assert tr['learned_regret_mean'] <= tr['heuristic_regret_mean'] + 0.05
    # the C planner's learned choice equals the argmin of the predictions
    sch, batch = schemas[11]
    eng = Engine(0)
    tens = to_device(sch)
    register_schema(eng, sch, tens)
    bid = eng.declare_batch(batch)
    chosen = eng.plan_learned(bid, model)
    i = int(np.argmin(costmodel.predict(model, recs[11]['feat'])))
    assert costmodel._opts_tuple(chosen) == recs[11]['cand'][i]
    eng.close()
