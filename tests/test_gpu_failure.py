"""Failure detection on the GPU without a fault: a bounded device wait runs
out on a barrier nothing arrives at, reports LMF_ERR_TIMEOUT through the
status word, and the context stays usable."""
import numpy as np
import pytest

from oracle import oracle
from workloads import config1

from lmf_testlib import ARITH_FLOOR, compare, run_engine

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    from paper_1906_08687_gb300 import Engine
    from paper_1906_08687_gb300.lmf import LMF_ERR_TIMEOUT
    eng = Engine(0)
    assert eng.wait_selftest() == LMF_ERR_TIMEOUT
    assert 'gave up' in eng.lib.lmf_error_message(eng.ctx).decode()
    sch, batch = config1(20_000)
    got, info, _ = run_engine(sch, batch, precision=1, batching=1, engine=eng)
    fails, _ = compare(got, oracle.evaluate(sch, batch), arith_floor=ARITH_FLOOR)
    assert not fails
    eng.close()
