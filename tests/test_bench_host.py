"""Host-side pieces of bench.py that need no GPU: the CPU-baseline leg, the
workload description, the ncu-summary lookup."""
import os

import bench
from workloads import config1, config2, config4


def test_cpu_baseline_leg():
    sch, batch = config1(20_000)
    cb = bench.cpu_baseline(sch, batch, n_fact=20_000, sample_rows=5_000, single_thread=True)
    assert cb['kind'] == 'oracle' and cb['unit'] == bench.UNIT
    assert cb['cores'] >= 1 and cb['value'] > 0 and cb['value_1thread'] > 0
    assert 'first 5000 fact rows' in cb['sample'] and f'all {len(batch)} aggregates' in cb['sample']
    assert isinstance(cb['cpu'], str) and cb['cpu']
    assert 'value_1thread' not in bench.cpu_baseline(sch, batch, 20_000, 1_000)


def test_fact_order_text_names_each_workloads_sort_keys():
    for gen, keys in [(config1, '(k2, k1)'), (config2, '(k3, k2, k1)'), (config4, '(k1, k2, k3, k4)')]:
        sch, _ = gen(1000)
        assert keys in bench.fact_order_text(sch, 'sorted')
        assert bench.fact_order_text(sch, 'random') == 'generation order (i.i.d. rows)'


def test_profiled_traffic_follows_the_kernel_sources():
    """A committed ncu summary counts only while its recorded source hash is
    the current one; every workload that names a summary has one."""
    h = bench.kernel_hash()
    assert len(h) == 16
    for name, spec in bench.WORKLOADS.items():
        summary = spec[6]
        if summary is None:
            continue
        path = os.path.join(bench.ROOT, 'profiles', summary)
        assert os.path.exists(path), name
        with open(path) as f:
            text = f.read()
        # a traffic figure with its source hash, or a statement that there is none
        assert 'traffic_bytes_per_launch[' in text or '`traffic` as null' in text, name
    assert bench.profiled_traffic('plain', os.path.join(bench.ROOT, 'profiles', 'no_such.md')) is None
    # the headline workload's summary was taken on the current kernel sources
    snow = os.path.join(bench.ROOT, 'profiles', bench.WORKLOADS['snowflake'][6])
    assert bench.profiled_traffic('keylevel', snow) is not None
