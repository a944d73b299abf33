"""The tree planner without a GPU: a tree level's aggregates decompose into
one node per leaf, one group of exclusive nodes, and a decision tree with one
entry per tree node and the level's depth, through which every point finds
the one node it satisfies (tests/tree_plan_check.cu)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.timeout(600)
def test_tree_planner(tmp_path):
    from paper_1906_08687_gb300 import build
    build.build()
    nvcc = build._nvcc()
    if shutil.which(nvcc) is None and not os.path.exists(nvcc):
        pytest.skip('nvcc not found')
    exe = tmp_path / 'tree_plan_check'
    csrc = os.path.join(ROOT, 'paper_1906_08687_gb300', 'csrc')
    cmd = [nvcc, '-std=c++17', '-O2'] + build.ARCH + [
        '--expt-relaxed-constexpr', '-I', csrc, '-I', os.path.join(ROOT, 'include'), '-I', build.OUT_DIR,
        os.path.join(ROOT, 'tests', 'tree_plan_check.cu'), '-o', str(exe)]
    c = subprocess.run(cmd, capture_output=True, text=True)
    assert c.returncode == 0, c.stderr[-3000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    ok = [l for l in r.stdout.splitlines() if l.startswith('ok ')]
    assert len(ok) == 12, r.stdout
