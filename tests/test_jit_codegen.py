"""The plan-time code generator without a GPU: sources generated for plans of
several shapes (sorted snowflake with resident key and category views,
fanning-out joins, more tables than the kernel parameters hold, FP64 and root
categories, wide z, a root without probe groups) compile for sm_103a with
NVRTC, for the plain and the tensor-core scan, and the key-level scan with its
bulk, runs and resident-key reverse views, and the tree pass with its
decision tree over the nodes' predicates (spelled out, or searched through
the device tables when too large)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.timeout(600)
def test_generated_sources_compile(tmp_path):
    from paper_1906_08687_gb300 import build
    build.build()
    nvcc = build._nvcc()
    if shutil.which(nvcc) is None and not os.path.exists(nvcc):
        pytest.skip('nvcc not found')
    exe = tmp_path / 'jit_codegen_check'
    csrc = os.path.join(ROOT, 'paper_1906_08687_gb300', 'csrc')
    cmd = [nvcc, '-std=c++17', '-I', csrc, '-I', os.path.join(ROOT, 'include'), '-I', build.OUT_DIR,
           os.path.join(ROOT, 'tests', 'jit_codegen_check.cu'), '-o', str(exe), '-ldl']
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=500)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    ok = [l for l in r.stdout.splitlines() if l.startswith('ok ')]
    assert len(ok) == 11, r.stdout
