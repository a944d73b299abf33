"""The tree planner without a GPU (tests/tree_plan_check.cu).

* A tree level's aggregates decompose into one node per leaf, one group of
  exclusive nodes, and a decision tree with one entry per tree node and the
  level's depth, through which every point finds the one node it satisfies.
* The node search that the plan-time compiler writes out as nested
  comparisons (the compiled tree pass) is compiled here as host code and
  gives, at points on, just below and just above every threshold and at
  random points, the node that a brute-force search over each group finds:
  for a complete level, for nested levels (several groups) and for random
  overlapping conjunctions.
"""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _check_exe(tmp_path):
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
    return exe


@pytest.fixture(scope='module')
def check_exe(tmp_path_factory):
    return _check_exe(tmp_path_factory.mktemp('tree_plan'))


@pytest.mark.timeout(600)
def test_tree_planner(check_exe):
    r = subprocess.run([str(check_exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    ok = [l for l in r.stdout.splitlines() if l.startswith('ok ')]
    assert len(ok) == 18, r.stdout


_HOST = r'''#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>
struct TreeDev {};
constexpr uint16_t kNoNode = 0xFFFF;
static inline float __uint_as_float(unsigned u) { float f; std::memcpy(&f, &u, 4); return f; }
%s
int main(int argc, char** argv) {
  FILE* f = std::fopen(argv[1], "r");
  int G, P, NZ;
  if (!f || std::fscanf(f, "%%d %%d %%d", &G, &P, &NZ) != 3) return 2;
  TreeDev d;
  long bad = 0, total = 0;
  std::vector<float> z(NZ);
  for (int t = 0; t < P; ++t) {
    for (int i = 0; i < NZ; ++i) {
      unsigned u;
      if (std::fscanf(f, "%%x", &u) != 1) return 2;
      z[i] = __uint_as_float(u);
    }
    for (int g = 0; g < G; ++g) {
      int want;
      if (std::fscanf(f, "%%d", &want) != 1) return 2;
      ++total;
      if (node(d, g, z.data()) != want) ++bad;
    }
  }
  std::printf("%%ld of %%ld differ\n", bad, total);
  return bad ? 1 : 0;
}
'''


@pytest.mark.timeout(600)
def test_generated_node_search(check_exe, tmp_path):
    gxx = shutil.which('g++') or shutil.which('c++')
    if gxx is None:
        pytest.skip('no host C++ compiler')
    out = tmp_path / 'cases'
    out.mkdir()
    r = subprocess.run([str(check_exe), '--emit', str(out)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    cases = sorted(p for p in os.listdir(out) if p.startswith('case_') and p.endswith('.cu'))
    assert len(cases) == 7, r.stdout
    groups = [int(m) for m in re.findall(r'(\d+) groups', r.stdout)]
    assert groups[0] == 1 and max(groups[1:]) > 1, r.stdout     # one group, and cases with several
    for name in cases:
        src = open(out / name).read()
        head = 'static __device__ __forceinline__ int node(const TreeDev& d, int g, const float* zrow) {'
        i = src.index(head)
        j = src.index('\n};\n}  // namespace lmf', i)
        fn = 'static int node(const TreeDev& d, int g, const float* zrow) {' + src[i + len(head):j]
        assert 'tree_node_of' not in fn        # written out, not the table search
        host = tmp_path / (name[:-3] + '_host.cpp')
        host.write_text(_HOST % fn)
        exe = tmp_path / (name[:-3] + '_host')
        c = subprocess.run([gxx, '-std=c++17', '-O1', str(host), '-o', str(exe)], capture_output=True, text=True)
        assert c.returncode == 0, c.stderr[-3000:]
        run = subprocess.run([str(exe), str(out / (name[:-3] + '.txt'))], capture_output=True, text=True,
                             timeout=120)
        assert run.returncode == 0, (name, run.stdout, run.stderr)


@pytest.mark.timeout(900)
def test_generated_row_pass(check_exe, tmp_path):
    from paper_1906_08687_gb300 import build
    out = tmp_path / 'cases'
    out.mkdir()
    r = subprocess.run([str(check_exe), '--emit', str(out)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    rows = sorted(p for p in os.listdir(out) if p.startswith('row_case_'))
    assert len(rows) == 3
    csrc = os.path.join(ROOT, 'paper_1906_08687_gb300', 'csrc')
    for name in rows:
        k = int(name[len('row_case_'):-3])
        src = open(out / name).read()
        head = ('static __device__ __forceinline__ long long row(const RootParams& p, int64_t r, float* zrow, '
                'int32_t* crow) {')
        i = src.index(head)
        j = src.index('  static __device__ __forceinline__ int node(', i)
        fn = ('static long long gen_row(const lmf::RootParams& p, int64_t r, float* zrow, int32_t* crow) {'
              + src[i + len(head):j])
        hdr = tmp_path / ('row_%d.h' % k)
        hdr.write_text(fn)
        exe = tmp_path / ('row_%d' % k)
        cmd = [build._nvcc(), '-std=c++17', '-O1', '-I', csrc, '-I', os.path.join(ROOT, 'include'),
               '-I', os.path.join(ROOT, 'tests'), '-DTREE_ROW_CASE=%d' % k, '-DTREE_ROW_HEADER="%s"' % hdr,
               os.path.join(ROOT, 'tests', 'tree_row_host.cu'), '-o', str(exe)]
        c = subprocess.run(cmd, capture_output=True, text=True)
        assert c.returncode == 0, c.stderr[-3000:]
        run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
        assert run.returncode == 0, (name, run.stdout, run.stderr)
