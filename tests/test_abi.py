"""The C-ABI library loads and exports every entry point include/lmf.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, 'include', 'lmf.h')) as f:
        text = f.read()
    text = re.sub(r'/\*.*?\*/', '', text, flags=re.S)
    return sorted(set(re.findall(r'\b(lmf_[a-z_0-9]+)\s*\(', text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ['lmf_create', 'lmf_destroy', 'lmf_register_relation', 'lmf_declare_join',
              'lmf_declare_batch', 'lmf_plan', 'lmf_run', 'lmf_sync', 'lmf_read_results',
              'lmf_result_info', 'lmf_status_string']:
        assert s in syms


def test_library_exports_every_declared_symbol():
    from paper_1906_08687_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_1906_08687_gb300 import lmf
    assert set(declared_symbols()) <= set(lmf._SIGNATURES), \
        set(declared_symbols()) - set(lmf._SIGNATURES)


def test_status_strings_without_gpu():
    from paper_1906_08687_gb300 import lmf
    lib = lmf.load()
    assert lib.lmf_status_string(0) == b'ok'
    assert b'tree' in lib.lmf_status_string(-2)
    # a context cannot be created without a device: the call fails cleanly
    h = ctypes.c_void_p()
    import torch
    if not torch.cuda.is_available():
        assert lib.lmf_create(0, ctypes.byref(h)) == lmf.LMF_ERR_CUDA


def test_struct_layouts_match_header(tmp_path):
    """ctypes mirrors of the ABI structs have the sizes and field offsets the C
    compiler gives the header's structs."""
    import subprocess
    from paper_1906_08687_gb300 import lmf
    structs = {'lmf_column': lmf.lmf_column, 'lmf_factor': lmf.lmf_factor,
               'lmf_agg_spec': lmf.lmf_agg_spec, 'lmf_plan_opts': lmf.lmf_plan_opts,
               'lmf_plan_stats': lmf.lmf_plan_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lmf.h"', 'int main(void) {']
    for name, cls in structs.items():
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ['  return 0;', '}']
    src = tmp_path / 'layout.c'
    src.write_text('\n'.join(lines))
    exe = tmp_path / 'layout'
    subprocess.run(['gcc', '-I', os.path.join(ROOT, 'include'), str(src), '-o', str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split('\n')
    want = dict(l.split() for l in out if l.strip())
    for name, cls in structs.items():
        assert int(want[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(want[f'{name}.{f}']) == getattr(cls, f).offset, (name, f)
