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
               'lmf_plan_stats': lmf.lmf_plan_stats, 'lmf_mi_pair': lmf.lmf_mi_pair}
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


def _prototypes():
    """name -> list of parameter declarations, from include/lmf.h."""
    with open(os.path.join(ROOT, 'include', 'lmf.h')) as f:
        text = f.read()
    text = re.sub(r'/\*.*?\*/', '', text, flags=re.S)
    text = re.sub(r'//[^\n]*', '', text)
    out = {}
    for name, params in re.findall(r'\b(lmf_[a-z_0-9]+)\s*\(([^;{)]*)\)\s*;', text, flags=re.S):
        params = ' '.join(params.split())
        out[name] = [] if params in ('', 'void') else [p.strip() for p in params.split(',')]
    return out


def test_binding_argument_types_match_the_prototypes():
    """Every binding signature has the header's parameter count, a pointer
    where the header has one, and a scalar of the header's width and kind
    elsewhere."""
    from paper_1906_08687_gb300 import lmf
    scalars = {'int': (4, int), 'int32_t': (4, int), 'uint32_t': (4, int), 'int64_t': (8, int),
               'uint64_t': (8, int),
               'size_t': (8, int), 'float': (4, float), 'double': (8, float),
               'lmf_status': (4, int), 'lmf_dtype': (4, int)}
    protos = _prototypes()
    assert set(protos) == set(declared_symbols())
    for name, params in protos.items():
        _, argtypes = lmf._SIGNATURES[name]
        assert len(argtypes) == len(params), (name, params, argtypes)
        for decl, ct in zip(params, argtypes):
            if '*' in decl:
                ok = (ct in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(ct, ctypes._Pointer)
                      or issubclass(ct, ctypes.Array))
                assert ok, (name, decl, ct)
                continue
            base = decl.replace('const ', '').split()[0]
            size, kind = scalars[base]
            assert ctypes.sizeof(ct) == size, (name, decl, ct)
            assert issubclass(ct, (ctypes.c_float, ctypes.c_double)) == (kind is float), (name, decl, ct)
