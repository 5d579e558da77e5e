"""CPU checks of the boundary: libslqr.so builds for sm_103a, loads, and
exports every entry point that include/*.h declares (no compute call: there is
no GPU here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \t\*]*?\b(slqr_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2506_09463_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ["slqr_create", "slqr_destroy", "slqr_factor", "slqr_apply_qt",
                     "slqr_solve_r", "slqr_sync", "slqr_last_error"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_2506_09463_gb300 import abi
    bound = {name for name, _, _ in abi.SIGNATURES}
    assert set(declared_symbols()) <= bound | {"slqr_create"}


def test_host_only_queries(lib):
    from paper_2506_09463_gb300 import abi
    assert abi.slqr_panel_width(256, 128) in (32, 64)
    nb = abi.slqr_panel_width(8192, 8192)
    K = 8191
    panels = (K + nb - 1) // nb
    assert abi.slqr_wy_size(8192, 8192) == panels * (2 * nb * nb + nb) * 8
    assert abi.slqr_wy_size(0, 0) == 0
    assert abi.slqr_max_rows() >= 16384


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2506_09463_gb300 import abi
    with pytest.raises(abi.SlqrError):
        abi.slqr_create(0, 0)


def test_null_context_is_rejected(lib):
    from paper_2506_09463_gb300 import abi
    assert abi.slqr_factor(None, 4, 2, None, 4, None, None, None) == abi.SLQR_EINVAL
    assert abi.slqr_solve_r(None, 2, None, 2, 1, None, 2, None) == abi.SLQR_EINVAL


def test_mixed_opts_and_info_layout_match_the_header(tmp_path):
    """The ctypes mirrors of slqr_mixed_opts / slqr_mixed_info have the field
    offsets and sizes the C compiler gives the header's structs."""
    import subprocess
    from paper_2506_09463_gb300 import abi
    src = tmp_path / "layout.c"
    fields = {"slqr_mixed_opts": abi.SlqrMixedOpts, "slqr_mixed_info": abi.SlqrMixedInfo}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "slqr.h"', 'int main(void) {']
    for cname, cls in fields.items():
        lines.append(f'  printf("%zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {f}));')
    lines.append('  return 0;\n}')
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", f"-I{os.path.join(ROOT, 'include')}", "-o", str(exe),
                           str(src)])
    out = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = []
    for cls in fields.values():
        want.append(ctypes.sizeof(cls))
        want += [getattr(cls, f).offset for f, _ in cls._fields_]
    assert out == want
