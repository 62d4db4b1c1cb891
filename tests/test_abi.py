"""The C-ABI library loads and exports every entry point include/starbc.h declares.

CPU only: no call here launches GPU work.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "starbc.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^SP_API\s+[\w\s\*]+?\b(sp_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_abi():
    names = declared_symbols()
    for must in ["sp_graph_create", "sp_graph_destroy", "sp_bc", "sp_bc_ex", "sp_bfs", "sp_sigma",
                 "sp_server_create", "sp_bc_submit", "sp_bc_poll", "sp_bc_wait", "sp_status_string",
                 "sp_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    import paper_2401_02472_gb300 as sp

    lib = ctypes.CDLL(sp.LIB_PATH)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(declared_symbols()) == set(sp.SIGNATURES), "binding and header disagree"


def test_status_strings_and_defaults():
    import paper_2401_02472_gb300 as sp

    assert sp.sp_status_string(sp.SP_OK) == "SP_OK"
    assert sp.sp_status_string(sp.SP_ERR_RANGE) == "SP_ERR_RANGE"
    assert sp.sp_status_string(12345) == "SP_ERR_UNKNOWN"
    o = sp.make_opts()
    assert (o.precision, o.form, o.batch, o.debug_flags) == (sp.SP_FP64, sp.SP_FORM_AUTO, 0, 0)
    assert ctypes.sizeof(sp.sp_bc_opts) == 40 and ctypes.sizeof(sp.sp_bc_stats) == 104
    assert ctypes.sizeof(sp.sp_graph_info) == 48


def test_binding_structs_match_the_header(tmp_path):
    """Every field of the ctypes structs sits at the offset the C compiler gives it."""
    import shutil
    import subprocess

    import paper_2401_02472_gb300 as sp

    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "starbc.h"', "int main(void) {"]
    structs = [sp.sp_bc_opts, sp.sp_bc_stats, sp.sp_graph_info]
    for cls in structs:
        c = cls.__name__
        lines.append(f'printf("{c} size %zu\\n", sizeof({c}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{c} {f} %zu\\n", offsetof({c}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "abi"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        c, f, v = line.split()
        got[(c, f)] = int(v)
    for cls in structs:
        c = cls.__name__
        assert got[(c, "size")] == ctypes.sizeof(cls), c
        for f, _ in cls._fields_:
            assert got[(c, f)] == getattr(cls, f).offset, (c, f)


def test_argument_errors_without_a_device():
    import numpy as np
    import torch

    import paper_2401_02472_gb300 as sp

    with pytest.raises(sp.StarbcError) as e:
        sp.sp_graph_create(np.zeros(3, np.int32), np.zeros(0, np.int32), n=-1)
    assert e.value.status == sp.SP_ERR_INVALID_ARG
    if not torch.cuda.is_available():
        with pytest.raises(sp.StarbcError) as e:
            sp.sp_graph_create(np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32))
        assert e.value.status == sp.SP_ERR_NO_DEVICE
    with pytest.raises(sp.StarbcError) as e:
        sp.sp_server_create(1 << 30, 0)
    assert e.value.status == sp.SP_ERR_INVALID_ARG
