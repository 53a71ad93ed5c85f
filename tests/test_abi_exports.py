"""The C-ABI library builds, loads and exports every function include/prism.h declares,
and the binding's struct layouts match the C compiler's (no GPU calls)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2606_23367_gb300 import build, prism

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "prism.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return prism.load_library()


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(prism_[a-z_]+)\s*\(", text)))


def test_every_declared_function_is_exported(lib):
    names = _declared_functions()
    assert "prism_solve_batch" in names and "prism_create_universe" in names
    assert "prism_solve_batch_backward" in names
    for n in names:
        assert hasattr(lib, n), n


def test_version_and_defaults_need_no_gpu(lib):
    assert "sm_103a" in prism.prism_version()
    o = prism.prism_default_opts()
    assert o["eps_kkt"] == 1e-6 and o["precision"] == prism.PRISM_BATCHED_BF16
    assert o["max_iter"] > 0 and 0 < o["alpha"] < 2


def test_struct_layouts_match_the_c_compiler(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "prism.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(prism_universe_desc),'
                   ' sizeof(prism_batch), sizeof(prism_solve_opts), sizeof(prism_result),'
                   ' offsetof(prism_result, t_device_ms), offsetof(prism_solve_opts, cuda_stream));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    got = [int(x) for x in out]
    want = [ctypes.sizeof(prism._UniverseDesc), ctypes.sizeof(prism._Batch), ctypes.sizeof(prism._Opts),
            ctypes.sizeof(prism._Result), prism._Result.t_device_ms.offset, prism._Opts.cuda_stream.offset]
    assert got == want


def test_every_field_offset_matches_the_c_compiler(tmp_path):
    """Field by field: the ctypes structures of the binding and the C header agree on every
    member's offset (a reordered or resized member in either fails here)."""
    structs = [(prism._UniverseDesc, "prism_universe_desc"), (prism._Batch, "prism_batch"),
               (prism._Opts, "prism_solve_opts"), (prism._Result, "prism_result")]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "prism.h"', 'int main(void){']
    want = []
    for cls, cname in structs:
        for name, _ in cls._fields_:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {name}));')
            want.append((cname, name, getattr(cls, name).offset))
    lines.append('return 0;}')
    src = tmp_path / "off.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "off"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert len(got) == len(want)
    bad = [(c, n, w, g) for (c, n, w), g in zip(want, got) if w != g]
    assert not bad, bad
