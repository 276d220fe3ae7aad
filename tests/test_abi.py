"""The C-ABI library builds, loads without a GPU, and exports what include/cgp.h declares."""

import os
import re

from paper_1812_00185_gb300 import binding

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "cgp.h")


def declared():
    txt = open(HDR).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cgp_[a-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported_and_bound():
    lib = binding.load()
    names = declared()
    assert "cgp_step" in names and "cgp_mesh_create" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(binding.exported_symbols()) | {n for n in names if hasattr(lib, n)}


def test_last_error_is_callable_without_gpu():
    assert binding.cgp_last_error() == ""


def test_struct_layouts_match_the_c_compiler(tmp_path):
    # compile a probe with the system C compiler and compare every field offset
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest
        pytest.skip("no C compiler")
    structs = {"cgp_mesh_desc": binding.MeshDesc, "cgp_params": binding.Params, "cgp_stats": binding.Stats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "cgp.h"', "int main(void){"]
    for cname, cls in structs.items():
        lines.append('printf("%%s %%zu\\n", "%s", sizeof(%s));' % (cname, cname))
        for f, _ in cls._fields_:
            lines.append('printf("%%s.%%s %%zu\\n", "%s", "%s", offsetof(%s, %s));' % (cname, f, cname, f))
    lines.append("return 0;}")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run([cc, "-I", os.path.dirname(HDR), str(src), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                          check=True).stdout.splitlines())
    for cname, cls in structs.items():
        assert int(out[cname]) == binding.ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(out["%s.%s" % (cname, f)]) == getattr(cls, f).offset, (cname, f)
