"""The C-ABI library loads and exports every entry point include/spamm.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "spamm.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^SPAMM_API [^(]*?\b(spamm_\w+)\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1906_08148_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_entry_points():
    from paper_1906_08148_gb300 import spamm
    assert _declared() == sorted(spamm.ENTRY_POINTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_1906_08148_gb300", "libspamm.so")],
                         capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert set(_declared()) <= exported
    assert all(s.startswith("spamm_") for s in exported if not s.startswith("_")), "only the ABI is exported"


def test_binding_loads_and_declares_signatures(lib):
    from paper_1906_08148_gb300 import spamm
    L = spamm.load()
    for name in spamm.ENTRY_POINTS:
        assert getattr(L, name).restype is not None


def test_header_compiles_as_plain_c(tmp_path):
    src = tmp_path / "t.c"
    src.write_text('#include "spamm.h"\nint main(void){ spamm_stats s; (void)s; return SPAMM_OK; }\n')
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-c",
                           str(src), "-o", str(tmp_path / "t.o")])


def test_stats_struct_layout_matches_header(tmp_path):
    from paper_1906_08148_gb300 import spamm
    src = tmp_path / "s.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "spamm.h"\n'
                   'int main(void){ printf("%zu %zu %zu\\n", sizeof(spamm_stats), offsetof(spamm_stats, ms_cnorm),'
                   ' sizeof(spamm_gen_params)); return 0; }\n')
    exe = tmp_path / "s"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    size, off, gsize = map(int, subprocess.check_output([str(exe)]).split())
    assert size == ctypes.sizeof(spamm.Stats)
    assert off == spamm.Stats.ms_cnorm.offset
    assert gsize == ctypes.sizeof(spamm.GenParams)


def test_missing_library_fails_loudly(tmp_path):
    from paper_1906_08148_gb300 import spamm
    saved = spamm._lib
    spamm._lib = None
    try:
        with pytest.raises(ImportError):
            spamm.load(str(tmp_path / "nope.so"))
    finally:
        spamm._lib = saved
