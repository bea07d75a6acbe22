"""The operand-term tile layout of the tensor-core forms (csrc/tcforms.cuh),
compiled for the host: for every K split (1, 2 or 4 parts, in the 128-,
64- and 32-byte swizzles) each element of a leaf's terms has its own
two-byte slot inside the leaf's terms, eight consecutive k share one 16-byte
chunk, every part of a leaf (all its terms) is one contiguous block, inside
it the 8-row atom g of term s sits at (g TERMS + s) x atom (so the 128-row
operand of term s over two such blocks is one strided matrix), and the chunk
order inside a row follows the swizzle (chunk index XOR the row bits above
the atom's row stride)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1906_08148_gb300", "csrc")
INC = os.path.join(ROOT, "include")


@pytest.fixture(scope="module")
def lay(tmp_path_factory):
    d = str(tmp_path_factory.mktemp("tcforms"))
    src = os.path.join(d, "shim.cpp")
    with open(src, "w") as f:
        f.write("#define __host__\n#define __device__\n#define __forceinline__ inline\n"
                '#include "tcforms.cuh"\n'
                'extern "C" void offsets(int kp, int terms, unsigned* out) {\n'
                "  int i = 0;\n"
                "  for (int s = 0; s < terms; ++s)\n"
                "    for (int r = 0; r < 64; ++r)\n"
                "      for (int k = 0; k < 64; ++k, ++i)\n"
                "        out[i] = kp == 1 ? spamm::term_offset<1>(terms, s, r, k)\n"
                "               : kp == 2 ? spamm::term_offset<2>(terms, s, r, k) : spamm::term_offset<4>(terms, s, r, k);\n"
                "}\n")
    so = os.path.join(d, "libshim.so")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-I", CSRC, "-I", INC, "-o", so, src])
    lib = ctypes.CDLL(so)
    lib.offsets.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    return lib


@pytest.mark.parametrize("kp", [1, 2, 4])
@pytest.mark.parametrize("terms", [2, 3, 4])
def test_term_layout_is_a_swizzled_bijection(lay, kp, terms):
    out = np.empty(terms * 64 * 64, np.uint32)
    lay.offsets(kp, terms, out.ctypes.data)
    off = out.reshape(terms, 64, 64).astype(np.int64)
    assert np.all(off % 2 == 0)
    assert np.array_equal(np.sort(off.ravel()), 2 * np.arange(terms * 4096))
    # eight consecutive k (one chunk) are one contiguous 16-byte chunk
    ch = off.reshape(terms, 64, 8, 8)
    assert np.all(ch[..., 0] % 16 == 0) and np.all(np.diff(ch, axis=-1) == 2)
    part = 8192 // kp
    kw = 64 // kp
    rowb = 2 * kw  # bytes per tile row
    atom = 8 * rowb
    for h in range(kp):
        blk = off[:, :, h * kw:(h + 1) * kw]
        base = h * terms * part
        assert blk.min() == base and blk.max() == base + terms * part - 2
        for s in range(terms):
            for g in range(8):
                a = blk[s, 8 * g:8 * g + 8] - base
                start = (g * terms + s) * atom
                assert a.min() == start and a.max() == start + atom - 2
                rel = a - start
                assert np.array_equal(rel // rowb, np.repeat(np.arange(8)[:, None], kw, axis=1))
                chunk = (rel % rowb) // 16
                nchunk = rowb // 16
                want = (np.arange(kw)[None, :] // 8) ^ ((np.arange(8)[:, None] * rowb >> 7) % nchunk)
                assert np.array_equal(chunk, want)
