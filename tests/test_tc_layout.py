"""The tensor-core operand layout and descriptors, checked on the CPU.

The tcgen05 kernels keep their operands K-major without swizzling: a matrix of
R rows x K elements is tiled into core matrices of 8 rows x 16 bytes, each one
contiguous 128-byte block (row r of it at byte 16 r); core matrices adjacent
along K are LBO bytes apart and groups of 8 rows SBO bytes apart.  The shared
memory descriptor carries start address / 16 in bits 0-13, LBO / 16 in bits
16-29, SBO / 16 in bits 32-45, the constant 0b001 in bits 46-48 and no
swizzle (bits 61-63 = 0); the instruction descriptor carries the F32
accumulator format, the operand formats, N / 8 and M / 16.

A host program compiled with nvcc calls the library's own header functions
(tc::core_offset, tc::smem_desc, tc::instr_desc) and prints their results; the
test checks them against that layout.  Exchanging LBO and SBO (the mistake the
GPU self-check once planted) breaks the layout and is caught here."""
import os
import shutil
import subprocess

import pytest

from conftest import ROOT

SRC = r"""
#include <cstdio>
#include <cstdlib>
#include "apd_tcgen05.cuh"
int main(int argc, char **argv) {
    const int eb = atoi(argv[1]), rows = atoi(argv[2]), K = atoi(argv[3]);
    const unsigned lbo = (unsigned)atoi(argv[4]), sbo = (unsigned)atoi(argv[5]);
    for (int r = 0; r < rows; ++r)
        for (int k = 0; k < K; ++k) printf("%u\n", apd::tc::core_offset(r, k, eb, lbo, sbo));
    printf("D %llu\n", (unsigned long long)apd::tc::smem_desc(0x12340u, lbo, sbo));
    printf("I %u %u\n", apd::tc::instr_desc(apd::tc::KIND_TF32, 128, 32), apd::tc::instr_desc(apd::tc::KIND_BF16, 128, 32));
    return 0;
}
"""


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("tclayout")
    src = d / "layout.cu"
    src.write_text(SRC)
    exe = d / "layout"
    inc = os.path.join(ROOT, "paper_2403_03571_gb300", "csrc")
    subprocess.run([nvcc, "-std=c++17", "-I", inc, "-o", str(exe), str(src)], check=True, capture_output=True)
    return str(exe)


def run(prog, eb, rows, K, lbo, sbo):
    out = subprocess.run([prog, str(eb), str(rows), str(K), str(lbo), str(sbo)], check=True,
                         capture_output=True, text=True).stdout.split("\n")
    offs = [int(v) for v in out[:rows * K]]
    desc = int(out[rows * K].split()[1])
    idesc = [int(v) for v in out[rows * K + 1].split()[1:]]
    return offs, desc, idesc


def layout_ok(offs, eb, rows, K, lbo, sbo):
    epr = 16 // eb
    size = rows * K * eb
    if sorted(offs) != list(range(0, size, eb)):
        return False  # not a bijection onto the operand's bytes
    for r in range(rows):
        for k in range(K):
            o = offs[r * K + k]
            base = (r // 8) * sbo + (k // epr) * lbo  # the core matrix's 128-byte block
            if not (base <= o < base + 128) or o - base != (r % 8) * 16 + (k % epr) * eb:
                return False
    return True


@pytest.mark.parametrize("eb,rows", [(4, 128), (2, 128), (4, 32), (2, 32)])
def test_core_matrix_layout_and_descriptors(prog, eb, rows):
    K = 32
    lbo, sbo = 128, (K // (16 // eb)) * 128  # the kernels' choice: K-adjacent core matrices contiguous
    offs, desc, idesc = run(prog, eb, rows, K, lbo, sbo)
    assert layout_ok(offs, eb, rows, K, lbo, sbo)
    assert desc & 0x3FFF == (0x12340 & 0x3FFFF) >> 4
    assert (desc >> 16) & 0x3FFF == lbo >> 4
    assert (desc >> 32) & 0x3FFF == sbo >> 4
    assert (desc >> 46) & 0x7 == 1
    assert (desc >> 49) & 0x7 == 0 and (desc >> 61) & 0x7 == 0
    for kind, d in zip(("tf32", "bf16"), idesc):
        assert (d >> 4) & 0x3 == 1                       # D: F32
        fmt = 2 if kind == "tf32" else 1
        assert (d >> 7) & 0x7 == fmt and (d >> 10) & 0x7 == fmt
        assert (d >> 15) & 0x3 == 0                      # A and B K-major
        assert (d >> 17) & 0x3F == 32 >> 3 and (d >> 24) & 0x1F == 128 >> 4


def test_exchanged_offsets_break_the_layout(prog):
    eb, rows, K = 2, 128, 32
    lbo, sbo = 128, (K // 8) * 128
    offs, _, _ = run(prog, eb, rows, K, sbo, lbo)  # planted mistake: LBO and SBO exchanged
    assert not layout_ok(offs, eb, rows, K, lbo, sbo)
