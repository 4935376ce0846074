"""The tcgen05 descriptor encodings (csrc/tc_desc.h), compiled on the host and
decoded field by field with the bit layouts of the PTX ISA's tcgen05
instruction descriptor (.kind::tf32) and shared-memory matrix descriptor."""
import os
import subprocess
import tempfile

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2302_07084_gb300", "csrc")

PROG = r"""
#include <stdio.h>
#include "tc_desc.h"
int main() {
    const int ns[] = {16, 48, 144, 160, 256};
    for (int i = 0; i < 5; ++i) printf("i %d %u\n", ns[i], lne::tc_idesc_tf32(128, ns[i]));
    const unsigned addrs[] = {0u, 1024u, 1056u, 70656u, 232448u - 1024u};
    for (int i = 0; i < 5; ++i) printf("s %u %llu\n", addrs[i], (unsigned long long)lne::tc_sdesc_sw128(addrs[i]));
    return 0;
}
"""


def bits(v, lo, hi):
    """Bits lo..hi (inclusive) of v."""
    return (v >> lo) & ((1 << (hi - lo + 1)) - 1)


@pytest.fixture(scope="module")
def values():
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "p.cc"), os.path.join(d, "p")
        with open(src, "w") as f:
            f.write(PROG)
        subprocess.run(["g++", "-std=c++17", "-I", CSRC, src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    idesc, sdesc = {}, {}
    for line in out:
        if not line:
            continue
        kind, a, v = line.split()
        (idesc if kind == "i" else sdesc)[int(a)] = int(v)
    return idesc, sdesc


def test_instruction_descriptor_fields(values):
    idesc, _ = values
    for n, v in idesc.items():
        assert bits(v, 0, 1) == 0 and bits(v, 2, 2) == 0 and bits(v, 3, 3) == 0   # dense, no saturate
        assert bits(v, 4, 5) == 1                          # D: F32
        assert bits(v, 6, 6) == 0
        assert bits(v, 7, 9) == 2 and bits(v, 10, 12) == 2  # A, B: TF32
        assert bits(v, 13, 14) == 0                        # no negation
        assert bits(v, 15, 15) == 0 and bits(v, 16, 16) == 0   # both K-major
        assert bits(v, 17, 22) == n >> 3                   # N / 8
        assert bits(v, 23, 23) == 0
        assert bits(v, 24, 28) == 128 >> 4                 # M / 16
        assert bits(v, 29, 31) == 0
        assert n % 16 == 0 and 16 <= n <= 256              # valid N for M = 128


def test_shared_memory_descriptor_fields(values):
    _, sdesc = values
    for addr, v in sdesc.items():
        assert bits(v, 0, 13) == (addr & 0x3FFFF) >> 4     # start address / 16
        assert bits(v, 14, 15) == 0
        assert bits(v, 16, 29) == 1                        # leading byte offset (unused by the swizzle)
        assert bits(v, 30, 31) == 0
        assert bits(v, 32, 45) == 1024 >> 4                # stride byte offset: 8 rows x 128 B
        assert bits(v, 46, 48) == 0b001                    # fixed constant
        assert bits(v, 49, 51) == 0                        # base offset
        assert bits(v, 52, 52) == 0                        # relative leading-offset mode
        assert bits(v, 53, 60) == 0
        assert bits(v, 61, 63) == 2                        # 128-byte swizzle
