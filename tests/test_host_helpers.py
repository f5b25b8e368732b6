"""Host-side checks of the index helpers the kernels share (Morton codes, the dense level
offsets, the slot of a V offset in the M2L operator table), compiled from the library's own
header with the host compiler.  Each is pinned to its definition, not to another copy of
the formula:

* m2l_slot: the rank of an offset among the 316 offsets with max(|o|) >= 2 of [-3, 3]^3,
  taken in the order of the code (ox + 3) + 7 (oy + 3) + 49 (oz + 3) (the M2L table layout);
* dense_off(l): the number of slots of the levels above l, sum of 8^m for m < l;
* morton3 / demorton3: inverse to each other, and a value worked out by hand.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2112_10059_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

PROBE = r'''
#include "sph_kernels.cuh"
#include <cstdio>
int main() {
    using namespace sph;
    for (int oz = -3; oz <= 3; ++oz)
        for (int oy = -3; oy <= 3; ++oy)
            for (int ox = -3; ox <= 3; ++ox) {
                const bool adj = ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1;
                printf("%d\n", adj ? -1 : m2l_slot(ox, oy, oz));
            }
    for (int l = 0; l < 11; ++l) printf("%lld\n", (long long)dense_off(l));
    int bad = 0;
    for (unsigned i = 0; i < 1024; i += 37)
        for (unsigned j = 0; j < 1024; j += 41)
            for (unsigned k = 0; k < 1024; k += 43) {
                unsigned a, b, c;
                demorton3(morton3(i, j, k), a, b, c);
                bad += a != i || b != j || c != k;
            }
    printf("%d\n%u\n", bad, morton3(5, 3, 6));
    return 0;
}
'''


@pytest.fixture(scope="module")
def probe_output(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("host compiler or CUDA headers missing")
    d = tmp_path_factory.mktemp("host_helpers")
    src = d / "probe.cpp"
    exe = d / "probe"
    src.write_text(PROBE)
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CUDA_INC, "-I", CSRC, str(src), "-o", str(exe)], check=True,
                   capture_output=True, timeout=120)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=60).stdout.split()
    return [int(x) for x in out]


def test_m2l_slot_is_the_rank_among_far_offsets(probe_output):
    slots = probe_output[:343]
    expect, rank = [], 0
    for code in range(343):
        ox, oy, oz = code % 7 - 3, (code // 7) % 7 - 3, code // 49 - 3
        if max(abs(ox), abs(oy), abs(oz)) <= 1:
            expect.append(-1)
        else:
            expect.append(rank)
            rank += 1
    assert rank == 316
    assert slots == expect


def test_dense_offsets_count_the_slots_above(probe_output):
    offs = probe_output[343:354]
    assert offs == [sum(8 ** m for m in range(l)) for l in range(11)]


def test_morton_round_trip_and_worked_value(probe_output):
    bad, m = probe_output[354], probe_output[355]
    assert bad == 0
    # x = 101b, y = 011b, z = 110b: bit triples (z y x) per level 011, 110, 101 -> 101 110 011b
    assert m == 0b101110011
