"""Host-side rules of the library's work split, compiled on the CPU.

The heavy-row split (parts of a bitmap row in the numeric and the symbolic
phase) and the heaviest-first buckets of the numeric bitmap work items are
plain functions in the library's internal header, shared by host and device
code.  This test compiles a small host program against that header with
nvcc (no GPU needed) and checks the functions' values against their stated
rules at and around every boundary."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1804_01698_gb300", "csrc")

PROGRAM = r'''
#include <cstdio>
#include "internal.h"
int main() {
  const long long w[] = {0, 1, 2, 16383, 16384, 32767, 32768, 65535, 65536, 131071, 131072,
                         262143, 262144, 524287, 524288, 1048575, 1048576, 1LL << 40};
  for (long long x : w) std::printf("bucket %lld %d\n", x, sg::bm_bucket_of(x, 1));
  std::printf("bucketp %d %d %d\n", sg::bm_bucket_of(1 << 20, 2), sg::bm_bucket_of(1 << 20, 0),
              sg::bm_bucket_of(3 << 18, 3));
  const long long f[] = {0, 32767, 65535, 65536, 98304, 131072, 32768LL * 64, 32768LL * 1000};
  for (long long x : f) std::printf("sym %lld %d\n", x, sg::sym_split_parts(x));
  const long long bf[][2] = {{600000, 5000}, {600000, 100000}, {131071, 1}, {131072, 1}, {1LL << 40, 10}};
  for (auto &b : bf) std::printf("bm %lld %lld %d\n", b[0], b[1], sg::bm_split_parts(b[0], b[1]));
  return 0;
}
'''


@pytest.fixture(scope="module")
def rules(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("rules")
    src = d / "rules.cu"
    src.write_text(PROGRAM)
    exe = d / "rules"
    subprocess.run([nvcc, "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    res = {"bucket": {}, "sym": {}, "bm": {}}
    for line in out.splitlines():
        f = line.split()
        if f[0] == "bucket":
            res["bucket"][int(f[1])] = int(f[2])
        elif f[0] == "bucketp":
            res["bucketp"] = [int(x) for x in f[1:]]
        elif f[0] == "sym":
            res["sym"][int(f[1])] = int(f[2])
        else:
            res["bm"][(int(f[1]), int(f[2]))] = int(f[3])
    return res


def test_buckets_halve_the_weight_from_2_to_the_20(rules):
    b = rules["bucket"]
    # bucket 0: 2^20 products and more; bucket q: [2^(20-q), 2^(21-q)); bucket 7: everything below 2^14
    assert b[1 << 40] == 0 and b[1048576] == 0
    assert b[1048575] == 1 and b[524288] == 1
    assert b[524287] == 2 and b[262144] == 2
    assert b[262143] == 3 and b[131072] == 3
    assert b[131071] == 4 and b[65536] == 4
    assert b[65535] == 5 and b[32768] == 5
    assert b[32767] == 6 and b[16384] == 6
    assert b[16383] == 7 and b[2] == 7 and b[1] == 7 and b[0] == 7
    # monotone: heavier items never land in a later bucket
    ws = sorted(b)
    assert all(b[x] >= b[y] for x, y in zip(ws, ws[1:]))


def test_bucket_weight_is_per_part(rules):
    # an item walks flop / parts products; parts 0 is taken as 1
    assert rules["bucketp"] == [1, 0, 2]


def test_symbolic_split_takes_one_part_per_32768_products(rules):
    s = rules["sym"]
    assert s[0] == 1 and s[32767] == 1 and s[65535] == 1     # below two parts' worth: whole
    assert s[65536] == 2 and s[98304] == 3 and s[131072] == 4
    assert s[32768 * 64] == 64 and s[32768 * 1000] == 64     # at most 64 parts


def test_numeric_split_keeps_8_products_per_entry_and_65536_per_part(rules):
    m = rules["bm"]
    assert m[(600000, 5000)] == 9          # unit max(65536, 8 * 5000) = 65536
    assert m[(600000, 100000)] == 1        # unit 800000 > flop: whole
    assert m[(131071, 1)] == 1 and m[(131072, 1)] == 2
    assert m[(1 << 40, 10)] == 64          # capped
