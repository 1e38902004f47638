"""The leaf tiles' register lists (csrc/rpf_select.cuh) on the host.

A batch merged in by insert8 / insert4 (sorting network, elementwise minimum
with the reversed batch, bitonic merge) must leave exactly the list that one
insert() per key leaves.  The header's functions are host-callable, so a small
host program built by nvcc checks every list length the kernels instantiate
on random keys, on keys with many repeats, and with empty (all-ones) keys
mixed in.  No GPU is needed."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1812_11689_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <random>
#include "rpf_select.cuh"

template <int KK> int check_u32(std::mt19937& g, int mode) {
  int bad = 0;
  for (int trial = 0; trial < 4000; ++trial) {
    TopU<KK> a, b;
    a.init();
    b.init();
    const int ncol = 8 * (1 + (int)(g() % 40));
    for (int c0 = 0; c0 < ncol; c0 += 8) {
      uint32_t kb[8];
      for (int j = 0; j < 8; ++j) {
        const int r = (int)(g() % 10);
        uint32_t x = mode == 0 ? (uint32_t)g() : (uint32_t)(g() % 64);
        if (r == 0) x = 0xffffffffu;
        if (r == 1) x = 0u;
        kb[j] = x;
        a.insert(x);
      }
      b.insert8(kb);
    }
    for (int q = 0; q < KK; ++q)
      if (a.v[q] != b.v[q]) { ++bad; break; }
  }
  return bad;
}

template <int KK> int check_u64(std::mt19937_64& g, int mode) {
  int bad = 0;
  for (int trial = 0; trial < 4000; ++trial) {
    Top64<KK> a, b;
    a.init();
    b.init();
    const int n = 1 + (int)(g() % 60);
    for (int c0 = 0; c0 < n; c0 += 4) {
      unsigned long long kb[4];
      for (int j = 0; j < 4; ++j) {
        unsigned long long x = mode == 0 ? g() : (((g() % 8) << 32) | (g() % 16));
        if (c0 + j >= n || g() % 10 == 0) x = ~0ull;
        kb[j] = x;
        if (x != ~0ull) a.insert(x);  // an empty key leaves the list as it is
      }
      b.insert4(kb);
    }
    for (int q = 0; q < KK; ++q)
      if (a.k[q] != b.k[q]) { ++bad; break; }
  }
  return bad;
}

int main() {
  std::mt19937 g(20181229);
  std::mt19937_64 g64(1812);
  int bad = 0;
  for (int mode = 0; mode < 2; ++mode) {
    // TopU<K + 2> for the tensor path's list lengths K in {4, 8, 10, 12, 16, 20, 24, 32}
    bad += check_u32<6>(g, mode) + check_u32<10>(g, mode) + check_u32<12>(g, mode) +
           check_u32<14>(g, mode) + check_u32<18>(g, mode) + check_u32<22>(g, mode) +
           check_u32<26>(g, mode) + check_u32<34>(g, mode);
    // Top64<K> for the re-rank and the plain tiles' list lengths
    bad += check_u64<4>(g64, mode) + check_u64<8>(g64, mode) + check_u64<10>(g64, mode) +
           check_u64<12>(g64, mode) + check_u64<16>(g64, mode) + check_u64<20>(g64, mode) +
           check_u64<24>(g64, mode) + check_u64<32>(g64, mode);
  }
  printf("mismatches %d\n", bad);
  return bad != 0;
}
"""


def _nvcc():
    cand = [shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"]
    for c in cand:
        if c and os.path.exists(c):
            return c
    return None


def test_batched_merges_keep_the_same_lists_as_single_insertions(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    src = tmp_path / "select_check.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "select_check"
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "-I", CSRC, "-o", str(exe), str(src)],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "mismatches 0" in r.stdout, r.stdout + r.stderr
