"""The bf16 slice planes' storage order against the tensor maps and the
tensor-core descriptors that read it, checked on the host.

A small host program is compiled against the library's own
`beor_common.cuh` (nvcc, no GPU needed) and checks, for planes of 128, 256
and 384 rows:

* `slice_elem_off` is a bijection of (row, col) onto the plane;
* reading a 4-D TMA box of the slice tensor map (256 contiguous elements x
  box_rows / 16 x one K-chunk, box order with x fastest) for every 128-row
  (A operand) and 64-row (B operand) block and every K-chunk places element
  (r, c) of the block at byte (r / 8) * 256 + ((c % 16) / 8) * 128 +
  (r % 8) * 16 + (c % 8) * 2 of the shared-memory image: the K-major layout
  without swizzle of 8-row x 16-byte core matrices, K halves 128 bytes apart
  (the descriptors' leading byte offset) and 8-row groups 256 bytes apart
  (their stride byte offset).
"""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2501_12928_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <vector>
#include "beor_common.cuh"

int main() {
  long long bad = 0;
  for (long long rows : {128LL, 256LL, 384LL}) {
    std::vector<int> seen((size_t)(rows * 128), 0);
    for (long long r = 0; r < rows; ++r)
      for (int c = 0; c < 128; ++c) {
        const long long o = slice_elem_off(r, c, rows);
        if (o < 0 || o >= rows * 128) { ++bad; continue; }
        ++seen[(size_t)o];
      }
    for (int s : seen) bad += s != 1;
    for (int box_rows : {128, 64})
      for (long long r0 = 0; r0 + box_rows <= rows; r0 += box_rows)
        for (int kc = 0; kc < 8; ++kc)
          for (long long r = r0; r < r0 + box_rows; ++r)
            for (int c = kc * 16; c < kc * 16 + 16; ++c) {
              // tensor map: element (x, y, z, w) at x + 256 y + rows*16 z + rows*128 w
              const long long within = slice_elem_off(r, c, rows) - (long long)kc * rows * 16;
              if (within < 0 || within >= rows * 16) { ++bad; continue; }
              const long long y = within / 256 - r0 / 16, x = within % 256;
              if (y < 0 || y >= box_rows / 16) { ++bad; continue; }
              const long long got = 2 * (y * 256 + x);
              const long long rr = r - r0, cc = c - kc * 16;
              const long long want = (rr / 8) * 256 + (cc / 8) * 128 + (rr % 8) * 16 + (cc % 8) * 2;
              bad += got != want;
            }
  }
  std::printf("mismatches %lld\n", bad);
  return bad != 0;
}
"""


def test_slice_planes_match_tma_boxes_and_core_matrices(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "layout.cu"
    exe = tmp_path / "layout"
    src.write_text(PROGRAM)
    subprocess.run([nvcc, "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True,
                   capture_output=True, timeout=300)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "mismatches 0" in r.stdout
