"""The bf16 slice planes' storage order against the tensor maps and the
tensor-core descriptors that read it, and the slice GEMM's product schedule,
checked on the host.

A small host program is compiled against the library's own
`beor_common.cuh` (nvcc, no GPU needed) and checks, for planes of 128, 256
and 384 rows:

* `slice_elem_off` is a bijection of (row, col) onto the plane;
* reading a 5-D TMA box of the slice tensor map (256 contiguous elements x
  box_rows / 16 x one K-chunk x parts x 5 slices, box order with x fastest)
  places element (r, c) of part p of slice s where the tensor-core
  descriptors read it: for the A operand (one part, 128 rows) at
  s * 4096 + core(r, c), for the B window (two parts, 64 rows) at row
  n = (s - t0) * 128 + (p - p0) * 64 + r of a descriptor starting at window
  slice t0, i.e. t0 * 4096 + core(n, c), where core(r, c) =
  (r / 8) * 256 + ((c % 16) / 8) * 128 + (r % 8) * 16 + (c % 8) * 2 is the
  K-major layout without swizzle of 8-row x 16-byte core matrices (K halves
  128 bytes apart, 8-row groups 256 bytes apart).

A second program emulates the schedule of tensor-core products
(`slice_mma_*`, two half-stages per K-chunk: part Im of A with the window
(Im, Re), part Re with (Re, -Im)) on integer digits and checks that every
level's [re | im] accumulator pair equals the complex product
sum over the pairs (s, t) of the level of A_s B_t^H (level min(s + t, 3)),
for the full pair set (s + t <= 4), the reduced one (s + t <= 3 and (2, 2),
slice 4 unread) and the seven-slice set of the precompute (s + t <= 6),
with the first products of a tile overwriting and every later one
accumulating.
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

static long long core(long long r, long long c) { return (r / 8) * 256 + ((c % 16) / 8) * 128 + (r % 8) * 16 + (c % 8) * 2; }

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
    // A operand: 128 rows, one part p; B window: 64 rows, parts p0, p0 + 1
    for (int box_rows : {128, 64}) {
      const int nparts = box_rows == 128 ? 1 : 2;
      for (int p0 = 0; p0 + nparts <= BEOR_NPART; ++p0)
        for (long long r0 = 0; r0 + box_rows <= rows; r0 += box_rows)
          for (int kc = 0; kc < 8; ++kc)
            for (int sl = 0; sl < BEOR_NSLICE; ++sl)
              for (int pt = p0; pt < p0 + nparts; ++pt)
                for (long long r = r0; r < r0 + box_rows; ++r)
                  for (int c = kc * 16; c < kc * 16 + 16; ++c) {
                    // the element's place in the plane buffer, decomposed by the
                    // tensor map's strides (elements): x + 256 y + rows*16 z +
                    // rows*128 part + rows*128*3 slice
                    const long long g = (long long)slice_plane(sl, pt) * rows * 128 + slice_elem_off(r, c, rows);
                    const long long gs = g / (rows * 128 * BEOR_NPART), g1 = g % (rows * 128 * BEOR_NPART);
                    const long long gp = g1 / (rows * 128), g2 = g1 % (rows * 128);
                    const long long gz = g2 / (rows * 16), g3 = g2 % (rows * 16);
                    if (gs != sl || gp != pt || gz != kc) { ++bad; continue; }
                    const long long y = g3 / 256 - r0 / 16, x = g3 % 256;
                    if (y < 0 || y >= box_rows / 16) { ++bad; continue; }
                    // box order: x fastest, then y, the K-chunk (1), the part, the slice
                    const long long got = 2 * ((((long long)sl * nparts + (pt - p0)) * (box_rows / 16) + y) * 256 + x);
                    const long long rr = r - r0, cc = c - kc * 16;
                    if (nparts == 1) {
                      bad += got != sl * 4096 + core(rr, cc);
                    } else {
                      for (int t0 = 0; t0 <= sl; t0 += 2) {
                        const long long n = (long long)(sl - t0) * 128 + (pt - p0) * 64 + rr;
                        bad += got != (long long)t0 * 4096 + core(n, cc);
                      }
                    }
                  }
    }
  }
  std::printf("mismatches %lld\n", bad);
  return bad != 0;
}
"""

SCHEDULE = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "beor_common.cuh"

// Integer digits: A (m rows), B (64 rows), K = 3, real and imaginary parts
// of ns slices; one pair set.  TMEM emulation: m lanes x 512 columns.
static long long check(int ns, int set, int* nmma) {
  const int m = 4, nb = 64, K = 3;
  std::vector<long long> A(2 * ns * m * K), Bd(2 * ns * nb * K);   // [part 0 re, 1 im][slice][row][k]
  auto a = [&](int p, int s, int r, int k) -> long long& { return A[((p * ns + s) * m + r) * K + k]; };
  auto b = [&](int p, int s, int r, int k) -> long long& { return Bd[((p * ns + s) * nb + r) * K + k]; };
  for (int p = 0; p < 2; ++p)
    for (int s = 0; s < ns; ++s) {
      for (int r = 0; r < m; ++r) for (int k = 0; k < K; ++k) a(p, s, r, k) = rand() % 257 - 128;
      for (int r = 0; r < nb; ++r) for (int k = 0; k < K; ++k) b(p, s, r, k) = rand() % 257 - 128;
    }
  auto in_set = [&](int s, int t) {
    if (set == SLICE_PAIRS_REDUCED) return s + t <= 3 || (s == 2 && t == 2);
    if (set == SLICE_PAIRS_FULL5) return s + t <= 4;
    return s + t <= 6;
  };
  // B planes in the library's part order
  auto bplane = [&](int s, int part, int r, int k) -> long long {
    if (part == BEOR_PART_RE) return b(0, s, r, k);
    if (part == BEOR_PART_IM) return b(1, s, r, k);
    if (part == BEOR_PART_NEGIM) return -b(1, s, r, k);
    return 1LL << 40;
  };
  std::vector<long long> T((size_t)m * 512, 777);   // stale contents must be overwritten
  std::vector<int> written(512, 0);
  long long bad = 0;
  *nmma = 0;
  for (int sa = 0; sa < ns; ++sa) *nmma += slice_mma_count(sa, set);
  for (int kc = 0; kc < 2; ++kc)
    for (int h = 0; h < 2; ++h) {
      const int apart = h == 0 ? 1 : 0;            // half-stage 0: A part Im, 1: A part Re
      const int p0 = h == 0 ? BEOR_PART_IM : BEOR_PART_RE;
      for (int sa = 0; sa < ns; ++sa)
        for (int q = 0; q < slice_mma_count(sa, set); ++q) {
          const bool acc = !(kc == 0 && h == 0 && sa == 0 && q < slice_mma_main(0));
          const int col = slice_mma_col(sa, q), t0 = slice_mma_t(sa, q, set), n = slice_mma_n(sa, q);
          if (col + n > 512 || n % 128 || n > 256 || n < 128) ++bad;
          for (int j = 0; j < n; ++j) {
            const int t = t0 + j / 128, part = p0 + (j / 64) % 2, br = j % 64;
            if (t >= ns || !in_set(sa, t)) { ++bad; continue; }
            if (!acc) written[col + j] = 1;
            else if (!written[col + j]) ++bad;           // accumulating into a column never overwritten
            for (int r = 0; r < m; ++r) {
              long long v = 0;
              for (int k = 0; k < K; ++k) v += a(apart, sa, r, k) * bplane(t, part, br, k);
              long long& d = T[(size_t)r * 512 + col + j];
              d = acc ? d + v : v;
            }
          }
        }
    }
  // expected: level l, re = sum Ar Br + Ai Bi, im = sum Ai Br - Ar Bi over the set's pairs of
  // the level (twice: two K-chunks of the same data); every pair of the set is covered once
  for (int l = 0; l < 4; ++l)
    for (int r = 0; r < m; ++r)
      for (int c = 0; c < nb; ++c) {
        long long re = 0, im = 0;
        for (int s = 0; s < ns; ++s)
          for (int t = 0; t < ns; ++t) {
            if (!in_set(s, t) || (s + t < 3 ? s + t : 3) != l) continue;
            for (int k = 0; k < K; ++k) {
              re += a(0, s, r, k) * b(0, t, c, k) + a(1, s, r, k) * b(1, t, c, k);
              im += a(1, s, r, k) * b(0, t, c, k) - a(0, s, r, k) * b(1, t, c, k);
            }
          }
        bad += T[(size_t)r * 512 + 128 * l + c] != 2 * re;
        bad += T[(size_t)r * 512 + 128 * l + 64 + c] != 2 * im;
      }
  return bad;
}

int main() {
  srand(7);
  int n5 = 0, nr = 0, n7 = 0;
  long long bad = check(5, SLICE_PAIRS_FULL5, &n5) + check(5, SLICE_PAIRS_REDUCED, &nr) +
                  check(7, SLICE_PAIRS_FULL7, &n7);
  std::printf("mismatches %lld products per half-stage %d (full) %d (reduced) %d (7 slices)\n", bad, n5, nr, n7);
  return bad != 0;
}
"""


def _build_run(tmp_path, name, text):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / f"{name}.cu"
    exe = tmp_path / name
    src.write_text(text)
    subprocess.run([nvcc, "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True,
                   capture_output=True, timeout=300)
    return subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)


def test_slice_planes_match_tma_boxes_and_core_matrices(tmp_path):
    r = _build_run(tmp_path, "layout", PROGRAM)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "mismatches 0" in r.stdout


def test_product_schedule_gives_each_level_its_complex_product(tmp_path):
    r = _build_run(tmp_path, "schedule", SCHEDULE)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "mismatches 0 products per half-stage 11 (full) 7 (reduced) 24 (7 slices)" in r.stdout
