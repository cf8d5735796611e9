"""The time-tiled block order of the stencil kernels (grid_pos_tiled in csrc/common.cuh), compiled for
the host with nvcc and checked on the CPU: for every grid the launchers make (nsys x nby blocks) it is a
bijection onto the (system, block) pairs, so every site block of every system is computed exactly once
and no block addresses a system or block outside the grid; tile 0 is the plain systems-fastest order.
The time-blocked site map of a 128-thread block (site_of_block, same header) is checked the same way:
for slabs of a multiple of 4 slices and S3h % 32 == 0 the n/128 blocks cover the n sites once, a warp
stays in one time slice, and the four warps of a block take the same 32 positions of four
consecutive slices."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1612_06424_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <vector>
#include "common.cuh"
int main() {
  const int nsys_list[] = {1, 2, 3, 12, 24, 37};
  const int nby_list[] = {1, 2, 5, 16, 54, 432, 433, 1000};
  const int tb_list[] = {0, 1, 3, 16, 53, 54, 100, 431, 432, 2000};
  long long checked = 0;
  for (int nsys : nsys_list)
    for (int nby : nby_list)
      for (int tb : tb_list) {
        std::vector<char> seen((size_t)nsys * nby, 0);
        for (int bid = 0; bid < nsys * nby; bid++) {
          int s, by;
          lq::grid_pos_tiled(bid, nsys, nby, tb, s, by);
          if (s < 0 || s >= nsys || by < 0 || by >= nby) { printf("OUT %d %d %d %d\n", nsys, nby, tb, bid); return 1; }
          char& c = seen[(size_t)s * nby + by];
          if (c) { printf("DUP %d %d %d %d\n", nsys, nby, tb, bid); return 1; }
          c = 1;
          if (tb <= 0 && (s != bid % nsys || by != bid / nsys)) { printf("ORDER %d\n", bid); return 1; }
          checked++;
        }
      }
  const int s3h_list[] = {32, 64, 2048, 16384, 55296};
  const int nsl_list[] = {4, 8, 12, 44, 52, 96};
  for (int S3h : s3h_list)
    for (int nsl : nsl_list) {
      const int n = nsl * S3h;
      if ((long long)n > 6000000) continue;
      for (int tblk = 0; tblk < 2; tblk++) {
        std::vector<char> seen((size_t)n, 0);
        for (int by = 0; by < n / 128; by++)
          for (int t = 0; t < 128; t++) {
            const int j = lq::site_of_block(tblk, S3h, by, t);
            if (j < 0 || j >= n || seen[j]) { printf("SITE %d %d %d %d %d\n", S3h, nsl, tblk, by, t); return 1; }
            seen[j] = 1;
            const int j0 = lq::site_of_block(tblk, S3h, by, t & 96);
            if (tblk && (j / S3h != j0 / S3h || j - j0 != (t & 31))) { printf("WARP %d %d\n", by, t); return 1; }
            if (tblk && t >= 32 && j - lq::site_of_block(tblk, S3h, by, t - 32) != S3h) { printf("SLICE %d %d\n", by, t); return 1; }
            if (!tblk && j != by * 128 + t) { printf("PLAIN %d %d\n", by, t); return 1; }
            checked++;
          }
      }
    }
  printf("ok %lld\n", checked);
  return 0;
}
"""


def test_grid_order_and_site_map_are_bijections(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "grid.cu"
    src.write_text(HARNESS)
    exe = tmp_path / "grid"
    subprocess.run([nvcc, "-std=c++17", "-I", CSRC, "-o", str(exe), str(src)], check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout
