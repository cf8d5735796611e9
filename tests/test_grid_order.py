"""The time-tiled block order of the stencil kernels (grid_pos_tiled in csrc/common.cuh), compiled for
the host with nvcc and checked on the CPU: for every grid the launchers make (nsys x nby blocks) it is a
bijection onto the (system, block) pairs, so every site block of every system is computed exactly once
and no block addresses a system or block outside the grid; tile 0 is the plain systems-fastest order."""
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
  printf("ok %lld\n", checked);
  return 0;
}
"""


def test_tiled_grid_order_is_a_bijection(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "grid.cu"
    src.write_text(HARNESS)
    exe = tmp_path / "grid"
    subprocess.run([nvcc, "-std=c++17", "-I", CSRC, "-o", str(exe), str(src)], check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout
