"""The shared-memory layouts of the tensor-core nucleon-block kernel (csrc/tc_layout.cuh), compiled for
the host with nvcc and checked exhaustively on the CPU:
* operands: for the 128-row A and the 256-row Bt of one K-step, every element (row r, K value q < 8) has
  its own 4-byte slot inside the operand's R * 32-byte block (a bijection onto the block), and the
  address the matrix descriptor forms from its leading / stride byte offsets (128, 256) is that slot;
  with the two byte offsets exchanged every address still lies inside the block, so a misread
  descriptor field could give wrong values but no access outside the operand;
* staging: the 56 spinor slots x 12 components of the 4 sites of a chunk map to distinct float2 words
  inside the staging array, the 16-byte accesses (even components) are 16-byte aligned, the 16-byte
  diquark reads of 8 consecutive j by a quarter warp fall on distinct banks, and the (k, alpha) reads
  of the Bt rows of a warp (16 distinct words) fall on distinct bank pairs."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1612_06424_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <vector>
#include "tc_layout.cuh"
using namespace lq;
int main() {
  const int rows[2] = {128, 256};
  for (int R : rows) {
    std::vector<char> seen(R * 8, 0);
    for (int r = 0; r < R; r++)
      for (int q = 0; q < 8; q++) {
        const int off = tc_operand_offset(r, q);
        if (off < 0 || off + 4 > R * 32 || off % 4) { printf("OUT %d %d %d\n", R, r, q); return 1; }
        if (seen[off / 4]++) { printf("DUP %d %d %d\n", R, r, q); return 1; }
        if (tc_desc_offset(r, q, TC_LBO, TC_SBO) != off) { printf("DESC %d %d %d\n", R, r, q); return 1; }
        const int sw = tc_desc_offset(r, q, TC_SBO, TC_LBO);
        if (sw < 0 || sw + 4 > R * 32) { printf("SWAP %d %d %d\n", R, r, q); return 1; }
      }
  }
  const int XS = 4, NSLOT = TC_TI + TC_TJ + TC_TK;
  std::vector<char> used(XS * TC_SITE_STG, 0);
  for (int x = 0; x < XS; x++)
    for (int slot = 0; slot < NSLOT; slot++)
      for (int comp = 0; comp < 12; comp++) {
        const int i = tc_stage_index(x, slot, comp);
        if (i < 0 || i >= XS * TC_SITE_STG) { printf("SOUT %d %d %d\n", x, slot, comp); return 1; }
        if (used[i]++) { printf("SDUP %d %d %d\n", x, slot, comp); return 1; }
        if (comp % 2 == 0 && i % 2) { printf("ALIGN %d %d %d\n", x, slot, comp); return 1; }
      }
  for (int x = 0; x < XS; x++)
    for (int e = 0; e < 6; e++)
      for (int j0 = 0; j0 < TC_TJ; j0 += 8) {
        int banks = 0;
        for (int jj = j0; jj < j0 + 8; jj++) {
          const int w = 2 * tc_stage_index(x, TC_TI + jj, 2 * e);
          for (int b = 0; b < 4; b++) {
            const int bit = 1 << ((w + b) % 32);
            if (banks & bit) { printf("BANK_A %d %d %d\n", x, e, jj); return 1; }
            banks |= bit;
          }
        }
      }
  for (int x = 0; x < XS; x++)
    for (int cc = 0; cc < 3; cc++)
      for (int k0 = 0; k0 < TC_TK; k0 += 4) {
        int banks = 0;
        for (int kk = k0; kk < k0 + 4; kk++)
          for (int al = 0; al < 4; al++) {
            const int w = 2 * tc_stage_index(x, TC_TI + TC_TJ + kk, al * 3 + cc);
            for (int b = 0; b < 2; b++) {
              const int bit = 1 << ((w + b) % 32);
              if (banks & bit) { printf("BANK_B %d %d %d %d\n", x, cc, kk, al); return 1; }
              banks |= bit;
            }
          }
      }
  printf("ok\n");
  return 0;
}
"""


def test_tensor_core_layouts(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "layout.cu"
    src.write_text(HARNESS)
    exe = tmp_path / "layout"
    subprocess.run([nvcc, "-std=c++17", "-I", CSRC, "-o", str(exe), str(src)], check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout
