"""Host-only launch-shape logic (association of a task, stacks of tasks on one
psi block), compiled with g++ against the planner sources: no CUDA, no GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2001_04890_gb300", "csrc")

PROG = r"""
#include "plan.hpp"
#include <cstdio>
#include <vector>
using namespace dmrg;

// multiply-adds of D += X Y Z in the two associations, counted by running the loops
static long count_normal(int m, int n, int p, int q) {
  long c = 0;
  for (int i = 0; i < m; ++i) for (int j = 0; j < p; ++j) for (int k = 0; k < n; ++k) ++c;  // T = X Y
  for (int i = 0; i < m; ++i) for (int l = 0; l < q; ++l) for (int j = 0; j < p; ++j) ++c;  // T Z
  return c;
}
static long count_transposed(int m, int n, int p, int q) {
  long c = 0;
  for (int l = 0; l < q; ++l) for (int k = 0; k < n; ++k) for (int j = 0; j < p; ++j) ++c;  // U = Z^T Y^T
  for (int l = 0; l < q; ++l) for (int i = 0; i < m; ++i) for (int k = 0; k < n; ++k) ++c;  // U X^T
  return c;
}

int main() {
  int fails = 0;
  for (int m = 1; m <= 7; ++m)
    for (int n = 1; n <= 7; ++n)
      for (int p = 1; p <= 7; ++p)
        for (int q = 1; q <= 7; ++q) {
          const bool want = count_transposed(m, n, p, q) < count_normal(m, n, p, q);
          if (prefer_transposed(m, n, p, q) != want) {
            std::printf("association m=%d n=%d p=%d q=%d\n", m, n, p, q);
            ++fails;
          }
        }
  struct Case { std::vector<uint64_t> keys; int cap; std::vector<int> runs; };
  const Case cases[] = {
      {{}, 4, {}},
      {{7}, 4, {1}},
      {{1, 1, 1, 2, 2, 3}, 8, {3, 2, 1}},
      {{1, 1, 1, 2, 2, 3}, 2, {2, 1, 2, 1}},
      {{5, 5, 5, 5, 5}, 1, {1, 1, 1, 1, 1}},
      {{5, 5, 5, 5, 5}, 0, {1, 1, 1, 1, 1}},
      {{1, 2, 3}, 8, {1, 1, 1}},
      {{9, 9, 9, 9, 9, 9, 9, 9, 9}, 8, {8, 1}},
  };
  for (const auto &c : cases) {
    const std::vector<int> got = stack_runs(c.keys, c.cap);
    if (got != c.runs) {
      std::printf("stack_runs case with %zu keys cap %d\n", c.keys.size(), c.cap);
      ++fails;
    }
    size_t total = 0;
    for (int r : got) total += r;
    if (total != c.keys.size()) ++fails;
  }
  std::printf("failures %d\n", fails);
  return fails == 0 ? 0 : 1;
}
"""


def test_launch_shape_host_logic(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    src = tmp_path / "host_logic.cpp"
    src.write_text(PROG)
    exe = tmp_path / "host_logic"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CSRC, str(src), os.path.join(CSRC, "plan.cpp"), "-o", str(exe)],
                   check=True, capture_output=True, timeout=300)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "failures 0" in out.stdout
