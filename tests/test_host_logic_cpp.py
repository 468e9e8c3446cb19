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


EIG_PROG = r"""
#include "plan.hpp"
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>
using namespace dmrg;

// Q diag(lambda) Q^T with Q a product of random plane rotations: eigenvalues known exactly
int main() {
  std::mt19937_64 g(7);
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  int fails = 0;
  for (int n = 1; n <= 16; ++n)
    for (int rep = 0; rep < 20; ++rep) {
      std::vector<double> lam(n), A(n * n, 0.0);
      for (int i = 0; i < n; ++i) lam[i] = (rep % 3 == 0 && i % 2) ? lam[i - 1] : u(g);  // some exact ties
      for (int i = 0; i < n; ++i) A[i * n + i] = lam[i];
      for (int r = 0; r < 3 * n; ++r) {
        int p = (int)(g() % n), q = (int)(g() % n);
        if (p == q) continue;
        const double t = u(g) * 3.14159, c = std::cos(t), s = std::sin(t);
        for (int k = 0; k < n; ++k) {  // A <- G A G^T
          const double a = A[p * n + k], b = A[q * n + k];
          A[p * n + k] = c * a - s * b;
          A[q * n + k] = s * a + c * b;
        }
        for (int k = 0; k < n; ++k) {
          const double a = A[k * n + p], b = A[k * n + q];
          A[k * n + p] = c * a - s * b;
          A[k * n + q] = s * a + c * b;
        }
      }
      std::vector<double> ev(n);
      small_symmetric_eigenvalues(n, A.data(), ev.data());
      std::sort(lam.begin(), lam.end());
      for (int i = 0; i < n; ++i)
        if (std::fabs(ev[i] - lam[i]) > 1e-12) {
          std::printf("n=%d rep=%d i=%d %.17g vs %.17g\n", n, rep, i, ev[i], lam[i]);
          ++fails;
        }
    }
  // entropies of a product pair state: pure, all zero; of the maximally mixed pair: ln 4, ln 4, ln 16
  double rho[256] = {0};
  rho[(4 * 1 + 2) * 17] = 1.0;
  double s[3];
  orbital_entropies(rho, s);
  if (std::fabs(s[0]) + std::fabs(s[1]) + std::fabs(s[2]) > 1e-15) ++fails;
  for (int i = 0; i < 256; ++i) rho[i] = 0.0;
  for (int i = 0; i < 16; ++i) rho[i * 17] = 1.0 / 16;
  orbital_entropies(rho, s);
  if (std::fabs(s[0] - std::log(4.0)) > 1e-14 || std::fabs(s[1] - std::log(4.0)) > 1e-14 ||
      std::fabs(s[2] - std::log(16.0)) > 1e-14)
    ++fails;
  std::printf("failures %d\n", fails);
  return fails == 0 ? 0 : 1;
}
"""


def test_small_eigensolver_and_entropy_limits_under_sanitizers(tmp_path):
    """The Jacobi eigensolver behind the two-orbital entropy on matrices with known
    spectra (ties included), and the entropy limits of a product and of a maximally
    mixed pair; built with address and undefined-behaviour checks."""
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    src = tmp_path / "eig.cpp"
    src.write_text(EIG_PROG)
    exe = tmp_path / "eig"
    flags = ["-std=c++17", "-O1", "-pthread", "-fsanitize=address,undefined", "-fno-sanitize-recover=all"]
    r = subprocess.run([gxx, *flags, "-I", CSRC, str(src), os.path.join(CSRC, "plan.cpp"), "-o", str(exe)],
                       capture_output=True, text=True, timeout=600)
    if r.returncode != 0 and "sanitize" in r.stderr:
        flags = ["-std=c++17", "-O1", "-pthread"]
        subprocess.run([gxx, *flags, "-I", CSRC, str(src), os.path.join(CSRC, "plan.cpp"), "-o", str(exe)],
                       check=True, capture_output=True, timeout=600)
    else:
        assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120,
                         env={**os.environ, "ASAN_OPTIONS": "detect_leaks=0"})
    assert out.returncode == 0, out.stdout + out.stderr
    assert "failures 0" in out.stdout
