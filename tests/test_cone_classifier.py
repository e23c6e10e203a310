"""The host setup classifies cousin points and parent interpolation points into cone segments by
comparing cosines with a table of cell-boundary cosines (no atan2); it must give exactly the cells
of the atan2 definition (cone_of) for every input, with and without the previous point's cells as
hints.  This test compiles the host setup source into a small program (g++, CPU only) and compares
the two on random points, on coherent walks, and on points placed on and around the cell
boundaries, on the axis and on the plane y = 0, for the cone counts of every level of the
benchmark trees."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2408_02274_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <random>
#include "host_setup.cpp"
using namespace ifgf;
int main() {
  long bad = 0, n = 0;
  std::mt19937_64 rng(7);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  const int counts[][2] = {{4, 3}, {4, 6}, {8, 12}, {16, 24}, {32, 48}, {64, 96}, {128, 192}, {512, 768}, {2, 2}};
  for (auto& nc : counts) {
    ConeGeom cg{0.37, nc[0], nc[1]};
    ConeClassifier cls(cg);
    int h2 = -1, h3 = -1;   // hints carried from point to point, as in the octree's sweeps
    auto check = [&](double x, double y, double z) {
      ++n;
      const cone_key ref = cone_of(cg, x, y, z);
      if (cls(x, y, z) != ref) ++bad;
      if (cls(x, y, z, h2, h3) != ref) ++bad;
    };
    for (int i = 0; i < 2000000; ++i) check(U(rng), U(rng), U(rng));
    // coherent walks (consecutive points close together, crossing cell boundaries now and then)
    double w[3] = {0.3, -0.2, 0.5};
    for (int i = 0; i < 1000000; ++i) {
      for (double& v : w) v = std::min(1.0, std::max(-1.0, v + 1e-3 * U(rng)));
      check(w[0], w[1], w[2]);
    }
    // directions on and next to every theta and phi boundary, both signs of y, several radii
    const double eps[] = {0.0, 1e-16, -1e-16, 1e-14, -1e-14, 1e-12, -1e-12, 5e-12, -5e-12, 1e-9, -1e-9};
    for (int k = 0; k <= 2 * cg.na; ++k)
      for (double e : eps)
        for (double rad : {0.5, 1.0, 3.7}) {
          const double a = k * cg.dth() + e;
          check(rad * std::cos(a), rad * std::sin(a), 0.3);                  // phi boundary
          check(rad * std::cos(a), rad * std::sin(a), -1.1);
          if (k <= cg.na) {
            check(rad * std::sin(a) * 0.6, rad * std::sin(a) * 0.8, rad * std::cos(a));   // theta
            check(-rad * std::sin(a) * 0.28, rad * std::sin(a) * 0.96, rad * std::cos(a));
          }
        }
    for (double v : {0.0, -0.0, 1e-300, -1e-300, 1e-17, -1e-17, 0.5, -0.5}) {
      check(0.3, v, 0.2); check(-0.3, v, 0.2); check(v, 0.0, 0.7); check(v, -0.0, -0.7);
      check(0.0, 0.0, v); check(v, v, 1.0); check(1.0, v, v);
    }
    // radial cells: points at the radial boundaries
    for (int k = 0; k <= cg.ns; ++k)
      for (double e : eps) {
        const double s = k * cg.ds() + e;
        if (s > 0) check(0.2 * cg.h / s, 0.3 * cg.h / s, std::sqrt(1 - 0.13) * cg.h / s);
      }
  }
  printf("checked %ld mismatches %ld\n", n, bad);
  return bad != 0;
}
"""


def test_cosine_table_classifier_equals_the_atan2_cells(tmp_path):
    gxx = shutil.which("g++")
    inc = "/usr/local/cuda/include"
    if gxx is None or not os.path.exists(os.path.join(inc, "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers are missing")
    src = tmp_path / "classifier.cpp"
    exe = tmp_path / "classifier"
    src.write_text(PROGRAM)
    subprocess.check_call([gxx, "-O2", "-std=c++17", "-pthread", f"-I{inc}", f"-I{CSRC}", str(src), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "mismatches 0" in out.stdout
