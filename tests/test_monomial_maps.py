"""The host-side Chebyshev -> monomial maps behind the dense evaluations of
the path kernel (degree-graded order up to degree 4, prefix-tree order up to
degree 6), checked on the CPU against the definition T_e(z) = cos(e arccos z):
for random Chebyshev coefficients alpha, the monomial coefficients beta the
map produces give the same polynomial at random points of [-1, 1]^{d+1}.
A small C++ program is compiled against csrc/multiindex.cpp with g++."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1102_4666_gb300", "csrc")

CHECK = r"""
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>
#include "multiindex.h"

static double cheb(int e, double z) { return std::cos(e * std::acos(z)); }

// monomial lists in the two orders the maps document
static void graded(int dp, int deg, std::vector<std::vector<int>>& out) {
  out.push_back({});
  for (int a = 0; a < dp; ++a) out.push_back({a});
  for (int a = 0; a < dp; ++a) for (int b = a; b < dp; ++b) out.push_back({a, b});
  for (int a = 0; a < dp; ++a) for (int b = a; b < dp; ++b) for (int c = b; c < dp; ++c)
    out.push_back({a, b, c});
  if (deg == 4)
    for (int a = 0; a < dp; ++a) for (int b = a; b < dp; ++b) for (int c = b; c < dp; ++c)
      for (int e = c; e < dp; ++e) out.push_back({a, b, c, e});
}
static void tree(int dp, int deg, std::vector<int>& pre, std::vector<std::vector<int>>& out) {
  out.push_back(pre);
  if ((int)pre.size() == deg) return;
  for (int x = pre.empty() ? 0 : pre.back(); x < dp; ++x) {
    pre.push_back(x);
    tree(dp, deg, pre, out);
    pre.pop_back();
  }
}

int main() {
  std::mt19937_64 rng(11);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  const int cases[][3] = {{1, 3, 0}, {5, 3, 0}, {10, 3, 0}, {2, 4, 0}, {5, 4, 0},
                          {1, 6, 1}, {2, 6, 1}, {5, 5, 1}, {5, 6, 1}, {10, 4, 1}, {3, 2, 1}};
  for (const auto& cs : cases) {
    const int d = cs[0], eta = cs[1], use_tree = cs[2], dp = d + 1;
    const auto nus = build_multi_indices(dp, eta, 1.0);
    std::vector<int> row, lidx;
    std::vector<double> coef;
    int md = 0;
    const int pm = use_tree ? build_cheb_to_mono_tree(nus, dp, row, lidx, coef, md)
                            : build_cheb_to_mono(nus, dp, 4, row, lidx, coef, md);
    std::vector<std::vector<int>> monos;
    std::vector<int> pre;
    if (use_tree) tree(dp, md, pre, monos); else graded(dp, md, monos);
    if (pm != (int)monos.size()) { printf("FAIL size d=%d eta=%d\n", d, eta); return 1; }
    std::vector<double> alpha(nus.size()), beta(pm, 0.0);
    for (auto& a : alpha) a = U(rng);
    for (int m = 0; m < pm; ++m)
      for (int q = row[m]; q < row[m + 1]; ++q) beta[m] += coef[q] * alpha[lidx[q]];
    double err = 0.0, scale = 0.0;
    for (int t = 0; t < 50; ++t) {
      std::vector<double> z(dp);
      for (auto& v : z) v = U(rng);
      double u1 = 0.0, u2 = 0.0;
      for (size_t l = 0; l < nus.size(); ++l) {
        double p = alpha[l];
        for (int v = 0; v < dp; ++v) p *= cheb(nus[l][v], z[v]);
        u1 += p;
      }
      for (int m = 0; m < pm; ++m) {
        double p = beta[m];
        for (int v : monos[m]) p *= z[v];
        u2 += p;
      }
      err = std::max(err, std::fabs(u1 - u2));
      scale = std::max(scale, std::fabs(u1));
    }
    printf("d=%d eta=%d tree=%d p=%zu pm=%d deg=%d err=%.3g scale=%.3g\n", d, eta, use_tree,
           nus.size(), pm, md, err, scale);
    if (!(err <= 1e-12 * std::max(1.0, scale))) { printf("FAIL\n"); return 1; }
  }
  // a degree above what each map handles is refused
  std::vector<int> row, lidx;
  std::vector<double> coef;
  int md = 0;
  if (build_cheb_to_mono(build_multi_indices(3, 5, 1.0), 3, 4, row, lidx, coef, md) != -1 ||
      build_cheb_to_mono_tree(build_multi_indices(2, 7, 1.0), 2, row, lidx, coef, md) != -1) {
    printf("FAIL refusal\n");
    return 1;
  }
  printf("OK\n");
  return 0;
}
"""


def test_chebyshev_to_monomial_maps_reproduce_the_polynomial(tmp_path):
    src = tmp_path / "check.cpp"
    exe = tmp_path / "check"
    src.write_text(CHECK)
    cc = subprocess.run(["g++", "-O2", "-std=c++17", "-I" + CSRC, str(src),
                         os.path.join(CSRC, "multiindex.cpp"), "-o", str(exe)],
                        capture_output=True, text=True)
    if cc.returncode != 0:
        pytest.fail(cc.stdout + cc.stderr)
    run = subprocess.run([str(exe)], capture_output=True, text=True)
    assert run.returncode == 0 and run.stdout.strip().endswith("OK"), run.stdout + run.stderr
