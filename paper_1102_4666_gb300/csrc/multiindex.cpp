// multiindex.cpp -- multi-index sets of the polynomial basis (Section 3.2.2):
// total degree <= eta (p = binomial(d'+eta, eta)) or the hyperbolic set
// {nu : (sum nu_i^q)^{1/q} <= eta} of eq. hyper_set.  Order: total degree
// ascending, then lexicographically descending with the time variate first.
#include "multiindex.h"

#include <cmath>

namespace {

void compositions(int dp, int v, int remaining, std::vector<int>& cur,
                  std::vector<std::vector<int>>& out) {
  if (v == dp - 1) {
    cur[v] = remaining;
    out.push_back(cur);
    return;
  }
  for (int e = remaining; e >= 0; --e) {
    cur[v] = e;
    compositions(dp, v + 1, remaining - e, cur, out);
  }
}

}  // namespace

std::vector<std::vector<int>> build_multi_indices(int dp, int eta, double q) {
  std::vector<std::vector<int>> all;
  std::vector<int> cur(dp, 0);
  for (int deg = 0; deg <= eta; ++deg) compositions(dp, 0, deg, cur, all);
  if (q >= 1.0) return all;
  std::vector<std::vector<int>> kept;
  for (const auto& nu : all) {
    double s = 0.0;
    for (int e : nu)
      if (e > 0) s += std::pow((double)e, q);
    const double norm = s > 0.0 ? std::pow(s, 1.0 / q) : 0.0;
    if (norm <= (double)eta * (1.0 + 1e-9)) kept.push_back(nu);
  }
  return kept;
}

bool pack_multi_indices(const std::vector<std::vector<int>>& nus, std::vector<uint32_t>& pairs_xy,
                        std::vector<uint8_t>& nnz, int& max_deg) {
  pairs_xy.assign(2 * nus.size(), 0u);
  nnz.assign(nus.size(), 0);
  max_deg = 0;
  for (size_t l = 0; l < nus.size(); ++l) {
    int a = 0;
    for (int v = 0; v < (int)nus[l].size(); ++v) {
      const int e = nus[l][v];
      if (e == 0) continue;
      if (v > 15 || e > 15 || a >= 8) return false;
      const uint32_t byte = ((uint32_t)v << 4) | (uint32_t)e;
      if (a < 4)
        pairs_xy[2 * l] |= byte << (8 * a);
      else
        pairs_xy[2 * l + 1] |= byte << (8 * (a - 4));
      if (e > max_deg) max_deg = e;
      ++a;
    }
    nnz[l] = (uint8_t)a;
  }
  return true;
}
