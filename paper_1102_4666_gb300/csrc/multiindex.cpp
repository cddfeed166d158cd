// multiindex.cpp -- multi-index sets of the polynomial basis (Section 3.2.2):
// total degree <= eta (p = binomial(d'+eta, eta)) or the hyperbolic set
// {nu : (sum nu_i^q)^{1/q} <= eta} of eq. hyper_set.  Order: total degree
// ascending, then lexicographically descending with the time variate first.
#include "multiindex.h"

#include <map>

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

// Chebyshev -> monomial map of a basis of total degree <= 3 or 4.  Monomials
// in the order constant, z_a, z_a z_b (a <= b), z_a z_b z_c (a <= b <= c)
// and, for a degree-4 basis, z_a z_b z_c z_e (a <= b <= c <= e), each group
// lexicographic.  T_1 = z, T_2 = 2 z^2 - 1, T_3 = 4 z^3 - 3 z,
// T_4 = 8 z^4 - 8 z^2 + 1.
int build_cheb_to_mono(const std::vector<std::vector<int>>& nus, int dp, int max_deg,
                       std::vector<int>& row, std::vector<int>& lidx, std::vector<double>& coef,
                       int& mono_deg) {
  int deg_max = 0;
  for (const auto& nu : nus) {
    int deg = 0;
    for (int e : nu) deg += e;
    if (deg > deg_max) deg_max = deg;
  }
  if (deg_max > max_deg || deg_max > 4) return -1;
  mono_deg = deg_max > 3 ? 4 : 3;
  // index of each sorted multiset of variates
  std::vector<std::vector<int>> monos;
  monos.push_back({});
  for (int a = 0; a < dp; ++a) monos.push_back({a});
  for (int a = 0; a < dp; ++a)
    for (int b = a; b < dp; ++b) monos.push_back({a, b});
  for (int a = 0; a < dp; ++a)
    for (int b = a; b < dp; ++b)
      for (int c = b; c < dp; ++c) monos.push_back({a, b, c});
  if (mono_deg == 4)
    for (int a = 0; a < dp; ++a)
      for (int b = a; b < dp; ++b)
        for (int c = b; c < dp; ++c)
          for (int e = c; e < dp; ++e) monos.push_back({a, b, c, e});
  const int pm = (int)monos.size();
  auto index_of = [&](const std::vector<int>& ms) {
    for (int m = 0; m < pm; ++m)
      if (monos[m] == ms) return m;
    return -1;
  };
  std::vector<std::vector<std::pair<int, double>>> rows(pm);
  // expansion of T_e as (power, coefficient)
  const std::vector<std::pair<int, double>> cheb[5] = {{{0, 1.0}},
                                                       {{1, 1.0}},
                                                       {{0, -1.0}, {2, 2.0}},
                                                       {{1, -3.0}, {3, 4.0}},
                                                       {{0, 1.0}, {2, -8.0}, {4, 8.0}}};
  for (size_t l = 0; l < nus.size(); ++l) {
    // cartesian product over the variates
    std::vector<std::pair<std::vector<int>, double>> terms = {{std::vector<int>(dp, 0), 1.0}};
    for (int v = 0; v < dp; ++v) {
      const int e = nus[l][v];
      if (e == 0) continue;
      std::vector<std::pair<std::vector<int>, double>> next;
      for (const auto& t : terms)
        for (const auto& pc : cheb[e]) {
          auto mu = t.first;
          mu[v] = pc.first;
          next.push_back({mu, t.second * pc.second});
        }
      terms.swap(next);
    }
    for (const auto& t : terms) {
      std::vector<int> ms;
      for (int v = 0; v < dp; ++v)
        for (int q = 0; q < t.first[v]; ++q) ms.push_back(v);
      const int m = index_of(ms);
      if (m < 0) return -1;
      rows[m].push_back({(int)l, t.second});
    }
  }
  row.assign(pm + 1, 0);
  lidx.clear();
  coef.clear();
  for (int m = 0; m < pm; ++m) {
    for (const auto& e : rows[m]) {
      lidx.push_back(e.first);
      coef.push_back(e.second);
    }
    row[m + 1] = (int)lidx.size();
  }
  return pm;
}

namespace {
// monomials of total degree <= deg as sorted variate lists, depth-first
void tree_monos(int dp, int deg, std::vector<int>& prefix, std::vector<std::vector<int>>& out) {
  out.push_back(prefix);
  if ((int)prefix.size() == deg) return;
  const int w = prefix.empty() ? 0 : prefix.back();
  for (int x = w; x < dp; ++x) {
    prefix.push_back(x);
    tree_monos(dp, deg, prefix, out);
    prefix.pop_back();
  }
}
}  // namespace

int build_cheb_to_mono_tree(const std::vector<std::vector<int>>& nus, int dp,
                            std::vector<int>& row, std::vector<int>& lidx,
                            std::vector<double>& coef, int& mono_deg) {
  int deg_max = 0;
  for (const auto& nu : nus) {
    int deg = 0;
    for (int e : nu) deg += e;
    if (deg > deg_max) deg_max = deg;
  }
  if (deg_max > 6) return -1;
  mono_deg = deg_max;
  std::vector<std::vector<int>> monos;
  std::vector<int> prefix;
  tree_monos(dp, deg_max, prefix, monos);
  const int pm = (int)monos.size();
  std::map<std::vector<int>, int> index;
  for (int m = 0; m < pm; ++m) index[monos[m]] = m;
  // T_e as (power, coefficient), from T_{e+1} = 2 z T_e - T_{e-1}
  std::vector<std::vector<double>> T(7);
  T[0] = {1.0};
  T[1] = {0.0, 1.0};
  for (int e = 1; e < 6; ++e) {
    std::vector<double> nxt(e + 2, 0.0);
    for (int q = 0; q <= e; ++q) nxt[q + 1] += 2.0 * T[e][q];
    for (int q = 0; q < (int)T[e - 1].size(); ++q) nxt[q] -= T[e - 1][q];
    T[e + 1] = nxt;
  }
  std::vector<std::vector<std::pair<int, double>>> rows(pm);
  for (size_t l = 0; l < nus.size(); ++l) {
    // cartesian product over the active variates of the powers of T_e
    std::vector<std::pair<std::vector<int>, double>> terms = {{std::vector<int>(dp, 0), 1.0}};
    for (int v = 0; v < dp; ++v) {
      const int e = nus[l][v];
      if (e == 0) continue;
      std::vector<std::pair<std::vector<int>, double>> next;
      for (const auto& t : terms)
        for (int q = 0; q <= e; ++q) {
          if (T[e][q] == 0.0) continue;
          auto mu = t.first;
          mu[v] = q;
          next.push_back({mu, t.second * T[e][q]});
        }
      terms.swap(next);
    }
    for (const auto& t : terms) {
      std::vector<int> ms;
      for (int v = 0; v < dp; ++v)
        for (int q = 0; q < t.first[v]; ++q) ms.push_back(v);
      const auto it = index.find(ms);
      if (it == index.end()) return -1;
      rows[it->second].push_back({(int)l, t.second});
    }
  }
  row.assign(pm + 1, 0);
  lidx.clear();
  coef.clear();
  for (int m = 0; m < pm; ++m) {
    for (const auto& e : rows[m]) {
      lidx.push_back(e.first);
      coef.push_back(e.second);
    }
    row[m + 1] = (int)lidx.size();
  }
  return pm;
}
