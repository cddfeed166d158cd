// multiindex.h -- host-side multi-index sets of the polynomial basis.
#pragma once
#include <stdint.h>

#include <vector>

// multi-indices in N^dp with total degree <= eta (q >= 1) or hyperbolic
// pseudo-norm <= eta (q < 1), graded, lexicographically descending
std::vector<std::vector<int>> build_multi_indices(int dp, int eta, double q);

// pack each multi-index as (variate << 4 | degree) bytes in increasing
// variate order, two 32-bit words per basis function; false when a variate
// or degree exceeds 15 or more than 8 variates are active
bool pack_multi_indices(const std::vector<std::vector<int>>& nus, std::vector<uint32_t>& pairs_xy,
                        std::vector<uint8_t>& nnz, int& max_deg);

// Chebyshev -> monomial map (CSR by monomial) of a basis of total degree
// deg <= max_deg (max_deg <= 4), deg the largest total degree in the basis;
// the monomials are those of total degree <= max(deg, 3).  Returns their
// number, C(dp + 3, 3) or C(dp + 4, 4), and sets mono_deg to 3 or 4; -1
// when a basis function has a degree above max_deg
int build_cheb_to_mono(const std::vector<std::vector<int>>& nus, int dp, int max_deg,
                       std::vector<int>& row, std::vector<int>& lidx, std::vector<double>& coef,
                       int& mono_deg);

// The same map for a basis of total degree deg <= 6 onto all monomials of
// total degree <= deg, in the depth-first pre-order of the prefix tree of
// sorted variate multisets (root = constant; the children of a multiset
// ending with variate w append a variate x >= w): the order in which the
// generic dense evaluation of the path kernel visits them.  Returns the
// number of monomials C(dp + deg, deg) and sets mono_deg = deg; -1 when deg
// is above 6.
int build_cheb_to_mono_tree(const std::vector<std::vector<int>>& nus, int dp,
                            std::vector<int>& row, std::vector<int>& lidx,
                            std::vector<double>& coef, int& mono_deg);
