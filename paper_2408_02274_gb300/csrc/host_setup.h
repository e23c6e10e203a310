// Host setup entry points (see host_setup.cpp).
#pragma once
#include <vector>

#include "plan.h"

namespace ifgf {

cone_key cone_of(const ConeGeom& cg, double x, double y, double z);
void interp_point(const ConeGeom& cg, cone_key cone, int q, double* X);

// Octree, cone counts, relevant cones and target lists.  Throws std::invalid_argument.
// max_leaf_pts > 0: deepen the (uniform) octree until no leaf box holds more points.
void build_tree(HostTree& t, const double* x, int N, double leaf_size, int min_levels, double k_max,
                int ns0, int na0, int max_leaf_pts = 0);

// Candidate singular patches per target (node-distance filter of the singular set).
void near_candidates(const double* x, int P, int nc, double delta, std::vector<double>& gap,
                     std::vector<int64_t>& cptr, std::vector<int>& cpatch);

// Nonzeros of the near matrix if every candidate were singular (an upper bound on the
// structure near_structure builds from the closest-point test).
int64_t near_nnz_bound(const HostTree& t, int P, int nc, const std::vector<int64_t>& cptr,
                       const std::vector<int>& cpatch);

// CSR structure of the near matrix given which candidates are singular.
void near_structure(const HostTree& t, int P, int nc, const std::vector<int64_t>& cptr,
                    const std::vector<int>& cpatch, const std::vector<uint8_t>& singular,
                    std::vector<int64_t>& row_ptr, host_array<int>& col, host_array<int>& pair);

}  // namespace ifgf
