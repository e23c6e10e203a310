// Host setup entry points (see host_setup.cpp).
#pragma once
#include <memory>
#include <utility>
#include <vector>

#include "plan.h"

namespace ifgf {

// Allocator that leaves elements default-initialised (no zero fill) on resize: the near-matrix
// index arrays run to several GB and are written in parallel right after they are sized, so
// their pages are first touched by the threads that fill them.
template <typename T>
struct uninit_alloc : std::allocator<T> {
  template <typename U>
  struct rebind {
    using other = uninit_alloc<U>;
  };
  uninit_alloc() = default;
  template <typename U>
  uninit_alloc(const uninit_alloc<U>&) noexcept {}
  template <typename U>
  void construct(U* q) noexcept {
    ::new ((void*)q) U;
  }
  template <typename U, typename... A>
  void construct(U* q, A&&... a) {
    ::new ((void*)q) U(std::forward<A>(a)...);
  }
};
template <typename T>
using host_array = std::vector<T, uninit_alloc<T>>;

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
