// Host-only C ABI over the octree / cone-segment setup (no CUDA calls).
#include <cstring>
#include <new>
#include <stdexcept>

#include "host_setup.h"

using namespace ifgf;

extern "C" {

ifgf_status ifgf_tree_create(const double* nodes, int32_t n, double leaf_size, int32_t min_levels,
                             double k_max, int32_t ns0, int32_t na0, int32_t max_leaf_pts, ifgf_tree* out) {
  if (!out) return IFGF_EINVAL;
  *out = nullptr;
  if (!nodes || n < 1 || !(leaf_size > 0) || !(k_max > 0) || ns0 < 1 || na0 < 1 || ns0 > 64 || na0 > 64 ||
      max_leaf_pts < 0 || max_leaf_pts > 1000000)
    return IFGF_EINVAL;
  ifgf_tree_t* t = new (std::nothrow) ifgf_tree_t();
  if (!t) return IFGF_ENOMEM;
  try {
    build_tree(*t, nodes, n, leaf_size, min_levels > 0 ? min_levels : 3, k_max, ns0, na0, max_leaf_pts);
  } catch (const std::bad_alloc&) {
    delete t;
    return IFGF_ENOMEM;
  } catch (const std::exception&) {
    delete t;
    return IFGF_EINVAL;
  }
  *out = t;
  return IFGF_OK;
}

ifgf_status ifgf_tree_destroy(ifgf_tree tree) {
  delete tree;
  return IFGF_OK;
}

ifgf_status ifgf_tree_info(ifgf_tree t, int32_t* levels, double* corner, double* h1) {
  if (!t) return IFGF_EINVAL;
  if (levels) *levels = t->D;
  if (corner) std::memcpy(corner, t->corner, sizeof(double) * 3);
  if (h1) *h1 = t->H1;
  return IFGF_OK;
}

ifgf_status ifgf_tree_perm(ifgf_tree t, int32_t* perm, int32_t* leaf_coords) {
  if (!t) return IFGF_EINVAL;
  const int n = (int)t->perm.size();
  if (perm)
    for (int s = 0; s < n; ++s) perm[s] = t->perm[s];
  if (leaf_coords)
    for (int l = 0; l < n; ++l)
      for (int k = 0; k < 3; ++k) leaf_coords[3 * l + k] = t->leafc[l][k];
  return IFGF_OK;
}

ifgf_status ifgf_tree_level(ifgf_tree t, int32_t d, int32_t* nboxes, int32_t* nslots, int32_t* ns, int32_t* na,
                            int32_t* box_coords, int32_t* box_slot_ptr, int64_t* slot_cone) {
  if (!t || d < 1 || d > t->D) return IFGF_EINVAL;
  const HostLevel& L = t->lv[d];
  if (nboxes) *nboxes = (int)L.key.size();
  if (nslots) *nslots = (int)L.slot_box.size();
  if (ns) *ns = L.ns;
  if (na) *na = L.na;
  if (box_coords)
    for (size_t b = 0; b < L.key.size(); ++b)
      for (int k = 0; k < 3; ++k) box_coords[3 * b + k] = L.ic[b][k];
  if (box_slot_ptr) {
    if (L.box_slot_ptr.empty())
      for (size_t b = 0; b <= L.key.size(); ++b) box_slot_ptr[b] = 0;
    else
      for (size_t b = 0; b <= L.key.size(); ++b) box_slot_ptr[b] = L.box_slot_ptr[b];
  }
  if (slot_cone)
    for (size_t s = 0; s < L.slot_cone.size(); ++s) slot_cone[s] = L.slot_cone[s];
  return IFGF_OK;
}

ifgf_status ifgf_tree_upward(ifgf_tree t, int32_t d, int64_t* ncompact, int32_t* up_cc, int32_t* up_order,
                             int64_t* ntask, int32_t* up_task, int32_t* up_task_ptr) {
  if (!t || d < 3 || d >= t->D) return IFGF_EINVAL;
  const HostLevel& L = t->lv[d];
  if (ncompact) *ncompact = (int64_t)L.upcone_list.size();
  if (ntask) *ntask = (int64_t)L.up_task.size();
  if (up_cc) std::memcpy(up_cc, L.up_cc.data(), sizeof(int32_t) * L.up_cc.size());
  if (up_order) std::memcpy(up_order, L.up_order.data(), sizeof(int32_t) * L.up_order.size());
  if (up_task) std::memcpy(up_task, L.up_task.data(), sizeof(int32_t) * L.up_task.size());
  if (up_task_ptr) std::memcpy(up_task_ptr, L.up_task_ptr.data(), sizeof(int32_t) * L.up_task_ptr.size());
  return IFGF_OK;
}

ifgf_status ifgf_tree_items(ifgf_tree t, int32_t d, int64_t* nitems, int32_t* items) {
  if (!t || d < 3 || d >= t->D) return IFGF_EINVAL;
  const HostLevel& L = t->lv[d];
  if (nitems) *nitems = (int64_t)(L.tc_item.size() / kTcBoxes);
  if (items) std::memcpy(items, L.tc_item.data(), sizeof(int32_t) * L.tc_item.size());
  return IFGF_OK;
}

ifgf_status ifgf_tree_targets(ifgf_tree t, int32_t d, int64_t* ninter, int64_t* tgt_ptr, int32_t* tgt_slot,
                              int32_t* slot_box) {
  if (!t || d < 3 || d > t->D) return IFGF_EINVAL;
  const HostLevel& L = t->lv[d];
  if (ninter) *ninter = (int64_t)L.tgt_slot.size();
  if (tgt_ptr)
    for (size_t s = 0; s < L.tgt_ptr.size(); ++s) tgt_ptr[s] = L.tgt_ptr[s];
  if (tgt_slot)
    for (size_t e = 0; e < L.tgt_slot.size(); ++e) tgt_slot[e] = L.tgt_slot[e];
  if (slot_box)
    for (size_t s = 0; s < L.slot_box.size(); ++s) slot_box[s] = L.slot_box[s];
  return IFGF_OK;
}

}  // extern "C"
