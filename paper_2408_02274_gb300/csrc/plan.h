// Internal plan layout of the CBIE-IFGF library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <memory>
#include <string>
#include <unordered_map>
#include <utility>
#include <vector>

#include "../../include/ifgf.h"
#include "common.cuh"

namespace ifgf {

// ------------------------------------------------------------------ host octree
// Allocator that leaves elements default-initialised (no zero fill) on resize: the host
// setup's large index arrays (cone records, target slots, near-matrix columns; up to several
// GB) are written in parallel right after they are sized, so their pages are first touched by
// the threads that fill them.
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

struct HostLevel {
  int d = 0;
  double H = 0, h = 0;
  int ns = 0, na = 0;
  std::vector<uint64_t> key;                  // Morton key per relevant box
  std::vector<std::array<int, 3>> ic;         // integer box coordinates
  std::vector<int> pt_begin, pt_end;          // sorted point range per box
  std::vector<int> parent;                    // box index at level d-1
  std::vector<std::array<int, 8>> child;      // box index at level d+1 (-1 absent)
  std::unordered_map<uint64_t, int> index;    // key -> box
  std::vector<std::vector<int>> nbr;          // neighbours (incl. self), Eq. box_neighbor
  std::vector<std::vector<int>> cousin;       // cousins, Eq. box_cousin
  // slots (relevant cones, sorted by box then cone)
  std::vector<int> slot_box, box_slot_ptr;
  std::vector<cone_key> slot_cone;
  // compact list of this level's relevant cone keys (sorted, distinct)
  std::vector<cone_key> upcone_list;          // compact -> cone key
  std::vector<int> slot_upidx;                // slot -> compact index
  std::vector<int> cmap;                      // [nboxes][ncompact] -> slot or -1 (levels >= 4)
  // this level as a parent of level d+1
  std::vector<int32_t> up_cc;                 // [ncompact][8][75] child cone, compact index at d+1
  std::vector<int32_t> up_order;              // [ncompact][8][75] points ranked by (group, child cone)
  std::vector<int32_t> up_task;               // runs start | len << 8 | octant << 16, per (cone, group)
  std::vector<int32_t> up_task_ptr;           // [ncompact * kUpGroups + 1] CSR offsets into up_task
  // the same step on the tensor cores: per (compact cone, octant) the points ranked by child cone,
  // units of at most kUpRunMax of them sharing one child cone (start | len << 8 | octant << 16,
  // CSR per compact cone), and groups of up to kTcBoxes slots of one compact cone (-1 padded)
  std::vector<int32_t> tc_order;              // [ncompact][8][75]
  std::vector<int32_t> tc_unit;
  std::vector<int32_t> tc_unit_ptr;           // [ncompact + 1]
  std::vector<int32_t> tc_item;               // [nitems][kTcBoxes]
  int tc_max_units = 0;                       // most units of one compact cone
  // target evaluation lists at this level: per sorted target, its slots
  std::vector<int64_t> tgt_ptr;
  host_array<int32_t> tgt_slot;
  std::vector<int32_t> tgt_chunk;             // (first sorted target, count <= 32) per chunk of a box with cousins
  ConeGeom cg() const { return ConeGeom{h, ns, na}; }
};

struct HostTree {
  int D = 0;
  double corner[3] = {0, 0, 0};
  double H1 = 0;
  std::vector<int> perm;                      // sorted -> original
  std::vector<int> iperm;                     // original -> sorted
  std::vector<std::array<int, 3>> leafc;      // per original node: integer leaf coordinates
  std::vector<std::vector<int>> box_of;       // [d][sorted point] -> box index at level d
  std::vector<HostLevel> lv;                  // index d = 0..D (0 unused)
};

// ------------------------------------------------------------------ device level tables
struct DevLevel {
  int d = 0, nboxes = 0, nslots = 0;
  int max_box_slots = 0;          // largest number of relevant cones of one box
  ConeGeom cg{};
  double H = 0;
  double* box_center = nullptr;   // [nboxes][3]
  int* cmap = nullptr;            // [nboxes][ncomp] -> slot or -1 (levels >= 4)
  int ncomp = 0;                  // distinct relevant cones of the level
  cone_key* ckeys = nullptr;      // [ncomp] compact index -> cone key
  int* slot_box = nullptr;        // [nslots]
  cone_key* slot_cone = nullptr;  // [nslots]
  int* box_slot_ptr = nullptr;    // [nboxes+1]
  int* box_pt_ptr = nullptr;      // [nboxes+1] sorted point ranges
  int* child = nullptr;           // [nboxes][8] boxes at level d+1
  int* slot_upidx = nullptr;      // [nslots] compact cone index (as parent)
  int* up_cc = nullptr;           // [ncompact][8][75]
  int* up_order = nullptr;        // [ncompact][8][75]
  int* up_task = nullptr;         // runs per (compact cone, group)
  int* up_task_ptr = nullptr;     // [ncompact * kUpGroups + 1]
  int* tc_order = nullptr;        // [ncompact][8][75]
  int* tc_unit = nullptr;         // units per compact cone
  int* tc_unit_ptr = nullptr;     // [ncompact + 1]
  int* tc_item = nullptr;         // [ntc_items][kTcBoxes]
  int ntc_items = 0;
  bool tc = false;                // the upward step into this level runs on the tensor cores
  int leaf_mode = 1;              // FP32 leaf step (level D): 0 SIMT products, 1 tensor-pipe products
  int up_mode = 0;                // FP32 SIMT upward step into this level: 0 runs per point group,
                                  // 1 a warp per parent slot over the unit tables
  int64_t* tgt_ptr = nullptr;     // [N+1]
  int* tgt_slot = nullptr;        // [ninter]
  double2* trig_th = nullptr;     // [na] (cos, sin) of g2 * pi / na: lower edges of the theta cells
  double2* trig_ph = nullptr;     // [2 na] (cos, sin) of g3 * pi / na: lower edges of the phi cells
  int64_t ninter = 0;
  int2* tgt_chunk = nullptr;      // [ntgt_chunks] (first sorted target, count <= 32), targets of one box
  int ntgt_chunks = 0;
  int tgt_mode = 0;               // FP32 target step at this level: 0 warp per target, 1 warp per box chunk
  void* coefs = nullptr;          // [batch][nslots][75][C] real (precision of the plan), C = 32, or
                                  // 2 x fields_per_pass for a plan of fewer fields per pass; one buffer
                                  // serves all levels of equal parity (two live levels at a time)
  size_t cstride = 0;             // nslots * 75 * C: coefficients per right-hand side
  float* img = nullptr;           // [batch][nslots][2][32 x 80] tensor-core operand images (hi, lo) of the
                                  // coefficients, when the upward step into level d-1 runs on the tensor
                                  // cores; one buffer per parity of d, like coefs
  size_t istride = 0;             // nslots * 5120: images per right-hand side
};

struct NodeGeom {           // per-node geometry, original order (FP64 SoA)
  double* x = nullptr;      // [N][3]
  double* xu = nullptr;     // [N][3]
  double* xv = nullptr;     // [N][3]
  double* n = nullptr;      // [N][3]
  double* t1 = nullptr;     // [N][3]
  double* t2 = nullptr;     // [N][3]
  double* J = nullptr;      // [N]
  double* w = nullptr;      // [N] quadrature weight J w_i w_j
  double* g = nullptr;      // [N][3] inverse metric (g^uu, g^uv, g^vv)
};

struct NearMatrix {
  int64_t nnz = 0;
  int64_t* row_ptr = nullptr;   // [N+1]
  int* col = nullptr;           // [nnz]
  double* val64 = nullptr;      // [nnz][4][2] (S_e, S_i, D_e, D_i)
  float* val32 = nullptr;       // [nnz][4][2]
};

struct GmresWork {               // per right-hand side r < batch (layouts below)
  int max_iter = 0;
  double* V = nullptr;          // [max_iter+1][nrhs][4N][2] Krylov basis (k-major)
  double* H = nullptr;          // [batch][max_iter+1][max_iter+1][2]
  double* cs = nullptr;         // [batch][max_iter+1][2]
  double* sn = nullptr;         // [batch][max_iter+1][2]
  double* g = nullptr;          // [batch][max_iter+1][2]
  double* h = nullptr;          // [batch][2][max_iter+1][2] projections (total, pass)
  double* part = nullptr;       // [batch][nblk][max_iter+1][2] partial dot products
  double* scal = nullptr;       // [batch][8]: |b|, beta, residual estimate
  double* w = nullptr;          // [batch][4N][2]
  double* b = nullptr;          // [batch][4N][2]
  double* y = nullptr;          // [batch][4N][2]
  double* inc = nullptr;        // [batch][6N][2]
  double* y_acc = nullptr;      // [batch][4N][2] refinement: the solution so far (refine > 0)
  double* b_orig = nullptr;     // [batch][4N][2] refinement: the right-hand side (refine > 0)
  int* active = nullptr;        // [batch] 1 while a right-hand side iterates
  int* kfin = nullptr;          // [batch] Krylov dimension at the end
  double* hres = nullptr;       // pinned host copy of scal
  int* hactive = nullptr;       // pinned host [batch]
  int* hk = nullptr;            // pinned host [batch]
};

// Learned right preconditioner: per-patch two-layer network (precond.cu).
struct TrainWork {              // minibatch scratch, allocated by the first training call
  int batch = 0;
  float *Xb = nullptr, *Tb = nullptr, *Hpre = nullptr, *H1 = nullptr, *Y = nullptr, *dY = nullptr, *dH = nullptr;
  float *gW1 = nullptr, *gb1 = nullptr, *gW2 = nullptr, *gb2 = nullptr;
  float *mW1 = nullptr, *vW1 = nullptr, *mb1 = nullptr, *vb1 = nullptr;   // Adam moments
  float *mW2 = nullptr, *vW2 = nullptr, *mb2 = nullptr, *vb2 = nullptr;
};
struct Precond {
  int hidden = 0, in = 0;       // in = 8 Nc^2 real features per patch
  int adam_t = 0;
  float *W1 = nullptr, *b1 = nullptr, *W2 = nullptr, *b2 = nullptr;   // FP32 master weights [in][H], [H], [H][in], [in]
  void *W1h = nullptr, *W2h = nullptr;   // BF16 copies used when applying the preconditioner
  double* Z = nullptr;          // flexible GMRES basis [max_iter+1][batch][4N][2]
  float* loss = nullptr;        // training losses of the last call (device)
  int loss_cap = 0;
  TrainWork tw;
};

// Block-Jacobi right preconditioner: inverses of the diagonal blocks (blockjacobi.cu).
struct BlockJacobi {
  int m = 0;                    // 4 Nc^2 unknowns per patch
  double* inv = nullptr;        // [P][m][m] complex128, row-major; null until built
};

// Per-kernel-kind CUDA-event timing of the per-apply work (optional).
enum TimedKind { TK_PREP = 0, TK_NEAR, TK_LEAF, TK_UP, TK_TARGET, TK_COMBINE, TK_FAR_DIRECT, TK_GMRES, TK_COUNT };
struct KernelTimer {
  bool on = false;
  std::vector<cudaEvent_t> pool;   // 2 events per record
  std::vector<int> kind;           // kind of each pending record
  int npending = 0;
  double total_ms[TK_COUNT] = {};
  int64_t calls[TK_COUNT] = {};
};

}  // namespace ifgf

struct ifgf_tree_t : ifgf::HostTree {};

namespace ifgf {
// Storage and arithmetic of the densities, near matrix, fields and combination: FP64 in the FP64
// and mixed plans.  The IFGF kernels (leaf, upward, target) run in FP64 only in the FP64 plan.
inline bool store64(const ifgf_plan_desc& d) { return d.precision != IFGF_FP32; }
inline bool ifgf64(const ifgf_plan_desc& d) { return d.precision == IFGF_FP64; }
// Fewer than all 16 IFGF fields per octree traversal (fields_per_pass 1 or 8), and the real
// columns of one cone segment's coefficient rows: 2 per complex field carried.
inline bool narrow_passes(const ifgf_plan_desc& d) { return d.fields_per_pass == 1 || d.fields_per_pass == 8; }
inline int coef_columns(const ifgf_plan_desc& d) { return narrow_passes(d) ? 2 * d.fields_per_pass : 32; }
}  // namespace ifgf

struct ifgf_plan_t {
  ifgf_plan_desc desc{};
  int N = 0, P = 0, nc = 0, ng = 0;
  int batch = 1;                // right-hand sides the per-apply buffers hold
  double omega = 0;
  bool poisoned = false;
  ifgf::KernelTimer timer;
  int64_t launches = 0;         // kernels launched by apply/solve since the last reset
  int device = 0;
  int num_sms = 0;
  int near_threads = 256;       // block size of the near-field matvec (set by ifgf_plan_tune)
  ifgf_tree_t tree;
  // device data
  ifgf::NodeGeom geo;
  int* dev_err = nullptr;       // device status word (bit 0: a tensor-core wait timed out)
  int inject = 0;               // fault injection for the timeout path (ifgf_plan_inject)
  ifgf_plan_t* resid = nullptr; // plan whose map forms the refinement residual (ifgf_plan_set_residual)
  std::vector<ifgf_plan_t*> resid_of;   // plans that use this one as their residual plan
  double* tab_D = nullptr;      // [nc][nc] Chebyshev differentiation matrix
  double* x_sorted = nullptr;   // [N][3] nodes in sorted order
  double* n_sorted = nullptr;   // [N][3]
  int* perm = nullptr;          // [N] sorted -> original
  int* leafc = nullptr;         // [N][3] integer leaf coordinates (original order)
  std::vector<ifgf::DevLevel> dl;  // index d
  ifgf::NearMatrix near;
  void* phi = nullptr;          // [batch][N][8][2] densities (plan precision), original order
  void* a_sorted = nullptr;     // [batch][N][8][2] phi * omega, sorted order
  void* a_orig = nullptr;       // [batch][N][8][2] phi * omega, original order (direct far)
  void* f28 = nullptr;          // [batch][N][28][2] scalar fields (plan precision)
  double* phi64 = nullptr;      // [batch][N][8][2] FP64 densities (prep output)
  ifgf::GmresWork gm;
  ifgf::Precond pc;             // hidden == 0: no network attached
  ifgf::BlockJacobi bj;         // inv == nullptr: no block-Jacobi preconditioner built
  ifgf_stats stats{};
  std::vector<void*> allocations;
};
