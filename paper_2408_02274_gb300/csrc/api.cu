// C ABI of the CBIE-IFGF library: plan creation (host octree + device setup
// kernels), forward map, raw scalar fields, GMRES solve, stats.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <mutex>
#include <new>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include "gmres.h"
#include "host_setup.h"
#include "kernels.h"

namespace ifgf {

static thread_local char g_last_err[512] = "";

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_last_err, sizeof(g_last_err), "%s: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}

// Explanation of the last non-CUDA failure of this thread, shown by ifgf_status_string for the
// status it was recorded with.
static thread_local char g_detail[512] = "";
static thread_local int g_detail_status = IFGF_OK;

void set_status_detail(int status, const char* msg) {
  g_detail_status = status;
  snprintf(g_detail, sizeof(g_detail), "%s", msg);
}

namespace {

struct Alloc {
  ifgf_plan_t* p;
  template <typename T>
  T* dev(size_t count) {
    if (count == 0) count = 1;
    void* ptr = nullptr;
    if (cudaMalloc(&ptr, count * sizeof(T)) != cudaSuccess) throw std::bad_alloc();
    p->allocations.push_back(ptr);
    p->stats.device_bytes += (int64_t)(count * sizeof(T));
    return static_cast<T*>(ptr);
  }
  template <typename T>
  T* upload(const std::vector<T>& v) {
    T* d = dev<T>(v.size());
    if (!v.empty() && cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
      throw std::runtime_error("cudaMemcpy H2D failed");
    return d;
  }
  template <typename T>
  T* upload(const T* v, size_t count) {
    T* d = dev<T>(count);
    if (count && cudaMemcpy(d, v, count * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
      throw std::runtime_error("cudaMemcpy H2D failed");
    return d;
  }
};

// Device arrays needed only while a plan is being built (candidate pairs, closest points,
// singular moments, fine-geometry coefficients ...): freed when the builder returns, so they
// neither stay on the device nor count in the plan's device_bytes.
struct Scratch {
  std::vector<void*> ptrs;
  ~Scratch() {
    for (void* q : ptrs) cudaFree(q);
  }
  template <typename T>
  T* dev(size_t count) {
    if (count == 0) count = 1;
    void* ptr = nullptr;
    if (cudaMalloc(&ptr, count * sizeof(T)) != cudaSuccess) throw std::bad_alloc();
    ptrs.push_back(ptr);
    return static_cast<T*>(ptr);
  }
  template <typename T>
  T* upload(const T* v, size_t count) {
    T* d = dev<T>(count);
    if (count && cudaMemcpy(d, v, count * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
      throw std::runtime_error("cudaMemcpy H2D failed");
    return d;
  }
  template <typename T>
  T* upload(const std::vector<T>& v) {
    return upload(v.data(), v.size());
  }
};

void free_all(ifgf_plan_t* p) {
  for (void* a : p->allocations) cudaFree(a);
  p->allocations.clear();
  if (p->gm.hres) cudaFreeHost(p->gm.hres);
  if (p->gm.hactive) cudaFreeHost(p->gm.hactive);
  if (p->gm.hk) cudaFreeHost(p->gm.hk);
  p->gm.hres = nullptr;
  p->gm.hactive = p->gm.hk = nullptr;
  for (auto& e : p->timer.pool)
    if (e) cudaEventDestroy(e);
  p->timer.pool.clear();
}

void check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    set_last_cuda_error(e, what, __FILE__, __LINE__);
    throw std::runtime_error(g_last_err);
  }
}

ifgf_status validate(const ifgf_plan_desc* d) {
  if (!d) return IFGF_EINVAL;
  if (d->num_patches < 1 || d->nc < 2 || d->nc > 24) return IFGF_EINVAL;
  if (!d->nodes || !d->dxdu || !d->dxdv || !d->fine) return IFGF_EINVAL;
  if (d->ng < 2 || d->ng > 48) return IFGF_EINVAL;
  if (!(d->k_ext > 0) || !(d->k_int > 0)) return IFGF_EINVAL;
  if (!(d->eps_ext > 0) || !(d->eps_int > 0) || !(d->mu_ext > 0) || !(d->mu_int > 0)) return IFGF_EINVAL;
  if (!(d->delta > 0)) return IFGF_EINVAL;
  if (d->n_beta < 4 || d->n_beta > 96) return IFGF_EINVAL;
  if (!(d->cov_d >= 2)) return IFGF_EINVAL;
  if (d->ns0 < 1 || d->na0 < 1 || d->ns0 > 64 || d->na0 > 64) return IFGF_EINVAL;
  if (d->leaf_size < 0 || d->gs_iters < 0 || d->gs_iters > 200) return IFGF_EINVAL;
  if (d->precision != IFGF_FP64 && d->precision != IFGF_FP32 && d->precision != IFGF_MIXED) return IFGF_EINVAL;
  if (d->far_mode != IFGF_FAR_IFGF && d->far_mode != IFGF_FAR_DIRECT) return IFGF_EINVAL;
  if (d->max_krylov < 0 || d->max_krylov > 1000) return IFGF_EINVAL;
  if (d->batch < 0 || d->batch > 1024) return IFGF_EINVAL;
  if (d->max_leaf_pts < 0 || d->max_leaf_pts > 1000000) return IFGF_EINVAL;
  if (d->gmres_scaling < 0 || d->gmres_scaling > 1) return IFGF_EINVAL;
  if (d->upward_tc < 0 || d->upward_tc > 1) return IFGF_EINVAL;
  if (d->refine < 0 || d->refine > 20) return IFGF_EINVAL;
  if (d->fields_per_pass != 0 && d->fields_per_pass != 1 && d->fields_per_pass != 8 && d->fields_per_pass != 16)
    return IFGF_EINVAL;
  if (narrow_passes(*d) && (d->far_mode != IFGF_FAR_IFGF || ifgf64(*d) || d->upward_tc != 0)) {
    set_status_detail(IFGF_EUNSUPPORTED,
                      "fields_per_pass 1 or 8 needs far_mode IFGF_FAR_IFGF, FP32 IFGF kernels and upward_tc 0");
    return IFGF_EUNSUPPORTED;
  }
  if (d->ps != 3 || d->pa != 5) return IFGF_EUNSUPPORTED;
  if ((int64_t)d->num_patches * d->nc * d->nc > (int64_t)1 << 30) return IFGF_EUNSUPPORTED;
  return IFGF_OK;
}

// The FP32 upward step into level L can run by units (the points of one octant in one child
// cone): the unit tables go to the device for FP32 and mixed IFGF plans.
bool unit_tables(const ifgf_plan_desc& d, const HostLevel& L) {
  return !ifgf64(d) && d.far_mode == IFGF_FAR_IFGF && L.tc_unit_ptr.size() > 1;
}

// The upward step into level L runs on the tensor cores when the plan asks for it (upward_tc),
// its IFGF kernels are FP32 (FP32 and mixed plans) and L has tensor-core tables whose cones fit
// the kernel's unit table.
bool upward_tc(const ifgf_plan_desc& d, const HostLevel& L) {
  return d.upward_tc == 1 && !ifgf64(d) && d.far_mode == IFGF_FAR_IFGF && !L.tc_item.empty() &&
         L.tc_max_units <= kTcMaxUnits;
}

void build(ifgf_plan_t* p) {
  const ifgf_plan_desc& d = p->desc;
  Alloc A{p};
  Scratch S;   // setup-only arrays
  const int N = p->N, P = p->P, nc = p->nc, ng = p->ng, npp = nc * nc;
  check(cudaGetDevice(&p->device), "cudaGetDevice");
  check(cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device), "attr");
  // ---------------- host octree and cone segments
  double leaf = d.leaf_size > 0 ? d.leaf_size : 0.25 * 2.0 * kPi / d.k_ext;
  double kmax = std::max(d.k_ext, d.k_int);
  using clk = std::chrono::steady_clock;
  auto since = [](clk::time_point a) { return std::chrono::duration<double>(clk::now() - a).count(); };
  clk::time_point t0 = clk::now();
  build_tree(p->tree, d.nodes, N, leaf, d.min_levels > 0 ? d.min_levels : 3, kmax, d.ns0, d.na0, d.max_leaf_pts);
  p->stats.setup_tree_s = since(t0);
  t0 = clk::now();
  const HostTree& t = p->tree;
  // ---------------- node geometry
  p->geo.x = A.upload(d.nodes, 3 * (size_t)N);
  p->geo.xu = A.upload(d.dxdu, 3 * (size_t)N);
  p->geo.xv = A.upload(d.dxdv, 3 * (size_t)N);
  p->geo.n = A.dev<double>(3 * (size_t)N);
  p->geo.t1 = A.dev<double>(3 * (size_t)N);
  p->geo.t2 = A.dev<double>(3 * (size_t)N);
  p->geo.J = A.dev<double>(N);
  p->geo.w = A.dev<double>(N);
  p->geo.g = A.dev<double>(3 * (size_t)N);
  double* fej = S.dev<double>(nc);
  double* Anc = S.dev<double>(npp);
  p->tab_D = A.dev<double>(npp);
  k_cheb_tables<<<(npp + 127) / 128, 128>>>(nc, fej, Anc, p->tab_D);
  k_node_geom<<<(N + 127) / 128, 128>>>(N, nc, fej, p->geo);
  double* Ang = S.dev<double>((size_t)ng * ng);
  k_cheb_tables<<<(ng * ng + 127) / 128, 128>>>(ng, nullptr, Ang, nullptr);
  double* fine = S.upload(d.fine, (size_t)P * ng * ng * 9);
  double* fcoef = S.dev<double>((size_t)P * ng * ng * 9);
  k_fine_coefs<<<P, 256>>>(ng, Ang, fine, fcoef);
  double* unodes_h = new double[nc];
  for (int k = 0; k < nc; ++k) unodes_h[k] = cheb_node(k, nc);
  double* unodes = S.upload(unodes_h, nc);
  delete[] unodes_h;
  check(cudaGetLastError(), "geometry kernels");
  // sorted geometry, permutations, leaf coordinates
  {
    std::vector<double> xs(3 * (size_t)N), ns(3 * (size_t)N);
    std::vector<double> nrm(3 * (size_t)N);
    check(cudaDeviceSynchronize(), "geometry sync");
    check(cudaMemcpy(nrm.data(), p->geo.n, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost), "normals D2H");
    for (int s = 0; s < N; ++s)
      for (int k = 0; k < 3; ++k) {
        xs[3 * (size_t)s + k] = d.nodes[3 * (size_t)t.perm[s] + k];
        ns[3 * (size_t)s + k] = nrm[3 * (size_t)t.perm[s] + k];
      }
    p->x_sorted = A.upload(xs);
    p->n_sorted = A.upload(ns);
    std::vector<int> pp(2 * (size_t)N);
    for (int s = 0; s < N; ++s) {
      pp[s] = t.perm[s];
      pp[N + s] = t.iperm[s];
    }
    p->perm = A.upload(pp);
    std::vector<int> lc(3 * (size_t)N);
    for (int l = 0; l < N; ++l)
      for (int k = 0; k < 3; ++k) lc[3 * (size_t)l + k] = t.leafc[l][k];
    p->leafc = A.upload(lc);
  }
  p->stats.setup_geometry_s = since(t0);
  // ---------------- near field: candidates, closest points, singular moments, matrix
  {
    Scratch SN;   // freed at the end of this block, before the IFGF tables are allocated
    t0 = clk::now();
    std::vector<double> gap;
    std::vector<int64_t> cptr;
    std::vector<int> cpatch;
    near_candidates(d.nodes, P, nc, d.delta, gap, cptr, cpatch);
    const int npairs = (int)cpatch.size();
    std::vector<int> ptgt(npairs);
    for (int l = 0; l < N; ++l)
      for (int64_t e = cptr[l]; e < cptr[l + 1]; ++e) ptgt[e] = l;
    p->stats.setup_near_host_s = since(t0);
    t0 = clk::now();
    int* d_ptgt = SN.upload(ptgt);
    int* d_ppatch = SN.upload(cpatch);
    double* d_uv = SN.dev<double>(2 * (size_t)npairs);
    uint8_t* d_sing = SN.dev<uint8_t>(npairs);
    int iters = d.gs_iters > 0 ? d.gs_iters : 20;
    k_closest<<<(npairs + 127) / 128, 128>>>(npairs, nc, ng, iters, d.delta, d_ptgt, d_ppatch, p->geo.x,
                                             fcoef, unodes, d_uv, d_sing);
    check(cudaGetLastError(), "k_closest launch");
    std::vector<uint8_t> sing(npairs);
    check(cudaMemcpy(sing.data(), d_sing, npairs, cudaMemcpyDeviceToHost), "singular flags D2H");
    p->stats.setup_closest_s = since(t0);
    cudaEvent_t ev[4];
    for (auto& e : ev) check(cudaEventCreate(&e), "setup event");
    std::vector<int> sp_pair, sp_of_pair(npairs, -1);
    for (int e = 0; e < npairs; ++e)
      if (sing[e]) {
        sp_of_pair[e] = (int)sp_pair.size();
        sp_pair.push_back(e);
      }
    const int nsp = (int)sp_pair.size();
    p->stats.singular_pairs = nsp;
    int* d_sp_pair = SN.upload(sp_pair);
    int* d_sp_of = SN.upload(sp_of_pair);
    double* W = SN.dev<double>((size_t)nsp * 8 * npp);
    std::vector<double> tb(d.n_beta);
    for (int k = 0; k < d.n_beta; ++k) tb[k] = cheb_node(k, d.n_beta);
    double* d_tb = SN.upload(tb);
    double* d_wb = SN.dev<double>(d.n_beta);
    k_cheb_tables<<<1, 128>>>(d.n_beta, d_wb, nullptr, nullptr);
    size_t smw = moments_smem_per_warp(nc, ng, d.n_beta);
    int wpb = 1;
    check(cudaFuncSetAttribute(k_moments, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(smw * wpb)),
          "moments smem attr");
    check(cudaEventRecord(ev[0]), "setup event");
    if (nsp > 0)
      k_moments<<<(nsp + wpb - 1) / wpb, 32 * wpb, smw * wpb>>>(nsp, d_sp_pair, d_ptgt, d_ppatch, d_uv, nc, ng,
          d.n_beta, d.cov_d, d_tb, d_wb, Anc, p->geo.x, p->geo.n, fcoef, d.k_ext, d.k_int, W);
    check(cudaGetLastError(), "k_moments launch");
    check(cudaEventRecord(ev[1]), "setup event");
    t0 = clk::now();
    std::vector<int64_t> row_ptr;
    host_array<int> col, pair;
    near_structure(t, P, nc, cptr, cpatch, sing, row_ptr, col, pair);   // overlaps the moments
    p->stats.setup_near_host_s += since(t0);
    p->near.nnz = (int64_t)col.size();
    p->stats.near_nnz = p->near.nnz;
    p->near.row_ptr = A.upload(row_ptr);
    p->near.col = A.upload(col.data(), col.size());
    int* d_pair = SN.upload(pair.data(), pair.size());
    // the near values in the plan's storage precision only
    if (store64(d))
      p->near.val64 = A.dev<double>(8 * (size_t)p->near.nnz);
    else
      p->near.val32 = A.dev<float>(8 * (size_t)p->near.nnz);
    check(cudaEventRecord(ev[2]), "setup event");
    k_near_values<<<(unsigned)(((size_t)N * 32 + 255) / 256), 256>>>(N, nc, p->near.row_ptr, p->near.col, d_pair,
        d_sp_of, W, p->geo.x, p->geo.n, p->geo.w, p->leafc, d.k_ext, d.k_int, p->near.val64, p->near.val32);
    check(cudaGetLastError(), "k_near_values launch");
    check(cudaEventRecord(ev[3]), "setup event");
    check(cudaDeviceSynchronize(), "near setup");
    float ms_m = 0, ms_v = 0;
    check(cudaEventElapsedTime(&ms_m, ev[0], ev[1]), "setup event");
    check(cudaEventElapsedTime(&ms_v, ev[2], ev[3]), "setup event");
    p->stats.setup_moments_s = 1e-3 * ms_m;
    p->stats.setup_near_values_s = 1e-3 * ms_v;
    for (auto& e : ev) cudaEventDestroy(e);
  }
  // ---------------- IFGF level tables
  p->dl.assign(t.D + 1, DevLevel());
  for (int dd = 3; dd <= t.D; ++dd) {
    const HostLevel& L = t.lv[dd];
    DevLevel& Dl = p->dl[dd];
    Dl.d = dd;
    Dl.nboxes = (int)L.key.size();
    Dl.nslots = (int)L.slot_box.size();
    Dl.cg = L.cg();
    Dl.H = L.H;
    std::vector<double> cen(3 * (size_t)Dl.nboxes);
    for (int b = 0; b < Dl.nboxes; ++b)
      for (int k = 0; k < 3; ++k) cen[3 * (size_t)b + k] = t.corner[k] + L.H * (L.ic[b][k] + 0.5);
    Dl.box_center = A.upload(cen);
    Dl.ncomp = (int)L.upcone_list.size();
    Dl.ckeys = A.upload(L.upcone_list);
    if (!L.cmap.empty()) Dl.cmap = A.upload(L.cmap);
    Dl.slot_box = A.upload(L.slot_box);
    Dl.slot_cone = A.upload(L.slot_cone);
    Dl.box_slot_ptr = A.upload(L.box_slot_ptr);
    for (int b = 0; b < Dl.nboxes; ++b)
      Dl.max_box_slots = std::max(Dl.max_box_slots, L.box_slot_ptr[b + 1] - L.box_slot_ptr[b]);
    std::vector<int> bp(Dl.nboxes + 1);
    for (int b = 0; b < Dl.nboxes; ++b) bp[b] = L.pt_begin[b];
    bp[Dl.nboxes] = N;
    Dl.box_pt_ptr = A.upload(bp);
    std::vector<int> ch(8 * (size_t)Dl.nboxes);
    for (int b = 0; b < Dl.nboxes; ++b)
      for (int o = 0; o < 8; ++o) ch[8 * (size_t)b + o] = L.child[b][o];
    Dl.child = A.upload(ch);
    Dl.slot_upidx = A.upload(L.slot_upidx);
    Dl.up_cc = A.upload(L.up_cc);
    Dl.up_order = A.upload(L.up_order);
    Dl.up_task = A.upload(L.up_task);
    Dl.up_task_ptr = A.upload(L.up_task_ptr);
    if (unit_tables(d, L)) {   // the FP32 upward step by units or items (SIMT candidates, tensor cores)
      Dl.tc_order = A.upload(L.tc_order);
      Dl.tc_unit = A.upload(L.tc_unit);
      Dl.tc_unit_ptr = A.upload(L.tc_unit_ptr);
      Dl.tc_item = A.upload(L.tc_item);
      Dl.ntc_items = (int)(L.tc_item.size() / kTcBoxes);
    }
    if (upward_tc(d, L)) Dl.tc = true;
    {
      std::vector<double2> th(L.na), ph(2 * (size_t)L.na);
      for (int g = 0; g < L.na; ++g) th[g] = make_double2(std::cos(g * kPi / L.na), std::sin(g * kPi / L.na));
      for (int g = 0; g < 2 * L.na; ++g) ph[g] = make_double2(std::cos(g * kPi / L.na), std::sin(g * kPi / L.na));
      Dl.trig_th = A.upload(th);
      Dl.trig_ph = A.upload(ph);
    }
    Dl.tgt_ptr = A.upload(L.tgt_ptr);
    Dl.tgt_chunk = reinterpret_cast<int2*>(A.upload(L.tgt_chunk));
    Dl.ntgt_chunks = (int)(L.tgt_chunk.size() / 2);
    // box chunks when the level has at least two waves of them (12 resident warps per SM), else
    // a warp per target; ifgf_plan_tune measures both
    Dl.tgt_mode = Dl.ntgt_chunks >= 2 * 12 * std::max(p->num_sms, 1) ? 1 : 0;
    Dl.tgt_slot = A.upload(L.tgt_slot.data(), L.tgt_slot.size());
    Dl.ninter = (int64_t)L.tgt_slot.size();
    Dl.cstride = (size_t)Dl.nslots * kQ * coef_columns(d);
    p->stats.boxes[dd] = Dl.nboxes;
    p->stats.cones[dd] = Dl.nslots;
    p->stats.ns[dd] = L.ns;
    p->stats.na[dd] = L.na;
    p->stats.interactions[dd] = Dl.ninter;
  }
  // Cone coefficients: a level's values are written by the leaf step (d = D) or the upward
  // step from d+1, and read by the target step at d and the upward step into d-1, so only
  // two consecutive levels are live at once: levels of equal parity share one buffer.
  if (d.far_mode == IFGF_FAR_IFGF) {
    size_t need[2] = {0, 0};
    for (int dd = 3; dd <= t.D; ++dd) need[dd & 1] = std::max(need[dd & 1], p->dl[dd].cstride * (size_t)p->batch);
    void* buf[2] = {nullptr, nullptr};
    for (int a = 0; a < 2; ++a)
      if (need[a]) buf[a] = ifgf64(d) ? (void*)A.dev<double>(need[a]) : (void*)A.dev<float>(need[a]);
    for (int dd = 3; dd <= t.D; ++dd) p->dl[dd].coefs = buf[dd & 1];
    // tensor-core operand images of level dd's coefficients, read by the upward step into dd-1
    // when it runs on the tensor cores (same parity sharing as the coefficients)
    size_t need_img[2] = {0, 0};
    for (int dd = 4; dd <= t.D; ++dd)
      if (upward_tc(d, t.lv[dd - 1]))
        need_img[dd & 1] = std::max(need_img[dd & 1], (size_t)p->dl[dd].nslots * kImgFloatsHost * (size_t)p->batch);
    float* ibuf[2] = {nullptr, nullptr};
    for (int a = 0; a < 2; ++a)
      if (need_img[a]) ibuf[a] = A.dev<float>(need_img[a]);
    for (int dd = 4; dd <= t.D; ++dd)
      if (upward_tc(d, t.lv[dd - 1])) {
        p->dl[dd].img = ibuf[dd & 1];
        p->dl[dd].istride = (size_t)p->dl[dd].nslots * kImgFloatsHost;
      }
  }
  for (int dd = 1; dd < 3 && dd <= t.D; ++dd) p->stats.boxes[dd] = (int)t.lv[dd].key.size();
  {
    const HostLevel& L = t.lv[t.D];
    int64_t lp = 0;
    for (size_t b = 0; b < L.key.size(); ++b)
      lp += (int64_t)(L.pt_end[b] - L.pt_begin[b]) * (L.box_slot_ptr[b + 1] - L.box_slot_ptr[b]) * kQ;
    p->stats.leaf_pairs = lp;
    int64_t up = 0;
    for (int dd = t.D; dd > 3; --dd) {
      const HostLevel& Pp = t.lv[dd - 1];
      for (size_t s = 0; s < Pp.slot_box.size(); ++s) {
        int nchild = 0;
        for (int o = 0; o < 8; ++o) nchild += Pp.child[Pp.slot_box[s]][o] >= 0;
        up += (int64_t)nchild * kQ;
      }
    }
    p->stats.up_pairs = up;
  }
  p->stats.n = N;
  p->stats.levels = t.D;
  check(setup_combine_kernels(), "combine kernel attributes");
  check(setup_ifgf_kernels(), "IFGF kernel attributes");
  check(setup_bj_kernels(), "block-Jacobi kernel attributes");
  // ---------------- per-apply buffers and GMRES workspace
  const size_t el = store64(d) ? sizeof(double) : sizeof(float);
  const size_t el_s = ifgf64(d) ? sizeof(double) : sizeof(float);   // weighted densities read by IFGF
  const size_t B = (size_t)p->batch;
  p->phi = A.dev<char>(16 * (size_t)N * el * B);
  p->a_sorted = A.dev<char>(16 * (size_t)N * el_s * B);
  p->a_orig = A.dev<char>(16 * (size_t)N * el * B);
  p->f28 = A.dev<char>(56 * (size_t)N * el * B);
  p->phi64 = A.dev<double>(16 * (size_t)N * B);
  p->dev_err = A.dev<int>(1);
  check(cudaMemset(p->dev_err, 0, sizeof(int)), "status word");
  GmresWork& G = p->gm;
  G.max_iter = d.max_krylov > 0 ? d.max_krylov : 300;
  const size_t n4 = 4 * (size_t)N, m1 = (size_t)(G.max_iter + 1);
  G.V = A.dev<double>(2 * n4 * m1 * B);
  G.H = A.dev<double>(2 * m1 * m1 * B);
  G.cs = A.dev<double>(2 * m1 * B);
  G.sn = A.dev<double>(2 * m1 * B);
  G.g = A.dev<double>(2 * m1 * B);
  G.h = A.dev<double>(4 * m1 * B);
  G.part = A.dev<double>(2 * (size_t)dots_blocks((int64_t)n4) * m1 * B);
  G.scal = A.dev<double>(8 * B);
  G.w = A.dev<double>(2 * n4 * B);
  G.b = A.dev<double>(2 * n4 * B);
  G.y = A.dev<double>(2 * n4 * B);
  G.inc = A.dev<double>(12 * (size_t)N * B);
  if (d.refine > 0) {
    G.y_acc = A.dev<double>(2 * n4 * B);
    G.b_orig = A.dev<double>(2 * n4 * B);
  }
  G.active = A.dev<int>(B);
  G.kfin = A.dev<int>(B);
  check(cudaMallocHost(&G.hres, 8 * B * sizeof(double)), "pinned scalars");
  check(cudaMallocHost(&G.hactive, B * sizeof(int)), "pinned flags");
  check(cudaMallocHost(&G.hk, B * sizeof(int)), "pinned counts");
  p->timer.pool.assign(256, nullptr);
  p->timer.kind.assign(128, 0);
  for (auto& e : p->timer.pool) check(cudaEventCreate(&e), "event");
  check(cudaDeviceSynchronize(), "plan_create sync");
}

bool is_device_ptr(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// out_r = A y_r for r < nrhs (y, out: device [nrhs][4N] complex128); one launch per kernel
cudaError_t forward(ifgf_plan_t* p, const double* y, double* out, int nrhs, cudaStream_t s) {
  cudaError_t e;
  if (p->timer.on && p->timer.npending > 0 && (e = timer_flush(p)) != cudaSuccess) return e;
  int r = timer_begin(p, TK_PREP, s);
  if ((e = launch_density_prep(p, y, nullptr, s, nrhs)) != cudaSuccess) return e;
  timer_end(p, r, s);
  r = timer_begin(p, TK_NEAR, s);
  if ((e = launch_near(p, s, nrhs)) != cudaSuccess) return e;
  timer_end(p, r, s);
  p->launches += 3;   // prep, near, combine
  if (p->desc.far_mode == IFGF_FAR_IFGF) {
    if ((e = launch_far_ifgf(p, s, nrhs)) != cudaSuccess) return e;
  } else {
    r = timer_begin(p, TK_FAR_DIRECT, s);
    if ((e = launch_far_direct(p, s, nrhs)) != cudaSuccess) return e;
    timer_end(p, r, s);
    ++p->launches;
  }
  r = timer_begin(p, TK_COMBINE, s);
  if ((e = launch_combine(p, y, out, s, nrhs)) != cudaSuccess) return e;
  timer_end(p, r, s);
  return cudaSuccess;
}

}  // namespace

int timer_begin(ifgf_plan_t* p, int kind, cudaStream_t s) {
  KernelTimer& T = p->timer;
  if (!T.on) return -1;
  if (2 * (T.npending + 1) > (int)T.pool.size()) {
    if (timer_flush(p) != cudaSuccess) return -1;
  }
  int r = T.npending++;
  T.kind[r] = kind;
  cudaEventRecord(T.pool[2 * r], s);
  return r;
}

void timer_end(ifgf_plan_t* p, int rec, cudaStream_t s) {
  if (rec < 0) return;
  cudaEventRecord(p->timer.pool[2 * rec + 1], s);
}

cudaError_t timer_flush(ifgf_plan_t* p) {
  KernelTimer& T = p->timer;
  if (T.npending == 0) return cudaSuccess;
  cudaError_t e = cudaEventSynchronize(T.pool[2 * T.npending - 1]);
  if (e != cudaSuccess) return e;
  for (int r = 0; r < T.npending; ++r) {
    float ms = 0;
    if ((e = cudaEventElapsedTime(&ms, T.pool[2 * r], T.pool[2 * r + 1])) != cudaSuccess) return e;
    T.total_ms[T.kind[r]] += ms;
    T.calls[T.kind[r]] += 1;
  }
  T.npending = 0;
  return cudaSuccess;
}

}  // namespace ifgf

using namespace ifgf;

// Byte counts of the device arrays ifgf_plan_create allocates, in the order build() allocates
// them (a zero-length array takes one element there too).  Keep in step with build().
namespace {
struct ByteCount {
  int64_t total = 0;
  template <typename T>
  void dev(size_t count) {
    total += (int64_t)((count ? count : 1) * sizeof(T));
  }
};
}  // namespace

extern "C" {

const char* ifgf_status_string(ifgf_status s) {
  switch (s) {
    case IFGF_OK: return "ok";
    case IFGF_EINVAL: return "invalid argument";
    case IFGF_ENOMEM: return "out of memory";
    case IFGF_ECUDA: return g_last_err[0] ? g_last_err : "CUDA error";
    case IFGF_ENOCONV: return "GMRES did not reach the tolerance";
    case IFGF_ETIMEOUT: return (g_detail_status == s && g_detail[0]) ? g_detail : "device wait timed out";
    case IFGF_EUNSUPPORTED: return (g_detail_status == s && g_detail[0]) ? g_detail : "unsupported option";
    case IFGF_EINTERNAL: return (g_detail_status == s && g_detail[0]) ? g_detail : "internal error";
    default: return "unknown status";
  }
}

ifgf_status ifgf_plan_create(const ifgf_plan_desc* desc, ifgf_plan* out) {
  if (!out) return IFGF_EINVAL;
  *out = nullptr;
  ifgf_status st = validate(desc);
  if (st != IFGF_OK) return st;
  auto t0 = std::chrono::steady_clock::now();
  ifgf_plan_t* p = new (std::nothrow) ifgf_plan_t();
  if (!p) return IFGF_ENOMEM;
  p->desc = *desc;
  p->P = desc->num_patches;
  p->nc = desc->nc;
  p->ng = desc->ng;
  p->N = p->P * p->nc * p->nc;
  p->batch = desc->batch > 0 ? desc->batch : 1;
  p->omega = desc->k_ext / std::sqrt(desc->eps_ext * desc->mu_ext);
  try {
    build(p);
  } catch (const std::bad_alloc&) {
    free_all(p);
    delete p;
    return IFGF_ENOMEM;
  } catch (const std::invalid_argument& e) {
    snprintf(g_last_err, sizeof(g_last_err), "%s", e.what());
    free_all(p);
    delete p;
    return IFGF_EINVAL;
  } catch (const std::exception& e) {
    if (!g_last_err[0]) snprintf(g_last_err, sizeof(g_last_err), "%s", e.what());
    free_all(p);
    delete p;
    return IFGF_ECUDA;
  }
  // descriptor pointers belong to the caller: do not keep them
  p->desc.nodes = p->desc.dxdu = p->desc.dxdv = p->desc.fine = nullptr;
  p->stats.setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  *out = p;
  return IFGF_OK;
}

ifgf_status ifgf_plan_estimate(const ifgf_plan_desc* desc, ifgf_plan_estimate_t* out) {
  if (!out) return IFGF_EINVAL;
  std::memset(out, 0, sizeof(*out));
  ifgf_status st = validate(desc);
  if (st != IFGF_OK) return st;
  const ifgf_plan_desc& d = *desc;
  const int P = d.num_patches, nc = d.nc, ng = d.ng, npp = nc * nc, N = P * npp;
  const size_t B = (size_t)(d.batch > 0 ? d.batch : 1);
  const size_t el = store64(d) ? sizeof(double) : sizeof(float);
  const size_t el_s = ifgf64(d) ? sizeof(double) : sizeof(float);
  try {
    HostTree t;
    const double leaf = d.leaf_size > 0 ? d.leaf_size : 0.25 * 2.0 * kPi / d.k_ext;
    build_tree(t, d.nodes, N, leaf, d.min_levels > 0 ? d.min_levels : 3, std::max(d.k_ext, d.k_int), d.ns0, d.na0,
               d.max_leaf_pts);
    std::vector<double> gap;
    std::vector<int64_t> cptr;
    std::vector<int> cpatch;
    near_candidates(d.nodes, P, nc, d.delta, gap, cptr, cpatch);
    const size_t npairs = cpatch.size();
    const int64_t nnz = near_nnz_bound(t, P, nc, cptr, cpatch);
    out->levels = t.D;
    out->candidate_pairs = (int64_t)npairs;
    out->near_nnz_max = nnz;
    // node geometry (x, x_u, x_v, n, t1, t2, J, w, g, D table), sorted copies, permutations
    ByteCount g;
    for (int k = 0; k < 6; ++k) g.dev<double>(3 * (size_t)N);
    g.dev<double>(N);
    g.dev<double>(N);
    g.dev<double>(3 * (size_t)N);
    g.dev<double>(npp);
    g.dev<double>(3 * (size_t)N);
    g.dev<double>(3 * (size_t)N);
    g.dev<int>(2 * (size_t)N);
    g.dev<int>(3 * (size_t)N);
    // near matrix
    ByteCount nm;
    nm.dev<int64_t>((size_t)N + 1);
    nm.dev<int>((size_t)nnz);
    if (el == sizeof(double))
      nm.dev<double>(8 * (size_t)nnz);
    else
      nm.dev<float>(8 * (size_t)nnz);
    // setup temporaries: outer (geometry interpolation) and near-field (closest points, moments)
    ByteCount so, sn;
    so.dev<double>(nc);
    so.dev<double>(npp);
    so.dev<double>((size_t)ng * ng);
    so.dev<double>((size_t)P * ng * ng * 9);
    so.dev<double>((size_t)P * ng * ng * 9);
    so.dev<double>(nc);
    sn.dev<int>(npairs);
    sn.dev<int>(npairs);
    sn.dev<double>(2 * npairs);
    sn.dev<uint8_t>(npairs);
    sn.dev<int>(npairs);                    // singular pairs (at most every candidate)
    sn.dev<int>(npairs);
    sn.dev<double>(npairs * 8 * (size_t)npp);
    sn.dev<double>((size_t)d.n_beta);
    sn.dev<double>((size_t)d.n_beta);
    sn.dev<int>((size_t)nnz);
    // level tables and cone coefficients
    ByteCount tb;
    size_t need[2] = {0, 0};
    for (int dd = 3; dd <= t.D; ++dd) {
      const HostLevel& L = t.lv[dd];
      const size_t nb = L.key.size(), nslots = L.slot_box.size();
      tb.dev<double>(3 * nb);
      tb.dev<cone_key>(L.upcone_list.size());
      if (!L.cmap.empty()) tb.dev<int>(L.cmap.size());
      tb.dev<int>(nslots);
      tb.dev<cone_key>(nslots);
      tb.dev<int>(L.box_slot_ptr.size());
      tb.dev<int>(nb + 1);
      tb.dev<int>(8 * nb);
      tb.dev<int>(L.slot_upidx.size());
      tb.dev<int32_t>(L.up_cc.size());
      tb.dev<int32_t>(L.up_order.size());
      tb.dev<int32_t>(L.up_task.size());
      tb.dev<int32_t>(L.up_task_ptr.size());
      if (unit_tables(d, L)) {
        tb.dev<int32_t>(L.tc_order.size());
        tb.dev<int32_t>(L.tc_unit.size());
        tb.dev<int32_t>(L.tc_unit_ptr.size());
        tb.dev<int32_t>(L.tc_item.size());
      }
      tb.dev<double2>((size_t)L.na);
      tb.dev<double2>(2 * (size_t)L.na);
      tb.dev<int64_t>(L.tgt_ptr.size());
      tb.dev<int32_t>(L.tgt_chunk.size());
      tb.dev<int32_t>(L.tgt_slot.size());
      out->cones[dd] = (int64_t)nslots;
      need[dd & 1] = std::max(need[dd & 1], nslots * kQ * (size_t)coef_columns(d) * B);
    }
    tb.dev<int>(1);   // the plan's device status word
    ByteCount cf;
    if (d.far_mode == IFGF_FAR_IFGF) {
      for (int a = 0; a < 2; ++a)
        if (need[a]) (el_s == sizeof(double)) ? cf.dev<double>(need[a]) : cf.dev<float>(need[a]);
      size_t need_img[2] = {0, 0};
      for (int dd = 4; dd <= t.D; ++dd)
        if (upward_tc(d, t.lv[dd - 1]))
          need_img[dd & 1] = std::max(need_img[dd & 1], t.lv[dd].slot_box.size() * kImgFloatsHost * B);
      for (int a = 0; a < 2; ++a)
        if (need_img[a]) cf.dev<float>(need_img[a]);
    }
    // per-apply buffers and GMRES workspace
    ByteCount ap, gm;
    for (int k = 0; k < 3; ++k) ap.dev<char>(16 * (size_t)N * (k == 1 ? el_s : el) * B);
    ap.dev<char>(56 * (size_t)N * el * B);
    ap.dev<double>(16 * (size_t)N * B);
    const size_t n4 = 4 * (size_t)N, m1 = (size_t)((d.max_krylov > 0 ? d.max_krylov : 300) + 1);
    gm.dev<double>(2 * n4 * m1 * B);
    gm.dev<double>(2 * m1 * m1 * B);
    for (int k = 0; k < 3; ++k) gm.dev<double>(2 * m1 * B);
    gm.dev<double>(4 * m1 * B);
    gm.dev<double>(2 * (size_t)dots_blocks((int64_t)n4) * m1 * B);
    gm.dev<double>(8 * B);
    for (int k = 0; k < 3; ++k) gm.dev<double>(2 * n4 * B);
    gm.dev<double>(12 * (size_t)N * B);
    if (d.refine > 0)
      for (int k = 0; k < 2; ++k) gm.dev<double>(2 * n4 * B);
    gm.dev<int>(B);
    gm.dev<int>(B);
    out->bytes_geometry = g.total;
    out->bytes_near_max = nm.total;
    out->bytes_tables = tb.total;
    out->bytes_coefs = cf.total;
    out->bytes_apply = ap.total;
    out->bytes_gmres = gm.total;
    out->bytes_plan_max = g.total + nm.total + tb.total + cf.total + ap.total + gm.total;
    // peak: while the near values are computed (geometry, near matrix and both temporaries
    // live), or at the end (the whole plan and the outer temporaries)
    out->bytes_setup_peak_max = std::max(g.total + nm.total + so.total + sn.total, out->bytes_plan_max + so.total);
  } catch (const std::bad_alloc&) {
    return IFGF_ENOMEM;
  } catch (const std::exception&) {
    return IFGF_EINVAL;
  }
  return IFGF_OK;
}

static void unlink_residual(ifgf_plan_t* p);

ifgf_status ifgf_plan_destroy(ifgf_plan plan) {
  if (!plan) return IFGF_OK;
  // residual-plan links in both directions end with the plan
  unlink_residual(plan);
  for (ifgf_plan_t* q : plan->resid_of) q->resid = nullptr;
  plan->resid_of.clear();
  cudaDeviceSynchronize();
  free_all(plan);
  delete plan;
  return IFGF_OK;
}

ifgf_status ifgf_apply_batch(ifgf_plan p, int32_t nrhs, const void* y, void* out, ifgf_stream stream) {
  if (!p || !y || !out || y == out) return IFGF_EINVAL;
  if (nrhs < 1 || nrhs > p->batch) return IFGF_EINVAL;
  if (p->poisoned) return IFGF_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = forward(p, (const double*)y, (double*)out, nrhs, s);
  if (e != cudaSuccess) {
    set_last_cuda_error(e, "ifgf_apply", __FILE__, __LINE__);
    p->poisoned = true;
    return IFGF_ECUDA;
  }
  return IFGF_OK;
}

ifgf_status ifgf_apply(ifgf_plan p, const void* y, void* out, ifgf_stream stream) {
  return ifgf_apply_batch(p, 1, y, out, stream);
}

ifgf_status ifgf_apply_direct_patches(ifgf_plan p, const void* y, void* out, const int32_t* patches,
                                      int32_t npatches, ifgf_stream stream) {
  if (!p || !y || !out || !patches || y == out) return IFGF_EINVAL;
  if (npatches < 1 || npatches > p->P) return IFGF_EINVAL;
  if (p->poisoned) return IFGF_ECUDA;
  std::vector<uint8_t> seen;
  try {
    seen.assign((size_t)p->P, 0);
  } catch (const std::bad_alloc&) {
    return IFGF_ENOMEM;
  }
  for (int32_t i = 0; i < npatches; ++i) {
    const int32_t q = patches[i];
    if (q < 0 || q >= p->P || seen[q]) return IFGF_EINVAL;
    seen[q] = 1;
  }
  // target blocks: the listed patches' node ranges cut at multiples of 128, so that every
  // listed row has the origin (the first node of its aligned run of 128) and the summation
  // order of the FP64 full map; ranges of adjacent listed patches merge
  std::vector<int32_t> blk;
  try {
    const int npp = p->nc * p->nc;
    for (int32_t q = 0; q < p->P; ++q) {
      if (!seen[q]) continue;
      int32_t a = q * npp, b = (q + 1) * npp;
      while (q + 1 < p->P && seen[q + 1]) b = (++q + 1) * npp;
      for (int32_t o = a / 128 * 128; o < b; o += 128) {
        blk.push_back(o);
        blk.push_back(std::max(a, o));
        blk.push_back(std::min(b, o + 128));
      }
    }
  } catch (const std::bad_alloc&) {
    return IFGF_ENOMEM;
  }
  const int nblk = (int)(blk.size() / 3);
  cudaStream_t s = (cudaStream_t)stream;
  int* d_blk = nullptr;   // the block list on the device
  if (cudaMalloc(&d_blk, sizeof(int) * blk.size()) != cudaSuccess) {
    cudaGetLastError();
    return IFGF_ENOMEM;
  }
  cudaError_t e = cudaMemcpyAsync(d_blk, blk.data(), sizeof(int) * blk.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_density_prep(p, (const double*)y, nullptr, s, 1);
  if (e == cudaSuccess) e = launch_near(p, s, 1);
  if (e == cudaSuccess) e = launch_far_direct_blocks(p, s, d_blk, nblk);
  if (e == cudaSuccess) e = launch_combine(p, (const double*)y, (double*)out, s, 1);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_blk);
  if (e != cudaSuccess) {
    set_last_cuda_error(e, "ifgf_apply_direct_patches", __FILE__, __LINE__);
    p->poisoned = true;
    return IFGF_ECUDA;
  }
  return IFGF_OK;
}

ifgf_status ifgf_far_field(ifgf_plan p, int32_t nrhs, const void* y, int32_t ndirs, const double* dirs, void* out,
                           ifgf_stream stream) {
  if (!p || !y || !dirs || !out || ndirs < 1 || ndirs > (1 << 24)) return IFGF_EINVAL;
  if (nrhs < 1 || nrhs > p->batch) return IFGF_EINVAL;
  if (p->poisoned) return IFGF_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch_density_prep(p, (const double*)y, nullptr, s, nrhs);
  if (e == cudaSuccess) e = launch_far_field(p, nrhs, ndirs, dirs, (double*)out, s);
  if (e != cudaSuccess) {
    set_last_cuda_error(e, "ifgf_far_field", __FILE__, __LINE__);
    p->poisoned = true;
    return IFGF_ECUDA;
  }
  return IFGF_OK;
}

// Autotuner: the launch shapes with a measured effect, timed on this plan's own tables and
// buffers (the fields buffer is scratch between applies).
static cudaError_t time_ms(cudaStream_t s, int reps, const std::function<cudaError_t()>& run, float* ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = run();   // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) e = run();
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

ifgf_status ifgf_plan_tune(ifgf_plan p, int32_t reps, int32_t* choices, float* times_ms, ifgf_stream stream) {
  if (!p || reps < 1 || reps > 1000) return IFGF_EINVAL;
  if (p->poisoned) return IFGF_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  try {
    if (choices)
      for (int k = 0; k < 64; ++k) choices[k] = -1;
    if (times_ms)
      for (int k = 0; k < 128; ++k) times_ms[k] = 0.f;
    // the far-field kernels below are the all-fields ones; a plan of fewer fields per pass has
    // coefficient buffers too narrow for them and keeps its single pass shapes
    const bool vec = p->desc.far_mode == IFGF_FAR_IFGF && !ifgf64(p->desc) && !narrow_passes(p->desc);
    // (c): per level, a warp per target or per box chunk
    if (vec) {
      for (int d = 3; d <= p->tree.D && e == cudaSuccess; ++d) {
        float t[2] = {0.f, 0.f};
        for (int m = 0; m < 2 && e == cudaSuccess; ++m)
          e = time_ms(s, reps, [&]() { return launch_target_level(p, d, m, s); }, &t[m]);
        if (e != cudaSuccess) break;
        p->dl[d].tgt_mode = (t[1] < t[0] && p->dl[d].ntgt_chunks > 0) ? 1 : 0;
        if (choices && d < 25) choices[d] = p->dl[d].tgt_mode;
        if (times_ms && d < 25) {
          times_ms[2 * d] = t[0] / reps;
          times_ms[2 * d + 1] = t[1] / reps;
        }
      }
    }
    // (a): the FP32 leaf step with SIMT or tensor-pipe density products
    if (e == cudaSuccess && vec) {
      float t[2] = {0.f, 0.f};
      for (int m = 0; m < 2 && e == cudaSuccess; ++m)
        e = time_ms(s, reps, [&]() { return launch_leaf_level(p, m, s); }, &t[m]);
      if (e == cudaSuccess) {
        p->dl[p->tree.D].leaf_mode = t[1] < t[0] ? 1 : 0;
        if (choices) choices[30] = p->dl[p->tree.D].leaf_mode;
        if (times_ms) {
          times_ms[60] = t[0] / reps;
          times_ms[61] = t[1] / reps;
        }
      }
    }
    // (b): per parent level, the FP32 SIMT upward step by point-group runs or a warp per slot
    if (e == cudaSuccess && vec) {
      for (int d = 3; d < p->tree.D && e == cudaSuccess; ++d) {
        DevLevel& Pp = p->dl[d];
        if (Pp.tc || !Pp.tc_unit_ptr || Pp.nslots == 0) continue;
        float t[3] = {0.f, 0.f, 0.f};
        for (int m = 0; m < 3 && e == cudaSuccess; ++m)
          e = time_ms(s, reps, [&]() { return launch_up_level(p, d, m, s); }, &t[m]);
        if (e != cudaSuccess) break;
        Pp.up_mode = 0;
        for (int m = 1; m < 3; ++m)
          if (t[m] < t[Pp.up_mode]) Pp.up_mode = m;
        if (choices && d < 25) choices[32 + d] = Pp.up_mode;
        if (times_ms && d < 25) {
          times_ms[64 + 2 * d] = t[0] / reps;
          times_ms[65 + 2 * d] = t[1] / reps;
          times_ms[100 + d] = t[2] / reps;
        }
      }
    }
    // (d): the near-field matvec's block size
    if (e == cudaSuccess) {
      const int sizes[2] = {128, 256};
      float t[2] = {0.f, 0.f};
      for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        p->near_threads = sizes[k];
        e = time_ms(s, reps, [&]() { return launch_near(p, s, 1); }, &t[k]);
      }
      if (e == cudaSuccess) {
        p->near_threads = t[0] < t[1] ? 128 : 256;
        if (choices) choices[25] = p->near_threads;
        if (times_ms) {
          times_ms[50] = t[0] / reps;
          times_ms[51] = t[1] / reps;
        }
      }
    }
  } catch (const std::bad_alloc&) {
    return IFGF_ENOMEM;
  } catch (const std::exception& ex) {
    set_status_detail(IFGF_EINTERNAL, ex.what());
    return IFGF_EINTERNAL;
  }
  if (e != cudaSuccess) {
    set_last_cuda_error(e, "ifgf_plan_tune", __FILE__, __LINE__);
    p->poisoned = true;
    return IFGF_ECUDA;
  }
  return IFGF_OK;
}

ifgf_status ifgf_apply_fields(ifgf_plan p, const void* phi, void* f28, int32_t which, ifgf_stream stream) {
  if (!p || !phi || !f28 || which < 1 || which > 3) return IFGF_EINVAL;
  if (p->poisoned) return IFGF_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch_density_prep(p, nullptr, (const double*)phi, s);
  if (e == cudaSuccess) e = (which & IFGF_PART_NEAR) ? launch_near(p, s) : launch_zero_f28(p, s);
  if (e == cudaSuccess && (which & IFGF_PART_FAR))
    e = (p->desc.far_mode == IFGF_FAR_IFGF) ? launch_far_ifgf(p, s) : launch_far_direct(p, s);
  if (e == cudaSuccess) e = launch_f28_export(p, (double*)f28, s);
  if (e != cudaSuccess) {
    set_last_cuda_error(e, "ifgf_apply_fields", __FILE__, __LINE__);
    p->poisoned = true;
    return IFGF_ECUDA;
  }
  return IFGF_OK;
}

// z = M v for the right preconditioner: the block-Jacobi inverse and/or the network (with both,
// the network's output corrects the block-Jacobi product).
static cudaError_t precond_apply(ifgf_plan_t* p, int nrhs, const double* v, double* z, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (p->bj.inv) e = launch_bj_apply(p, nrhs, v, z, s);
  if (e == cudaSuccess && p->pc.hidden > 0) e = launch_mlp_apply(p, nrhs, v, z, s, p->bj.inv ? z : v);
  return e;
}

// Reads and clears the plan's device status word (after the work queued on s); *word = its value.
static cudaError_t take_status_word(ifgf_plan_t* p, cudaStream_t s, int* word) {
  *word = 0;
  cudaError_t e = cudaMemcpyAsync(word, p->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && *word != 0) e = cudaMemsetAsync(p->dev_err, 0, sizeof(int), s);
  return e;
}

static const char* kTimeoutMsg =
    "a bounded tensor-core wait of the upward step (upward_tc) expired; the results of the applies "
    "queued since the last check are not valid";

// Residual refinement after GMRES (plan field refine): r = b - A y is formed in FP64 from the
// residual plan's map (ifgf_plan_set_residual; the plan's own map without one); while |r| / |b|
// > tol and falling (by at least 10% a sweep), GMRES with the plan's own map solves
// A d = r from zero to the relative accuracy 0.5 tol |b| / |r| and y += d.  A sweep that does not
// lower a right-hand side's residual is undone for it.  On return p->gm.y holds y, rr the formed
// residuals and it the Krylov dimensions summed over the sweeps.  Right-hand sides that are done
// enter the next GMRES with b = 0, which freezes them at zero iterations.
static cudaError_t refine(ifgf_plan_t* p, int nrhs, double tol, int max_iter, const MatvecFn& mv,
                          const MatvecFn* pc, bool scaled, double cm, double cj, std::vector<int>& it,
                          std::vector<double>& rr, cudaStream_t s) {
  GmresWork& G = p->gm;
  ifgf_plan_t* q = p->resid ? p->resid : p;   // the map that forms the residual
  if (q->poisoned) return cudaErrorInvalidResourceHandle;
  const size_t n2 = 8 * (size_t)p->N;   // doubles per right-hand side
  const size_t bytes = sizeof(double) * n2 * nrhs;
  // b_orig: the right-hand side; y_acc: the solution so far; G.b: after each GMRES, a copy of
  // y_acc before the correction (restored exactly for a right-hand side the sweep did not help)
  cudaError_t e = cudaMemcpyAsync(G.b_orig, G.b, bytes, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(G.y_acc, G.y, bytes, cudaMemcpyDeviceToDevice, s);
  std::vector<double> prev(nrhs, HUGE_VAL);
  std::vector<int> go(nrhs, 0), it2(nrhs, 0);
  std::vector<double> rr2(nrhs, 0.0);
  for (int sweep = 0; e == cudaSuccess; ++sweep) {
    e = forward(q, G.y_acc, G.w, nrhs, s);
    if (e == cudaSuccess) e = gmres_residual(p, nrhs, G.b_orig, G.w, G.w, s);   // r in G.w
    if (e == cudaSuccess) e = cudaMemcpyAsync(G.hres, G.scal, sizeof(double) * 8 * nrhs, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) break;
    double tol_in = 0.5;
    int active = 0;
    for (int r = 0; r < nrhs && e == cudaSuccess; ++r) {
      const double nb = G.hres[8 * r + 4], nr = G.hres[8 * r + 3];
      const double rel = nb > 0 ? nr / nb : 0.0;
      if (sweep > 0 && go[r] && !(rel < prev[r])) {
        // no gain: back to the solution before this sweep (its residual is prev[r])
        e = cudaMemcpyAsync(G.y_acc + r * n2, G.b + r * n2, sizeof(double) * n2, cudaMemcpyDeviceToDevice, s);
        go[r] = 0;
      } else {
        go[r] = rel > tol && (sweep == 0 || rel < 0.9 * prev[r]) && sweep < p->desc.refine;
        rr[r] = rel;
        prev[r] = rel;
      }
      if (go[r]) {
        ++active;
        tol_in = std::min(tol_in, 0.5 * tol / rel);
      }
    }
    if (e != cudaSuccess || active == 0) break;
    // GMRES on A d = r for the right-hand sides still going (b = 0 freezes the others at d = 0)
    e = cudaMemcpyAsync(G.b, G.w, bytes, cudaMemcpyDeviceToDevice, s);
    for (int r = 0; r < nrhs && e == cudaSuccess; ++r)
      if (!go[r]) e = cudaMemsetAsync(G.b + r * n2, 0, sizeof(double) * n2, s);
    if (e == cudaSuccess)
      e = gmres_run(p, mv, nrhs, std::max(tol_in, 1e-14), max_iter, it2.data(), rr2.data(), s, pc);
    if (e == cudaSuccess && scaled) e = launch_block_scale(p->N, nrhs, cm, cj, G.y, G.y, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(G.b, G.y_acc, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = gmres_accumulate(p, nrhs, G.y, G.y_acc, s, false);
    for (int r = 0; r < nrhs; ++r) it[r] += it2[r];
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(G.y, G.y_acc, bytes, cudaMemcpyDeviceToDevice, s);
  return e;
}

static ifgf_status solve_impl(ifgf_plan p, int32_t nrhs, const void* inc, double tol, int32_t max_iter, void* y,
                              int32_t* iters, double* relres, ifgf_stream stream, bool flexible) {
  if (!p || !inc || !y || !(tol > 0) || max_iter < 1) return IFGF_EINVAL;
  if (flexible && p->pc.hidden == 0 && !p->bj.inv) return IFGF_EINVAL;
  if (nrhs < 1 || nrhs > p->batch) return IFGF_EINVAL;
  if (max_iter > p->gm.max_iter) return IFGF_EINVAL;
  if (p->poisoned) return IFGF_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n4 = 4 * (size_t)p->N;
  cudaError_t e = cudaSuccess;
  const double* dinc = (const double*)inc;
  if (!is_device_ptr(inc)) {
    e = cudaMemcpyAsync(p->gm.inc, inc, sizeof(double) * 12 * (size_t)p->N * nrhs, cudaMemcpyHostToDevice, s);
    dinc = p->gm.inc;
  }
  if (e == cudaSuccess) e = launch_rhs(p, dinc, p->gm.b, s, nrhs);
  ++p->launches;
  std::vector<int> it(nrhs, 0);
  std::vector<double> rr(nrhs, 0.0);
  if (e == cudaSuccess) {
    // right scaling: GMRES iterates on A D (D constant on the m and j blocks), y = D z after
    const bool scaled = p->desc.gmres_scaling == 1 && !flexible;
    const double cm = 2.0 / (p->desc.mu_ext + p->desc.mu_int), cj = 2.0 / (p->desc.eps_ext + p->desc.eps_int);
    MatvecFn mv = [p, nrhs, scaled, cm, cj](const double* v, double* w, cudaStream_t st) {
      if (!scaled) return forward(p, v, w, nrhs, st);
      double* tmp = p->gm.inc;   // [nrhs][6N] complex: free once the right-hand side is formed
      cudaError_t er = launch_block_scale(p->N, nrhs, cm, cj, v, tmp, st);
      ++p->launches;
      return er != cudaSuccess ? er : forward(p, tmp, w, nrhs, st);
    };
    MatvecFn pc = [p, nrhs](const double* v, double* z, cudaStream_t st) { return precond_apply(p, nrhs, v, z, st); };
    e = gmres_run(p, mv, nrhs, tol, max_iter, it.data(), rr.data(), s, flexible ? &pc : nullptr);
    if (e == cudaSuccess && scaled) e = launch_block_scale(p->N, nrhs, cm, cj, p->gm.y, p->gm.y, s);
    if (e == cudaSuccess && p->desc.refine > 0)
      e = refine(p, nrhs, tol, max_iter, mv, flexible ? &pc : nullptr, scaled, cm, cj, it, rr, s);
  }
  if (e == cudaSuccess) {
    if (is_device_ptr(y))
      e = cudaMemcpyAsync(y, p->gm.y, sizeof(double) * 2 * n4 * nrhs, cudaMemcpyDeviceToDevice, s);
    else
      e = cudaMemcpyAsync(y, p->gm.y, sizeof(double) * 2 * n4 * nrhs, cudaMemcpyDeviceToHost, s);
  }
  int word = 0;
  if (e == cudaSuccess) e = take_status_word(p, s, &word);
  if (e != cudaSuccess) {
    set_last_cuda_error(e, "bie_solve", __FILE__, __LINE__);
    p->poisoned = true;
    return IFGF_ECUDA;
  }
  if (word != 0) {
    set_status_detail(IFGF_ETIMEOUT, kTimeoutMsg);
    return IFGF_ETIMEOUT;
  }
  bool all = true;
  for (int r = 0; r < nrhs; ++r) {
    if (iters) iters[r] = it[r];
    if (relres) relres[r] = rr[r];
    all = all && rr[r] <= tol;
  }
  return all ? IFGF_OK : IFGF_ENOCONV;
}

ifgf_status ifgf_plan_check(ifgf_plan p, ifgf_stream stream) {
  if (!p) return IFGF_EINVAL;
  if (p->poisoned) return IFGF_ECUDA;
  int word = 0;
  cudaError_t e = take_status_word(p, (cudaStream_t)stream, &word);
  if (e != cudaSuccess) {
    set_last_cuda_error(e, "ifgf_plan_check", __FILE__, __LINE__);
    p->poisoned = true;
    return IFGF_ECUDA;
  }
  if (word != 0) {
    set_status_detail(IFGF_ETIMEOUT, kTimeoutMsg);
    return IFGF_ETIMEOUT;
  }
  return IFGF_OK;
}

static void unlink_residual(ifgf_plan_t* p) {
  if (!p->resid) return;
  auto& v = p->resid->resid_of;
  v.erase(std::remove(v.begin(), v.end(), p), v.end());
  p->resid = nullptr;
}

ifgf_status ifgf_plan_set_residual(ifgf_plan p, ifgf_plan r) {
  if (!p || r == p) return IFGF_EINVAL;
  if (r && (r->N != p->N || r->batch < p->batch || r->resid || !p->resid_of.empty())) return IFGF_EINVAL;
  try {
    if (r) r->resid_of.reserve(r->resid_of.size() + 1);
  } catch (const std::bad_alloc&) {
    return IFGF_ENOMEM;
  }
  unlink_residual(p);
  if (r) {
    r->resid_of.push_back(p);
    p->resid = r;
  }
  return IFGF_OK;
}

ifgf_status ifgf_plan_inject(ifgf_plan p, int32_t which) {
  if (!p || which < 0 || which > 1) return IFGF_EINVAL;
  p->inject = which;
  return IFGF_OK;
}

ifgf_status bie_rhs(ifgf_plan p, int32_t nrhs, const void* inc, void* b, ifgf_stream stream) {
  if (!p || !inc || !b || nrhs < 1) return IFGF_EINVAL;
  if (p->poisoned) return IFGF_ECUDA;
  cudaError_t e = launch_rhs(p, (const double*)inc, (double*)b, (cudaStream_t)stream, nrhs);
  if (e != cudaSuccess) {
    set_last_cuda_error(e, "bie_rhs", __FILE__, __LINE__);
    p->poisoned = true;
    return IFGF_ECUDA;
  }
  return IFGF_OK;
}

// No C++ exception leaves the C ABI: a failed host allocation is IFGF_ENOMEM.
ifgf_status bie_solve_batch(ifgf_plan p, int32_t nrhs, const void* inc, double tol, int32_t max_iter, void* y,
                            int32_t* iters, double* relres, ifgf_stream stream) {
  try {
    return solve_impl(p, nrhs, inc, tol, max_iter, y, iters, relres, stream, false);
  } catch (const std::bad_alloc&) {
    return IFGF_ENOMEM;
  } catch (const std::exception& e) {
    set_status_detail(IFGF_EINTERNAL, e.what());
    return IFGF_EINTERNAL;
  } catch (...) {
    set_status_detail(IFGF_EINTERNAL, "bie_solve_batch: unknown exception");
    return IFGF_EINTERNAL;
  }
}

ifgf_status bie_solve_precond(ifgf_plan p, int32_t nrhs, const void* inc, double tol, int32_t max_iter, void* y,
                              int32_t* iters, double* relres, ifgf_stream stream) {
  try {
    return solve_impl(p, nrhs, inc, tol, max_iter, y, iters, relres, stream, true);
  } catch (const std::bad_alloc&) {
    return IFGF_ENOMEM;
  } catch (const std::exception& e) {
    set_status_detail(IFGF_EINTERNAL, e.what());
    return IFGF_EINTERNAL;
  } catch (...) {
    set_status_detail(IFGF_EINTERNAL, "bie_solve_precond: unknown exception");
    return IFGF_EINTERNAL;
  }
}

ifgf_status ifgf_precond_attach(ifgf_plan p, int32_t hidden, const float* W1, const float* b1, const float* W2,
                                const float* b2) {
  if (!p || hidden < 1 || hidden > 512 || !W1 || !b1 || !W2 || !b2) return IFGF_EINVAL;
  if (p->poisoned) return IFGF_ECUDA;
  Precond& M = p->pc;
  const int in = 8 * p->nc * p->nc;
  if (M.hidden != 0 && M.hidden != hidden) return IFGF_EINVAL;
  try {
    Alloc A{p};
    if (M.hidden == 0) {
      M.in = in;
      M.W1 = A.dev<float>((size_t)in * hidden);
      M.b1 = A.dev<float>(hidden);
      M.W2 = A.dev<float>((size_t)in * hidden);
      M.b2 = A.dev<float>(in);
      M.W1h = A.dev<uint16_t>((size_t)in * hidden);
      M.W2h = A.dev<uint16_t>((size_t)in * hidden);
      M.Z = A.dev<double>(2 * 4 * (size_t)p->N * (p->gm.max_iter + 1) * p->batch);
    }
    check(cudaMemcpy(M.W1, W1, sizeof(float) * in * hidden, cudaMemcpyHostToDevice), "weights");
    check(cudaMemcpy(M.b1, b1, sizeof(float) * hidden, cudaMemcpyHostToDevice), "weights");
    check(cudaMemcpy(M.W2, W2, sizeof(float) * in * hidden, cudaMemcpyHostToDevice), "weights");
    check(cudaMemcpy(M.b2, b2, sizeof(float) * in, cudaMemcpyHostToDevice), "weights");
    M.hidden = hidden;
    M.adam_t = 0;
    if (M.tw.batch > 0) {   // restart the optimiser
      check(cudaMemset(M.tw.mW1, 0, sizeof(float) * in * hidden), "adam");
      check(cudaMemset(M.tw.vW1, 0, sizeof(float) * in * hidden), "adam");
      check(cudaMemset(M.tw.mW2, 0, sizeof(float) * in * hidden), "adam");
      check(cudaMemset(M.tw.vW2, 0, sizeof(float) * in * hidden), "adam");
      check(cudaMemset(M.tw.mb1, 0, sizeof(float) * hidden), "adam");
      check(cudaMemset(M.tw.vb1, 0, sizeof(float) * hidden), "adam");
      check(cudaMemset(M.tw.mb2, 0, sizeof(float) * in), "adam");
      check(cudaMemset(M.tw.vb2, 0, sizeof(float) * in), "adam");
    }
    check(mlp_refresh_bf16(p, nullptr), "bf16 weights");
    check(cudaDeviceSynchronize(), "precond attach");
  } catch (const std::bad_alloc&) {
    return IFGF_ENOMEM;
  } catch (const std::exception&) {
    return IFGF_ECUDA;
  }
  return IFGF_OK;
}

ifgf_status ifgf_precond_get(ifgf_plan p, float* W1, float* b1, float* W2, float* b2) {
  if (!p || p->pc.hidden == 0) return IFGF_EINVAL;
  const Precond& M = p->pc;
  const size_t n1 = (size_t)M.in * M.hidden;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess && W1) e = cudaMemcpy(W1, M.W1, sizeof(float) * n1, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && b1) e = cudaMemcpy(b1, M.b1, sizeof(float) * M.hidden, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && W2) e = cudaMemcpy(W2, M.W2, sizeof(float) * n1, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && b2) e = cudaMemcpy(b2, M.b2, sizeof(float) * M.in, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    set_last_cuda_error(e, "ifgf_precond_get", __FILE__, __LINE__);
    return IFGF_ECUDA;
  }
  return IFGF_OK;
}

ifgf_status ifgf_precond_apply(ifgf_plan p, int32_t nrhs, const void* v, void* z, ifgf_stream stream) {
  if (!p || !v || !z || v == z || (p->pc.hidden == 0 && !p->bj.inv) || nrhs < 1 || nrhs > p->batch)
    return IFGF_EINVAL;
  if (p->poisoned) return IFGF_ECUDA;
  cudaError_t e = precond_apply(p, nrhs, (const double*)v, (double*)z, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    set_last_cuda_error(e, "ifgf_precond_apply", __FILE__, __LINE__);
    p->poisoned = true;
    return IFGF_ECUDA;
  }
  return IFGF_OK;
}

ifgf_status ifgf_precond_features(ifgf_plan p, int32_t nrhs, const void* v, const void* e, float* X, float* T,
                                  ifgf_stream stream) {
  if (!p || !v || !e || !X || !T || p->pc.hidden == 0 || nrhs < 1) return IFGF_EINVAL;
  if (p->poisoned) return IFGF_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  double* base = nullptr;   // with block Jacobi: the targets are the error left by its product
  cudaError_t err = cudaSuccess;
  if (p->bj.inv) {
    if (nrhs > p->batch) return IFGF_EINVAL;
    if (cudaMalloc(&base, sizeof(double) * 8 * (size_t)p->N * nrhs) != cudaSuccess) {
      cudaGetLastError();
      return IFGF_ENOMEM;
    }
    err = launch_bj_apply(p, nrhs, (const double*)v, base, s);
  }
  if (err == cudaSuccess) err = launch_mlp_features(p, nrhs, (const double*)v, (const double*)e, X, T, s, base);
  if (base) {
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    cudaFree(base);
  }
  if (err != cudaSuccess) {
    set_last_cuda_error(err, "ifgf_precond_features", __FILE__, __LINE__);
    p->poisoned = true;
    return IFGF_ECUDA;
  }
  return IFGF_OK;
}

ifgf_status ifgf_precond_block_jacobi(ifgf_plan p, ifgf_stream stream) {
  if (!p) return IFGF_EINVAL;
  if (p->poisoned) return IFGF_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const int m = 4 * p->nc * p->nc;
  int* ipiv = nullptr;
  int* err_dev = nullptr;
  try {
    Alloc A{p};
    if (!p->bj.inv) {
      p->bj.inv = A.dev<double>(2 * (size_t)p->P * m * m);
      p->bj.m = m;
    }
    if (!p->pc.Z)   // the flexible-GMRES basis (also allocated by ifgf_precond_attach)
      p->pc.Z = A.dev<double>(2 * 4 * (size_t)p->N * (p->gm.max_iter + 1) * p->batch);
  } catch (const std::exception&) {
    cudaGetLastError();
    return IFGF_ENOMEM;
  }
  if (cudaMalloc(&ipiv, sizeof(int) * (size_t)p->P * m) != cudaSuccess ||
      cudaMalloc(&err_dev, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(ipiv);
    return IFGF_ENOMEM;
  }
  // probe buffers: the first two right-hand-side blocks of the Krylov basis (free between solves)
  double* yb = p->gm.V;
  double* ob = p->gm.V + 8 * (size_t)p->N * p->batch;
  int herr = 0;
  cudaError_t e = cudaMemsetAsync(err_dev, 0, sizeof(int), s);
  if (e == cudaSuccess) e = bj_build(p, yb, ob, ipiv, err_dev, s);
  if (e == cudaSuccess) e = cudaMemcpy(&herr, err_dev, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(ipiv);
  cudaFree(err_dev);
  if (e != cudaSuccess) {
    set_last_cuda_error(e, "ifgf_precond_block_jacobi", __FILE__, __LINE__);
    p->poisoned = true;
    return IFGF_ECUDA;
  }
  if (herr != 0) {
    p->bj.inv = nullptr;   // stays allocated with the plan; not used
    set_status_detail(IFGF_EINTERNAL, "ifgf_precond_block_jacobi: a diagonal block is singular");
    return IFGF_EINTERNAL;
  }
  return IFGF_OK;
}

ifgf_status ifgf_precond_train(ifgf_plan p, int64_t nsamples, const float* X, const float* T, int32_t steps,
                               int32_t batch, float lr, uint64_t seed, float* loss, ifgf_stream stream) {
  if (!p || !X || !T || nsamples < 1 || steps < 1 || batch < 1 || batch > 65535 || !(lr > 0)) return IFGF_EINVAL;
  if (p->pc.hidden == 0) return IFGF_EINVAL;
  if (p->poisoned) return IFGF_ECUDA;
  Precond& M = p->pc;
  TrainWork& W = M.tw;
  const int in = M.in, H = M.hidden;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    Alloc A{p};
    if (W.batch == 0) {   // optimiser state and gradients: sized by the network
      const size_t n1 = (size_t)in * H;
      W.gW1 = A.dev<float>(n1); W.gW2 = A.dev<float>(n1); W.gb1 = A.dev<float>(H); W.gb2 = A.dev<float>(in);
      W.mW1 = A.dev<float>(n1); W.vW1 = A.dev<float>(n1); W.mW2 = A.dev<float>(n1); W.vW2 = A.dev<float>(n1);
      W.mb1 = A.dev<float>(H); W.vb1 = A.dev<float>(H); W.mb2 = A.dev<float>(in); W.vb2 = A.dev<float>(in);
      for (float* a : {W.mW1, W.vW1, W.mW2, W.vW2}) check(cudaMemset(a, 0, sizeof(float) * n1), "adam");
      for (float* a : {W.mb1, W.vb1}) check(cudaMemset(a, 0, sizeof(float) * H), "adam");
      for (float* a : {W.mb2, W.vb2}) check(cudaMemset(a, 0, sizeof(float) * in), "adam");
    }
    if (batch > W.batch) {   // minibatch scratch (grows, never shrinks)
      W.Xb = A.dev<float>((size_t)batch * in); W.Tb = A.dev<float>((size_t)batch * in);
      W.Y = A.dev<float>((size_t)batch * in); W.dY = A.dev<float>((size_t)batch * in);
      W.Hpre = A.dev<float>((size_t)batch * H); W.H1 = A.dev<float>((size_t)batch * H);
      W.dH = A.dev<float>((size_t)batch * H);
      W.batch = batch;
    }
    if (steps > M.loss_cap) {
      M.loss = A.dev<float>(steps);
      M.loss_cap = steps;
    }
    check(cudaMemsetAsync(M.loss, 0, sizeof(float) * steps, s), "loss");
    check(mlp_train(p, nsamples, X, T, steps, batch, lr, seed, M.loss, s), "training");
    if (loss) check(cudaMemcpyAsync(loss, M.loss, sizeof(float) * steps, cudaMemcpyDeviceToHost, s), "loss");
    check(cudaStreamSynchronize(s), "training");
  } catch (const std::bad_alloc&) {
    return IFGF_ENOMEM;
  } catch (const std::exception&) {
    p->poisoned = true;
    return IFGF_ECUDA;
  }
  return IFGF_OK;
}

ifgf_status bie_solve(ifgf_plan p, const void* inc, double tol, int32_t max_iter, void* y, int32_t* iters,
                      double* relres, ifgf_stream stream) {
  return bie_solve_batch(p, 1, inc, tol, max_iter, y, iters, relres, stream);
}

ifgf_status bie_solve_many(int32_t nplans, const ifgf_plan* plans, const int32_t* nrhs, const void* const* incs,
                           double tol, int32_t max_iter, void* const* ys, int32_t* const* iters,
                           double* const* relres, ifgf_status* status, const ifgf_stream* streams) {
  if (nplans < 1 || !plans || !nrhs || !incs || !ys) return IFGF_EINVAL;
  for (int i = 0; i < nplans; ++i) {
    if (!plans[i] || !incs[i] || !ys[i]) return IFGF_EINVAL;
    for (int j = 0; j < i; ++j) {
      if (plans[j] == plans[i]) return IFGF_EINVAL;
      if (streams && streams[i] && streams[j] == streams[i]) return IFGF_EINVAL;
      // a residual plan's buffers serve one solve at a time
      if (plans[i]->resid && (plans[i]->resid == plans[j] || plans[i]->resid == plans[j]->resid))
        return IFGF_EINVAL;
      if (plans[j]->resid == plans[i]) return IFGF_EINVAL;
    }
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return IFGF_ECUDA;
  std::vector<ifgf_status> st;
  try {
    st.assign(nplans, IFGF_OK);
  } catch (const std::bad_alloc&) {
    return IFGF_ENOMEM;
  }
  // the message a failed solve leaves in its worker thread's status strings, handed back to this
  // thread (the first failure in plan order) after the join
  std::vector<std::string> msg;
  try {
    msg.assign(nplans, std::string());
  } catch (const std::bad_alloc&) {
    return IFGF_ENOMEM;
  }
  auto work = [&](int i) {
    if (cudaSetDevice(dev) != cudaSuccess) {
      st[i] = IFGF_ECUDA;
      return;
    }
    cudaStream_t s = streams ? (cudaStream_t)streams[i] : nullptr;
    const bool own = (s == nullptr);
    if (own && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      st[i] = IFGF_ECUDA;
      return;
    }
    st[i] = bie_solve_batch(plans[i], nrhs[i], incs[i], tol, max_iter, ys[i], iters ? iters[i] : nullptr,
                            relres ? relres[i] : nullptr, (ifgf_stream)s);
    if (st[i] != IFGF_OK && st[i] != IFGF_ENOCONV) {
      try {
        msg[i] = ifgf_status_string(st[i]);
      } catch (...) {
      }
    }
    if (own) cudaStreamDestroy(s);
  };
  // one host thread per plan; a solve whose thread cannot be started runs here afterwards
  std::vector<std::thread> workers;
  int started = 0;
  try {
    workers.reserve(nplans);
    for (; started < nplans; ++started) workers.emplace_back(work, started);
  } catch (...) {
  }
  for (int i = started; i < nplans; ++i) work(i);
  for (auto& w : workers) w.join();
  for (int i = 0; i < nplans; ++i)
    if (!msg[i].empty()) {
      if (st[i] == IFGF_ECUDA)
        snprintf(g_last_err, sizeof(g_last_err), "%s", msg[i].c_str());
      else
        set_status_detail(st[i], msg[i].c_str());
      break;
    }
  ifgf_status out = IFGF_OK;
  for (int i = 0; i < nplans; ++i) {
    if (status) status[i] = st[i];
    if (st[i] != IFGF_OK && st[i] != IFGF_ENOCONV && (out == IFGF_OK || out == IFGF_ENOCONV)) out = st[i];
    else if (st[i] == IFGF_ENOCONV && out == IFGF_OK) out = IFGF_ENOCONV;
  }
  return out;
}

ifgf_status ifgf_plan_stats(ifgf_plan p, ifgf_stats* st) {
  if (!p || !st) return IFGF_EINVAL;
  *st = p->stats;
  return IFGF_OK;
}

ifgf_status ifgf_set_timing(ifgf_plan p, int32_t enable) {
  if (!p) return IFGF_EINVAL;
  if (timer_flush(p) != cudaSuccess) return IFGF_ECUDA;
  p->timer.on = enable != 0;
  for (int k = 0; k < TK_COUNT; ++k) {
    p->timer.total_ms[k] = 0;
    p->timer.calls[k] = 0;
  }
  p->launches = 0;
  return IFGF_OK;
}

ifgf_status ifgf_get_timing(ifgf_plan p, double* ms, int64_t* calls, int64_t* launches) {
  if (!p) return IFGF_EINVAL;
  if (timer_flush(p) != cudaSuccess) return IFGF_ECUDA;
  for (int k = 0; k < TK_COUNT; ++k) {
    if (ms) ms[k] = p->timer.total_ms[k];
    if (calls) calls[k] = p->timer.calls[k];
  }
  if (launches) *launches = p->launches;
  return IFGF_OK;
}

ifgf_status ifgf_plan_tree(ifgf_plan p, ifgf_tree* out) {
  if (!p || !out) return IFGF_EINVAL;
  *out = &p->tree;
  return IFGF_OK;
}

}  // extern "C"
