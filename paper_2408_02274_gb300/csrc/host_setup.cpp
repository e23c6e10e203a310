// One-time host setup of the IFGF octree and cone segments (Sec. III-F):
// relevant boxes (Eq. rele_boxes), neighbours and cousins (Eqs. box_neighbor,
// box_cousin), cone-segment counts per level (Remark 2), relevant cone
// segments (Eq. rele_cone_d) and the per-target evaluation lists of step 3 of
// the algorithm summary.  Integer and FP64 geometric work only.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <exception>
#include <new>
#include <stdexcept>
#include <thread>
#include <unordered_map>

#include "host_setup.h"

namespace ifgf {

static uint64_t spread3(uint64_t v) {
  v &= 0x1fffffULL;
  v = (v | (v << 32)) & 0x1f00000000ffffULL;
  v = (v | (v << 16)) & 0x1f0000ff0000ffULL;
  v = (v | (v << 8)) & 0x100f00f00f00f00fULL;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ULL;
  v = (v | (v << 2)) & 0x1249249249249249ULL;
  return v;
}
static uint64_t morton(int x, int y, int z) {
  return spread3((uint64_t)x) | (spread3((uint64_t)y) << 1) | (spread3((uint64_t)z) << 2);
}

// Cone segment of the point (x, y, z) relative to a box centre (Eq. box_cone_seg):
// half-open cells in s, theta, phi, clamped at the top (reading of the cone intervals).
cone_key cone_of(const ConeGeom& cg, double x, double y, double z) {
  double rho = std::sqrt(x * x + y * y);
  double r = std::sqrt(rho * rho + z * z);
  double s = cg.h / r;
  double th = std::atan2(rho, z);
  double ph = std::atan2(y, x);
  if (ph < 0) ph += 2 * kPi;
  int g1 = (int)std::floor(s / cg.ds());
  int g2 = (int)std::floor(th / cg.dth());
  int g3 = (int)std::floor(ph / cg.dth());
  g1 = std::min(std::max(g1, 0), cg.ns - 1);
  g2 = std::min(std::max(g2, 0), cg.na - 1);
  g3 = std::min(std::max(g3, 0), 2 * cg.na - 1);
  return cone_encode(g1, g2, g3);
}

// The cells of cone_of without its two atan2: theta by comparing cos(theta) = z / r, and phi by
// comparing cos(phi) = x / rho (on the side given by the sign of y), with the cosines of the cell
// boundaries k pi / na.  Where a cosine lies within kMargin of a boundary's cosine (there the
// rounding of either computation could decide the cell), on the axis (rho = 0), on the plane
// y = 0 and for r = 0, cone_of itself decides, so the result is always cone_of's: away from the
// margin the true angle is more than kMargin from the boundary (|d cos / d angle| <= 1), far
// beyond the few-ulp errors of atan2, of the quotient by the cell width and of the cosines.
// The radial cell is computed with cone_of's own operations.
struct ConeClassifier {
  static constexpr double kMargin = 4e-12;
  ConeGeom cg;
  double ds, inv_dth;
  std::vector<double> cb;   // cos(k dth), k = 0 .. na (decreasing)
  explicit ConeClassifier(const ConeGeom& g) : cg(g), ds(g.ds()), inv_dth(1.0 / g.dth()), cb(g.na + 1) {
    for (int k = 0; k <= g.na; ++k) cb[k] = std::cos(k * g.dth());
  }
  // k with cb[k] >= c > cb[k + 1] (0 <= k < na), or -1 where c is within the margin of either.
  // Few cells: bisection.  Many: the search starts from acos(c) ~ sqrt(1 - |c|) p(|c|), p a
  // least-squares cubic on [0, 1] (error < 2e-4 rad, under one cell on every level), and the
  // table steps make k exact.
  int cell(double c) const {
    if (!(c < cb[0] - kMargin) || !(c > cb[cg.na] + kMargin)) return -1;
    int k;
    if (cg.na <= 12) {          // a few bisection steps
      int lo = 0, hi = cg.na;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (cb[mid] >= c) lo = mid; else hi = mid;
      }
      k = lo;
    } else {
      const double a = std::fabs(c);
      double t = std::sqrt(1.0 - a) * (1.57065637 + a * (-0.21156586 + a * (0.07332775 - 0.01831046 * a)));
      if (c < 0) t = kPi - t;
      k = std::min(std::max((int)(t * inv_dth), 0), cg.na - 1);
      while (k > 0 && cb[k] < c) --k;
      while (k < cg.na - 1 && cb[k + 1] >= c) ++k;
    }
    if (!(std::fabs(c - cb[k]) >= kMargin) || !(std::fabs(c - cb[k + 1]) >= kMargin)) return -1;
    return k;
  }
  // cell(c), trying first the previous point's cell `hint` (kept only when c lies inside it by
  // more than the margin); hint is updated
  int cell(double c, int& hint) const {
    if (hint >= 0 && c < cb[hint] - kMargin && c > cb[hint + 1] + kMargin) return hint;
    hint = cell(c);
    return hint;
  }
  cone_key operator()(double x, double y, double z) const {
    int h2 = -1, h3 = -1;
    return (*this)(x, y, z, h2, h3);
  }
  // with the theta and phi cells of the previous point as hints (updated; -1: none)
  cone_key operator()(double x, double y, double z, int& h2, int& h3) const {
    double rho = std::sqrt(x * x + y * y);
    double r = std::sqrt(rho * rho + z * z);
    if (!(rho > 0) || y == 0.0) return cone_of(cg, x, y, z);
    const int g2 = cell(z / r, h2);
    int g3 = cell(x / rho, h3);
    if (g2 < 0 || g3 < 0) return cone_of(cg, x, y, z);
    if (y < 0) g3 = 2 * cg.na - 1 - g3;   // phi = 2 pi - psi with cos(psi) = x / rho
    double s = cg.h / r;
    int g1 = (int)std::floor(s / ds);
    g1 = std::min(std::max(g1, 0), cg.ns - 1);
    return cone_encode(g1, g2, g3);
  }
};

// Interpolation point q of a cone segment relative to the box centre:
// tensor product of Ps x Pa x Pa open Chebyshev nodes mapped to the cone domain.
void interp_point(const ConeGeom& cg, cone_key cone, int q, double* X) {
  int g1, g2, g3;
  cone_decode(cone, &g1, &g2, &g3);
  int is = q / (kPa * kPa), it = (q / kPa) % kPa, ip = q % kPa;
  double s = (g1 + 0.5 * (1.0 + cheb_node(is, kPs))) * cg.ds();
  double th = (g2 + 0.5 * (1.0 + cheb_node(it, kPa))) * cg.dth();
  double ph = (g3 + 0.5 * (1.0 + cheb_node(ip, kPa))) * cg.dth();
  double r = cg.h / s;
  X[0] = r * std::sin(th) * std::cos(ph);
  X[1] = r * std::sin(th) * std::sin(ph);
  X[2] = r * std::cos(th);
}

// interp_point for every cone of one level from tables: the radius of each (radial cell, radial
// node) and the sines and cosines of each (angular cell, angular node), formed with
// interp_point's own expressions, so the points are interp_point's to the bit.
struct ConePoints {
  ConeGeom cg;
  std::vector<double> r, st, ct, sp, cp;   // [ns][kPs], [na][kPa] (theta), [2na][kPa] (phi)
  explicit ConePoints(const ConeGeom& g)
      : cg(g), r((size_t)g.ns * kPs), st((size_t)g.na * kPa), ct(st.size()), sp((size_t)2 * g.na * kPa),
        cp(sp.size()) {
    for (int g1 = 0; g1 < g.ns; ++g1)
      for (int i = 0; i < kPs; ++i) r[(size_t)g1 * kPs + i] = g.h / ((g1 + 0.5 * (1.0 + cheb_node(i, kPs))) * g.ds());
    for (int g2 = 0; g2 < g.na; ++g2)
      for (int i = 0; i < kPa; ++i) {
        const double th = (g2 + 0.5 * (1.0 + cheb_node(i, kPa))) * g.dth();
        st[(size_t)g2 * kPa + i] = std::sin(th);
        ct[(size_t)g2 * kPa + i] = std::cos(th);
      }
    for (int g3 = 0; g3 < 2 * g.na; ++g3)
      for (int i = 0; i < kPa; ++i) {
        const double ph = (g3 + 0.5 * (1.0 + cheb_node(i, kPa))) * g.dth();
        sp[(size_t)g3 * kPa + i] = std::sin(ph);
        cp[(size_t)g3 * kPa + i] = std::cos(ph);
      }
  }
  void operator()(cone_key cone, int q, double* X) const {
    int g1, g2, g3;
    cone_decode(cone, &g1, &g2, &g3);
    const int is = q / (kPa * kPa), it = (q / kPa) % kPa, ip = q % kPa;
    const double rr = r[(size_t)g1 * kPs + is], s_t = st[(size_t)g2 * kPa + it];
    X[0] = rr * s_t * cp[(size_t)g3 * kPa + ip];
    X[1] = rr * s_t * sp[(size_t)g3 * kPa + ip];
    X[2] = rr * ct[(size_t)g2 * kPa + it];
  }
};

// Group (0 .. kUpGroups-1) of interpolation point q = (is * 5 + it) * 5 + ip: the points ranked
// by angular position (it, ip) in snake order (ip reversed on odd it), radial index is within a
// position, cut into chunks of 19, 19, 19 and 18 points (balanced warps; neighbouring points,
// which mostly share child cones, stay together).
static int up_group(int q) {
  const int is = q / (kPa * kPa), a = q % (kPa * kPa), it = a / kPa, ip = a % kPa;
  const int rank = (it * kPa + ((it & 1) ? kPa - 1 - ip : ip)) * kPs + is;
  return rank < 19 ? 0 : (rank < 38 ? 1 : (rank < 57 ? 2 : 3));
}

static void box_center(const HostTree& t, int d, const std::array<int, 3>& ic, double* c) {
  double H = t.lv[d].H;
  for (int a = 0; a < 3; ++a) c[a] = t.corner[a] + H * (ic[a] + 0.5);
}

// Host threads for the setup: IFGF_HOST_THREADS when set to a positive number (a cap for
// shared hosts), else the hardware concurrency; at most 64.  The tables built do not depend on it.
static int host_threads() {
  int64_t n = std::max(1u, std::thread::hardware_concurrency());
  if (const char* e = std::getenv("IFGF_HOST_THREADS")) {
    const long v = std::strtol(e, nullptr, 10);
    if (v > 0) n = v;
  }
  return (int)std::min<int64_t>(n, 64);
}

// f(begin, end) over [0, n) split into contiguous static chunks, one per host thread; an
// exception thrown by a chunk is rethrown here after all threads have joined.
template <typename F>
static void parallel_for(int64_t n, F&& f) {
  const int nth = (int)std::max<int64_t>(1, std::min<int64_t>(host_threads(), n / 64 + 1));
  if (nth == 1) {
    f((int64_t)0, n);
    return;
  }
  std::vector<std::exception_ptr> err(nth);
  auto run = [&](int i) {
    try {
      f(n * i / nth, n * (i + 1) / nth);
    } catch (...) {
      err[i] = std::current_exception();
    }
  };
  std::vector<std::thread> th;
  int started = 1;
  try {
    for (; started < nth; ++started) th.emplace_back(run, started);
  } catch (...) {   // no more threads: the remaining chunks run here
  }
  for (int i = started; i < nth; ++i) run(i);
  run(0);
  for (auto& x : th) x.join();
  for (auto& e : err)
    if (e) std::rethrow_exception(e);
}

// Number of workers parallel_dynamic uses for n items.
static int dynamic_workers(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(host_threads(), n));
}

// f(worker, begin, end) over [0, n) in chunks of `chunk` items handed out on demand, for loops
// whose items differ widely in cost (boxes: a few large ones on the top levels, many small
// ones below).  Workers are numbered 0 .. dynamic_workers(n) - 1 for per-worker scratch; the
// result must not depend on which worker takes which chunk.
template <typename F>
static void parallel_dynamic(int64_t n, int64_t chunk, F&& f) {
  const int nth = dynamic_workers(n);
  std::atomic<int64_t> next{0};
  std::vector<std::exception_ptr> err(nth);
  auto run = [&](int w) {
    try {
      for (int64_t i0; (i0 = next.fetch_add(chunk)) < n;) f(w, i0, std::min(n, i0 + chunk));
    } catch (...) {
      err[w] = std::current_exception();
      next.store(n);
    }
  };
  std::vector<std::thread> th;
  int started = 1;
  try {
    for (; started < nth; ++started) th.emplace_back(run, started);
  } catch (...) {   // no more threads: worker 0 takes the remaining chunks
  }
  run(0);
  for (auto& x : th) x.join();
  for (auto& e : err)
    if (e) std::rethrow_exception(e);
}

void build_tree(HostTree& t, const double* x, int N, double leaf_size, int min_levels,
                double k_max, int ns0, int na0, int max_leaf_pts) {
  if (N <= 0) throw std::invalid_argument("no nodes");
  // levels are capped at 21: the Morton keys hold 21 bits per axis
  if (min_levels > 21) throw std::invalid_argument("min_levels above 21 (the octree has at most 21 levels)");
  for (int64_t i = 0; i < 3 * (int64_t)N; ++i)
    if (!std::isfinite(x[i])) throw std::invalid_argument("node coordinates must be finite");
  double lo[3] = {x[0], x[1], x[2]}, hi[3] = {x[0], x[1], x[2]};
  for (int i = 0; i < N; ++i)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], x[3 * i + a]);
      hi[a] = std::max(hi[a], x[3 * i + a]);
    }
  double ext = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
  if (!(ext > 0)) throw std::invalid_argument("degenerate bounding box");
  // level-1 cube: slightly larger than the bounding box, centred on it (reading R11)
  t.H1 = ext * (1.0 + 1e-9);
  for (int a = 0; a < 3; ++a) t.corner[a] = 0.5 * (lo[a] + hi[a]) - 0.5 * t.H1;
  int D = std::max(3, min_levels);
  while (t.H1 / std::ldexp(1.0, D - 1) > leaf_size && D < 21) ++D;
  // point-count leaf rule: refine until no leaf box holds more than max_leaf_pts points
  if (max_leaf_pts > 0) {
    std::unordered_map<uint64_t, int> count;
    while (D < 21) {
      count.clear();
      const double HD = t.H1 / std::ldexp(1.0, D - 1);
      const int nside = 1 << (D - 1);
      int mx = 0;
      for (int i = 0; i < N; ++i) {
        int c[3];
        for (int a = 0; a < 3; ++a)
          c[a] = std::min(nside - 1, std::max(0, (int)std::floor((x[3 * i + a] - t.corner[a]) / HD)));
        mx = std::max(mx, ++count[morton(c[0], c[1], c[2])]);
      }
      if (mx <= max_leaf_pts) break;
      ++D;
    }
  }
  t.D = D;
  t.lv.assign(D + 1, HostLevel());
  for (int d = 1; d <= D; ++d) {
    t.lv[d].d = d;
    t.lv[d].H = t.H1 / std::ldexp(1.0, d - 1);
    t.lv[d].h = 0.5 * std::sqrt(3.0) * t.lv[d].H;
  }
  // cone counts (Remark 2, reading R9): n_{.;d} = a_d n_{.;d+1}, a_d = 2 iff k_max H_d > 1/2;
  // the radial count is kept at least 2 n_{s;D+1} (reading R25: on low-frequency leaf levels,
  // k_max H_D <= 1/2, the radial profile of the factored field needs the finer s cells)
  int ns = ns0, na = na0;
  for (int d = D; d >= 1; --d) {
    int a = (k_max * t.lv[d].H > 0.5) ? 2 : 1;
    if (d >= 3) {
      ns *= a;
      na *= a;
    }
    t.lv[d].ns = (d >= 3) ? std::max(ns, 2 * ns0) : 0;
    t.lv[d].na = (d >= 3) ? na : 0;
    // a cone key holds g1 < ns and g3 < 2 na in 21 bits each
    if (d >= 3 && (t.lv[d].ns > (1 << kConeBits) || 2 * t.lv[d].na > (1 << kConeBits)))
      throw std::invalid_argument("cone-segment counts exceed the 21-bit cone key fields "
                                  "(k_max times the body size is too large for ns0, na0)");
  }
  // leaf keys and Morton order
  const int nside = 1 << (D - 1);
  const double HD = t.lv[D].H;
  t.leafc.resize(N);
  std::vector<uint64_t> key(N);
  for (int i = 0; i < N; ++i) {
    std::array<int, 3> k;
    for (int a = 0; a < 3; ++a) {
      int v = (int)std::floor((x[3 * i + a] - t.corner[a]) / HD);
      k[a] = std::min(std::max(v, 0), nside - 1);
    }
    t.leafc[i] = k;
    key[i] = morton(k[0], k[1], k[2]);
  }
  t.perm.resize(N);
  for (int i = 0; i < N; ++i) t.perm[i] = i;
  std::stable_sort(t.perm.begin(), t.perm.end(), [&](int a, int b) { return key[a] < key[b]; });
  t.iperm.resize(N);
  for (int s = 0; s < N; ++s) t.iperm[t.perm[s]] = s;
  // relevant boxes per level (Eq. rele_boxes): runs of equal key prefixes in Morton order
  t.box_of.assign(D + 1, std::vector<int>(N, -1));
  for (int d = D; d >= 1; --d) {
    HostLevel& L = t.lv[d];
    int shift = 3 * (D - d);
    uint64_t prev = ~0ULL;
    for (int s = 0; s < N; ++s) {
      uint64_t k = key[t.perm[s]] >> shift;
      if (k != prev) {
        if (!L.key.empty()) L.pt_end.push_back(s);
        L.key.push_back(k);
        L.pt_begin.push_back(s);
        const auto& lc = t.leafc[t.perm[s]];
        L.ic.push_back({lc[0] >> (D - d), lc[1] >> (D - d), lc[2] >> (D - d)});
        prev = k;
      }
      t.box_of[d][s] = (int)L.key.size() - 1;
    }
    L.pt_end.push_back(N);
    for (int b = 0; b < (int)L.key.size(); ++b) L.index[L.key[b]] = b;
  }
  // parents, children
  for (int d = 1; d <= D; ++d) {
    HostLevel& L = t.lv[d];
    int nb = (int)L.key.size();
    L.parent.assign(nb, -1);
    L.child.assign(nb, {-1, -1, -1, -1, -1, -1, -1, -1});
    if (d > 1) {
      HostLevel& Pp = t.lv[d - 1];
      for (int b = 0; b < nb; ++b) {
        int p = Pp.index.at(L.key[b] >> 3);
        L.parent[b] = p;
        int o = (L.ic[b][0] & 1) | ((L.ic[b][1] & 1) << 1) | ((L.ic[b][2] & 1) << 2);
        Pp.child[p][o] = b;
      }
    }
  }
  // neighbours (infinity-norm, reading R10) and cousins
  for (int d = 1; d <= D; ++d) {
    HostLevel& L = t.lv[d];
    int nb = (int)L.key.size();
    int side = 1 << (d - 1);
    L.nbr.assign(nb, {});
    for (int b = 0; b < nb; ++b) {
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            int X = L.ic[b][0] + dx, Y = L.ic[b][1] + dy, Z = L.ic[b][2] + dz;
            if (X < 0 || Y < 0 || Z < 0 || X >= side || Y >= side || Z >= side) continue;
            auto it = L.index.find(morton(X, Y, Z));
            if (it != L.index.end()) L.nbr[b].push_back(it->second);
          }
      std::sort(L.nbr[b].begin(), L.nbr[b].end());
    }
    L.cousin.assign(nb, {});
    if (d >= 2) {
      HostLevel& Pp = t.lv[d - 1];
      for (int b = 0; b < nb; ++b) {
        for (int pn : Pp.nbr[L.parent[b]])
          for (int o = 0; o < 8; ++o) {
            int c = Pp.child[pn][o];
            if (c < 0) continue;
            if (!std::binary_search(L.nbr[b].begin(), L.nbr[b].end(), c)) L.cousin[b].push_back(c);
          }
        std::sort(L.cousin[b].begin(), L.cousin[b].end());
      }
    }
  }
  // relevant cone segments, top-down from level 3 (Eq. rele_cone_d), and the
  // per-target evaluation lists of step 3 (cousin points of every source box).  Relevant
  // cones are kept per box as sorted key lists (the cone count of a level, ns * na * 2na,
  // is far too large for dense per-box maps on deep trees).  Every step runs over host
  // threads on disjoint outputs, so the tables do not depend on the thread count.
  std::vector<double> xs(3 * (size_t)N);   // node coordinates in sorted order
  parallel_for(N, [&](int64_t s0, int64_t s1) {
    for (int64_t s = s0; s < s1; ++s)
      for (int a = 0; a < 3; ++a) xs[3 * s + a] = x[3 * (size_t)t.perm[s] + a];
  });
  for (int d = 3; d <= D; ++d) {
    HostLevel& L = t.lv[d];
    ConeGeom cg = L.cg();
    const ConeClassifier cls(cg);
    const int nb = (int)L.key.size();
    // (1) the cone of every cousin point: target s in box A and the j-th cousin B of A give
    // the cone of s relative to B's centre.  Records are numbered in target order, ptr[s] + j
    // (the evaluation lists), but the cones are stored box by box, column j of box A holding
    // the cones of all of A's points relative to B contiguously:
    // rc[ptr[pt_begin[A]] + j * |A| + (s - pt_begin[A])].
    std::vector<int64_t> ptr(N + 1, 0);
    for (int s = 0; s < N; ++s) ptr[s + 1] = ptr[s] + (int64_t)L.cousin[t.box_of[d][s]].size();
    host_array<cone_key> rc(ptr[N]);
    parallel_dynamic(nb, 1, [&](int, int64_t a0, int64_t a1) {
      for (int64_t A = a0; A < a1; ++A) {
        const int64_t b = L.pt_begin[A], n = L.pt_end[A] - b;
        const std::vector<int>& cs = L.cousin[A];
        for (size_t j = 0; j < cs.size(); ++j) {
          double c[3];
          box_center(t, d, L.ic[cs[j]], c);
          cone_key* out = &rc[ptr[b] + (int64_t)j * n];
          int h2 = -1, h3 = -1;   // neighbouring points of A mostly share B's cells
          for (int64_t i = 0; i < n; ++i) {
            const double* p = &xs[3 * (size_t)(b + i)];
            out[i] = cls(p[0] - c[0], p[1] - c[1], p[2] - c[2], h2, h3);
          }
        }
      }
    });
    // (2) cones containing interpolation points of the parent's relevant cones: the child
    // cone of parent point q of compact parent cone ci in octant o (box independent)
    std::vector<cone_key> cc_key;
    int ncomp_p = 0;
    if (d >= 4) {
      HostLevel& Pp = t.lv[d - 1];
      const ConePoints pts(Pp.cg());
      ncomp_p = (int)Pp.upcone_list.size();
      cc_key.assign((size_t)ncomp_p * 8 * kQ, 0);
      parallel_for(ncomp_p, [&](int64_t c0, int64_t c1) {
        for (int64_t ci = c0; ci < c1; ++ci) {
          cone_key pc = Pp.upcone_list[ci];
          for (int q = 0; q < kQ; ++q) {
            double X[3];
            pts(pc, q, X);
            for (int o = 0; o < 8; ++o) {
              double off = 0.5 * L.H;
              double cx = X[0] - off * ((o & 1) ? 1 : -1);
              double cy = X[1] - off * ((o & 2) ? 1 : -1);
              double cz = X[2] - off * ((o & 4) ? 1 : -1);
              cc_key[((size_t)ci * 8 + o) * kQ + q] = cls(cx, cy, cz);
            }
          }
        }
      });
    }
    // The relevant cones of box B: the distinct cones of (1) relative to B (the cousin
    // relation is symmetric, so B's cousin points are the points of the boxes A in cousin[B],
    // column B of each A) and of (2) for B's octant of each relevant parent cone, sorted.
    // Where the level's cone count is small enough, duplicates are dropped through a
    // per-worker bit per cone (cell-major index, the order of the keys); otherwise all keys
    // are gathered, sorted and made distinct.
    std::vector<std::vector<cone_key>> ukeys(nb);
    {
      const int64_t ndense = (int64_t)cg.ns * cg.na * 2 * cg.na;
      const bool use_bits = ndense <= ((int64_t)1 << 24);
      std::vector<std::vector<uint64_t>> bits(dynamic_workers(nb));
      std::vector<std::vector<cone_key>> bufs(bits.size());
      parallel_dynamic(nb, 1, [&](int w, int64_t b0, int64_t b1) {
        std::vector<uint64_t>& seen = bits[w];
        std::vector<cone_key>& buf = bufs[w];
        if (use_bits && seen.empty()) seen.assign((size_t)((ndense + 63) / 64), 0);
        for (int64_t B = b0; B < b1; ++B) {
          buf.clear();
          auto add = [&](const cone_key* k, int64_t n) {
            if (!use_bits) {
              buf.insert(buf.end(), k, k + n);
              return;
            }
            for (int64_t i = 0; i < n; ++i) {
              int g1, g2, g3;
              cone_decode(k[i], &g1, &g2, &g3);
              const int64_t c = ((int64_t)g1 * cg.na + g2) * (2 * cg.na) + g3;
              const uint64_t m = 1ULL << (c & 63);
              if (!(seen[c >> 6] & m)) {
                seen[c >> 6] |= m;
                buf.push_back(k[i]);
              }
            }
          };
          for (int A : L.cousin[B]) {
            const std::vector<int>& ca = L.cousin[A];
            const auto it = std::lower_bound(ca.begin(), ca.end(), (int)B);
            if (it == ca.end() || *it != (int)B) throw std::logic_error("cousin relation not symmetric");
            const int64_t j = it - ca.begin(), b = L.pt_begin[A], n = L.pt_end[A] - b;
            add(&rc[ptr[b] + j * n], n);
          }
          if (d >= 4) {
            const HostLevel& Pp = t.lv[d - 1];
            const int p = L.parent[B];
            const int o = (L.ic[B][0] & 1) | ((L.ic[B][1] & 1) << 1) | ((L.ic[B][2] & 1) << 2);
            for (int ps = Pp.box_slot_ptr[p]; ps < Pp.box_slot_ptr[p + 1]; ++ps)
              add(&cc_key[((size_t)Pp.slot_upidx[ps] * 8 + o) * kQ], kQ);
          }
          std::sort(buf.begin(), buf.end());
          if (use_bits) {
            for (cone_key k : buf) {
              int g1, g2, g3;
              cone_decode(k, &g1, &g2, &g3);
              const int64_t c = ((int64_t)g1 * cg.na + g2) * (2 * cg.na) + g3;
              seen[c >> 6] &= ~(1ULL << (c & 63));
            }
          } else {
            buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
          }
          ukeys[B].assign(buf.begin(), buf.end());
        }
      });
    }
    // slots: relevant (box, cone) pairs sorted by box then cone
    L.box_slot_ptr.assign(nb + 1, 0);
    for (int b = 0; b < nb; ++b) L.box_slot_ptr[b + 1] = L.box_slot_ptr[b] + (int)ukeys[b].size();
    const int nslots = L.box_slot_ptr[nb];
    L.slot_box.resize(nslots);
    L.slot_cone.resize(nslots);
    parallel_for(nb, [&](int64_t b0, int64_t b1) {
      for (int64_t b = b0; b < b1; ++b) {
        std::copy(ukeys[b].begin(), ukeys[b].end(), L.slot_cone.begin() + L.box_slot_ptr[b]);
        std::fill(L.slot_box.begin() + L.box_slot_ptr[b], L.slot_box.begin() + L.box_slot_ptr[b + 1], (int)b);
      }
    });
    std::vector<std::vector<cone_key>>().swap(ukeys);
    // compact list of this level's relevant cone keys (sorted, distinct), and the slot -> compact map
    L.upcone_list = L.slot_cone;
    std::sort(L.upcone_list.begin(), L.upcone_list.end());
    L.upcone_list.erase(std::unique(L.upcone_list.begin(), L.upcone_list.end()), L.upcone_list.end());
    const int ncomp = (int)L.upcone_list.size();
    auto compact_of = [&](cone_key c) {
      return (int)(std::lower_bound(L.upcone_list.begin(), L.upcone_list.end(), c) - L.upcone_list.begin());
    };
    L.slot_upidx.resize(nslots);
    parallel_for(nslots, [&](int64_t s0, int64_t s1) {
      for (int64_t s = s0; s < s1; ++s) L.slot_upidx[s] = compact_of(L.slot_cone[s]);
    });
    // (box, compact cone) -> slot, read by the upward step from this level
    if (d >= 4) {
      if ((double)nb * ncomp > 2.0e9) throw std::bad_alloc();
      L.cmap.assign((size_t)nb * ncomp, -1);
      parallel_for(nb, [&](int64_t b0, int64_t b1) {
        for (int64_t b = b0; b < b1; ++b)
          for (int s = L.box_slot_ptr[b]; s < L.box_slot_ptr[b + 1]; ++s)
            L.cmap[(size_t)b * ncomp + L.slot_upidx[s]] = s;
      });
    }
    // the parent's upward tables, with child cones as compact indices of this level
    if (d >= 4) {
      HostLevel& Pp = t.lv[d - 1];
      // (a key that no child box holds belongs to octants without a child; never read: -1)
      Pp.up_cc.resize(cc_key.size());
      parallel_for((int64_t)cc_key.size(), [&](int64_t e0, int64_t e1) {
        for (int64_t e = e0; e < e1; ++e) {
          const int c = compact_of(cc_key[e]);
          Pp.up_cc[e] = (c < ncomp && L.upcone_list[c] == cc_key[e]) ? c : -1;
        }
      });
      // The 75 points of a parent cone are split into kUpGroups fixed groups, one per warp
      // of the upward block: contiguous chunks of the 5 x 5 angular grid in snake order
      // (all three radial points of an angular position together), so a group's points
      // fall in few child cones.  A warp only ever adds into its own group's points, for
      // every octant, so no two warps write the same parent value.  Per (parent cone,
      // octant) the points are ranked by (group, child cone); per (parent cone, group) the
      // runs of at most kUpRunMax consecutive ranked points that share one child cone, over
      // all octants, are listed longest first as start | len << 8 | octant << 16.
      Pp.up_order.assign((size_t)ncomp_p * 8 * kQ, 0);
      std::vector<std::vector<int32_t>> ci_tasks(ncomp_p);
      std::vector<int32_t> ci_count((size_t)ncomp_p * kUpGroups, 0);
      int grp[kQ];
      for (int q = 0; q < kQ; ++q) grp[q] = up_group(q);
      parallel_for(ncomp_p, [&](int64_t c0, int64_t c1) {
        std::vector<int32_t> runs[kUpGroups];
        std::vector<int32_t> by_len;
        for (int64_t ci = c0; ci < c1; ++ci) {
          for (auto& r : runs) r.clear();
          for (int o = 0; o < 8; ++o) {
            const size_t g = (size_t)ci * 8 + o;
            const int32_t* cc = &Pp.up_cc[g * kQ];
            int32_t* ord = &Pp.up_order[g * kQ];
            // rank by (group, child cone, point): distinct keys, so the order is the stable one
            int64_t key[kQ];
            for (int q = 0; q < kQ; ++q) key[q] = ((int64_t)grp[q] << 48) | ((int64_t)(cc[q] + 1) << 8) | q;
            std::sort(key, key + kQ);
            for (int q = 0; q < kQ; ++q) ord[q] = (int32_t)(key[q] & 255);
            int r = 0;
            while (r < kQ) {
              const int w = grp[ord[r]];
              int len = 1;
              while (len < kUpRunMax && r + len < kQ && grp[ord[r + len]] == w && cc[ord[r + len]] == cc[ord[r]])
                ++len;
              runs[w].push_back(r | (len << 8) | (o << 16));
              r += len;
            }
          }
          std::vector<int32_t>& out = ci_tasks[ci];
          for (int w = 0; w < kUpGroups; ++w) {
            // longest first, runs of equal length in their order of creation
            by_len.clear();
            for (int len = kUpRunMax; len >= 1; --len)
              for (int32_t rr : runs[w])
                if (((rr >> 8) & 255) == len) by_len.push_back(rr);
            out.insert(out.end(), by_len.begin(), by_len.end());
            ci_count[(size_t)ci * kUpGroups + w] = (int32_t)by_len.size();
          }
        }
      });
      Pp.up_task_ptr.assign((size_t)ncomp_p * kUpGroups + 1, 0);
      for (size_t i = 0; i < ci_count.size(); ++i) Pp.up_task_ptr[i + 1] = Pp.up_task_ptr[i] + ci_count[i];
      Pp.up_task.resize(Pp.up_task_ptr.back());
      parallel_for(ncomp_p, [&](int64_t c0, int64_t c1) {
        for (int64_t ci = c0; ci < c1; ++ci)
          std::copy(ci_tasks[ci].begin(), ci_tasks[ci].end(), Pp.up_task.begin() + Pp.up_task_ptr[ci * kUpGroups]);
      });
      // Tensor-core tables: per (parent cone, octant) the points ranked by (child cone, point)
      // and cut into units of at most kUpRunMax points of one child cone (points whose child
      // cone no child box holds are left out: their octant has no child in any box of this
      // cone); per parent cone its units in octant order.
      Pp.tc_order.assign((size_t)ncomp_p * 8 * kQ, 0);
      std::vector<std::vector<int32_t>> ci_units(ncomp_p);
      parallel_for(ncomp_p, [&](int64_t c0, int64_t c1) {
        for (int64_t ci = c0; ci < c1; ++ci) {
          std::vector<int32_t>& out = ci_units[ci];
          out.clear();
          for (int o = 0; o < 8; ++o) {
            const size_t g = (size_t)ci * 8 + o;
            const int32_t* cc = &Pp.up_cc[g * kQ];
            int32_t* ord = &Pp.tc_order[g * kQ];
            int64_t key[kQ];
            for (int q = 0; q < kQ; ++q) key[q] = ((int64_t)(cc[q] + 1) << 8) | q;
            std::sort(key, key + kQ);
            for (int q = 0; q < kQ; ++q) ord[q] = (int32_t)(key[q] & 255);
            int r = 0;
            while (r < kQ) {
              int len = 1;
              while (len < kUpRunMax && r + len < kQ && cc[ord[r + len]] == cc[ord[r]]) ++len;
              if (cc[ord[r]] >= 0) out.push_back(r | (len << 8) | (o << 16));
              r += len;
            }
          }
        }
      });
      Pp.tc_unit_ptr.assign((size_t)ncomp_p + 1, 0);
      Pp.tc_max_units = 0;
      for (int64_t ci = 0; ci < ncomp_p; ++ci) {
        Pp.tc_unit_ptr[ci + 1] = Pp.tc_unit_ptr[ci] + (int32_t)ci_units[ci].size();
        Pp.tc_max_units = std::max(Pp.tc_max_units, (int)ci_units[ci].size());
      }
      Pp.tc_unit.resize(Pp.tc_unit_ptr.back());
      for (int64_t ci = 0; ci < ncomp_p; ++ci)
        std::copy(ci_units[ci].begin(), ci_units[ci].end(), Pp.tc_unit.begin() + Pp.tc_unit_ptr[ci]);
      // slots of one parent cone in groups of kTcBoxes, slots with equal child sets together
      // (rows of an absent child are computed but not used)
      {
        const size_t ns_p = Pp.slot_box.size();
        std::vector<int64_t> key(ns_p);
        for (size_t sl = 0; sl < ns_p; ++sl) {
          int mask = 0;
          for (int o = 0; o < 8; ++o) mask |= (Pp.child[Pp.slot_box[sl]][o] >= 0) << o;
          key[sl] = ((int64_t)Pp.slot_upidx[sl] << 40) | ((int64_t)mask << 32) | (int64_t)sl;
        }
        std::sort(key.begin(), key.end());
        Pp.tc_item.clear();
        size_t a = 0;
        while (a < ns_p) {
          const int64_t ci = key[a] >> 40;
          size_t b = a;
          while (b < ns_p && (key[b] >> 40) == ci) ++b;
          for (size_t c = a; c < b; c += kTcBoxes)
            for (int j = 0; j < kTcBoxes; ++j)
              Pp.tc_item.push_back(c + j < b ? (int32_t)(key[c + j] & 0xffffffff) : -1);
          a = b;
        }
        // items in the order of their first slot (slots are numbered box by box, boxes in Morton
        // order): the items running at one time then read the child coefficients of neighbouring
        // boxes, which stay in L2 for all of them, instead of one cone's children everywhere
        const size_t ni = Pp.tc_item.size() / kTcBoxes;
        std::vector<int64_t> io(ni);
        for (size_t i = 0; i < ni; ++i) io[i] = ((int64_t)Pp.tc_item[i * kTcBoxes] << 32) | (int64_t)i;
        std::sort(io.begin(), io.end());
        std::vector<int32_t> items(Pp.tc_item.size());
        for (size_t i = 0; i < ni; ++i)
          std::copy_n(&Pp.tc_item[(size_t)(io[i] & 0xffffffff) * kTcBoxes], kTcBoxes, &items[i * kTcBoxes]);
        Pp.tc_item.swap(items);
      }
    }
    // chunks of at most 32 consecutive targets of one box (boxes with cousins): the unit of the
    // FP32 target step, whose targets share their cousin boxes
    // (listed longest first: work n x cousins, so that the last wave holds the short ones)
    L.tgt_chunk.clear();
    {
      std::vector<std::array<int64_t, 3>> ch;   // (work, first target, count)
      for (int A = 0; A < nb; ++A) {
        if (L.cousin[A].empty()) continue;
        for (int s0 = L.pt_begin[A]; s0 < L.pt_end[A]; s0 += 32) {
          const int n = std::min(32, L.pt_end[A] - s0);
          ch.push_back({(int64_t)n * (int64_t)L.cousin[A].size(), s0, n});
        }
      }
      std::stable_sort(ch.begin(), ch.end(), [](const std::array<int64_t, 3>& a, const std::array<int64_t, 3>& b) {
        return a[0] > b[0];
      });
      for (const auto& c : ch) {
        L.tgt_chunk.push_back((int32_t)c[1]);
        L.tgt_chunk.push_back((int32_t)c[2]);
      }
    }
    // per-target slots: each record (s, j) of (1), found in the sorted cones of box cousin[A][j]
    L.tgt_ptr = ptr;
    L.tgt_slot.resize(ptr[N]);
    parallel_dynamic(nb, 1, [&](int, int64_t a0, int64_t a1) {
      for (int64_t A = a0; A < a1; ++A) {
        const int64_t b = L.pt_begin[A], n = L.pt_end[A] - b;
        const std::vector<int>& cs = L.cousin[A];
        for (size_t j = 0; j < cs.size(); ++j) {
          const int lo = L.box_slot_ptr[cs[j]], hi = L.box_slot_ptr[cs[j] + 1];
          const auto first = L.slot_cone.begin() + lo, last = L.slot_cone.begin() + hi;
          const cone_key* k = &rc[ptr[b] + (int64_t)j * n];
          cone_key prev = -1;
          int slot = -1;
          for (int64_t i = 0; i < n; ++i) {
            if (k[i] != prev) {   // neighbouring points mostly share a cone: search only on a change
              prev = k[i];
              slot = lo + (int)(std::lower_bound(first, last, prev) - first);
            }
            L.tgt_slot[ptr[b + i] + j] = slot;
          }
        }
      }
    });
  }
}

void near_candidates(const double* x, int P, int nc, double delta, std::vector<double>& gap,
                     std::vector<int64_t>& cptr, std::vector<int>& cpatch) {
  const int npp = nc * nc;
  const int N = P * npp;
  gap.assign(P, 0.0);
  std::vector<double> cen(3 * (size_t)P, 0.0), rad(P, 0.0);
  auto X = [&](int p, int i, int j) { return x + 3 * ((size_t)p * npp + i * nc + j); };
  for (int p = 0; p < P; ++p) {
    double g = 0;
    for (int i = 0; i + 1 < nc; ++i)
      for (int j = 0; j + 1 < nc; ++j) {
        const double *a = X(p, i, j), *b = X(p, i + 1, j + 1), *c = X(p, i + 1, j), *e = X(p, i, j + 1);
        double d1 = 0, d2 = 0;
        for (int k = 0; k < 3; ++k) {
          d1 += (a[k] - b[k]) * (a[k] - b[k]);
          d2 += (c[k] - e[k]) * (c[k] - e[k]);
        }
        g = std::max(g, std::max(std::sqrt(d1), std::sqrt(d2)));
      }
    gap[p] = 2.0 * g;   // twice the largest node-cell diagonal (reading R15)
    for (int m = 0; m < npp; ++m)
      for (int k = 0; k < 3; ++k) cen[3 * p + k] += x[3 * ((size_t)p * npp + m) + k] / npp;
    for (int m = 0; m < npp; ++m) {
      double dd = 0;
      for (int k = 0; k < 3; ++k) {
        double v = x[3 * ((size_t)p * npp + m) + k] - cen[3 * p + k];
        dd += v * v;
      }
      rad[p] = std::max(rad[p], std::sqrt(dd));
    }
  }
  // patch centres binned in a uniform grid whose cell is the largest reach rad + delta + gap:
  // every patch that can be a candidate of a target has its centre in one of the 27 cells
  // around the target's cell
  double reach = 0, lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int p = 0; p < P; ++p) {
    reach = std::max(reach, rad[p] + delta + gap[p]);
    for (int k = 0; k < 3; ++k) {
      lo[k] = std::min(lo[k], cen[3 * p + k]);
      hi[k] = std::max(hi[k], cen[3 * p + k]);
    }
  }
  for (int l = 0; l < N; ++l)
    for (int k = 0; k < 3; ++k) {
      lo[k] = std::min(lo[k], x[3 * (size_t)l + k]);
      hi[k] = std::max(hi[k], x[3 * (size_t)l + k]);
    }
  const double cell = std::max(reach, 1e-300);
  int dim[3];
  for (int k = 0; k < 3; ++k) dim[k] = std::max(1, std::min(4096, (int)std::floor((hi[k] - lo[k]) / cell) + 1));
  auto cell_of = [&](const double* q, int* c) {
    for (int k = 0; k < 3; ++k) c[k] = std::min(dim[k] - 1, std::max(0, (int)std::floor((q[k] - lo[k]) / cell)));
  };
  const size_t ncell = (size_t)dim[0] * dim[1] * dim[2];
  std::vector<int> cell_ptr(ncell + 1, 0), cell_patch(P);
  std::vector<size_t> pc(P);
  for (int p = 0; p < P; ++p) {
    int c[3];
    cell_of(&cen[3 * p], c);
    pc[p] = ((size_t)c[2] * dim[1] + c[1]) * dim[0] + c[0];
    ++cell_ptr[pc[p] + 1];
  }
  for (size_t c = 0; c < ncell; ++c) cell_ptr[c + 1] += cell_ptr[c];
  {
    std::vector<int> fill(cell_ptr.begin(), cell_ptr.end() - 1);
    for (int p = 0; p < P; ++p) cell_patch[fill[pc[p]]++] = p;   // patches ascending within a cell
  }
  // targets in chunks handed to host threads on demand; each chunk keeps its targets' candidates
  // (each target's in increasing patch order) and the chunks are joined in target order, so the
  // lists do not depend on the thread count
  const int64_t kChunk = 4096;
  const int64_t nchunk = ((int64_t)N + kChunk - 1) / kChunk;
  std::vector<std::vector<int>> part(nchunk);
  cptr.assign(N + 1, 0);
  parallel_dynamic(nchunk, 1, [&](int, int64_t c0, int64_t c1) {
    std::vector<int> found;
    for (int64_t ch = c0; ch < c1; ++ch) {
      std::vector<int>& out = part[ch];
      const int l0 = (int)(ch * kChunk), l1 = (int)std::min<int64_t>(N, (ch + 1) * kChunk);
      for (int l = l0; l < l1; ++l) {
        const double* xl = x + 3 * (size_t)l;
        const int pl = l / npp;
        found.clear();
        found.push_back(pl);
        int c[3];
        cell_of(xl, c);
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              const int cx = c[0] + dx, cy = c[1] + dy, cz = c[2] + dz;
              if (cx < 0 || cy < 0 || cz < 0 || cx >= dim[0] || cy >= dim[1] || cz >= dim[2]) continue;
              const size_t ci = ((size_t)cz * dim[1] + cy) * dim[0] + cx;
              for (int e = cell_ptr[ci]; e < cell_ptr[ci + 1]; ++e) {
                const int p = cell_patch[e];
                if (p == pl) continue;
                double dc = 0;
                for (int k = 0; k < 3; ++k) dc += (xl[k] - cen[3 * p + k]) * (xl[k] - cen[3 * p + k]);
                if (std::sqrt(dc) - rad[p] > delta + gap[p]) continue;
                double dmin = INFINITY;
                for (int m = 0; m < npp; ++m) {
                  const double* y = x + 3 * ((size_t)p * npp + m);
                  double dd = 0;
                  for (int k = 0; k < 3; ++k) dd += (xl[k] - y[k]) * (xl[k] - y[k]);
                  dmin = std::min(dmin, std::sqrt(dd));
                }
                if (dmin <= delta + gap[p]) found.push_back(p);
              }
            }
        std::sort(found.begin(), found.end());
        out.insert(out.end(), found.begin(), found.end());
        cptr[l + 1] = (int64_t)found.size();   // counts; prefix sums below
      }
    }
  });
  for (int l = 0; l < N; ++l) cptr[l + 1] += cptr[l];
  cpatch.resize(cptr[N]);
  parallel_for(nchunk, [&](int64_t c0, int64_t c1) {
    for (int64_t ch = c0; ch < c1; ++ch)
      std::copy(part[ch].begin(), part[ch].end(), cpatch.begin() + cptr[ch * kChunk]);
  });
}

int64_t near_nnz_bound(const HostTree& t, int P, int nc, const std::vector<int64_t>& cptr,
                       const std::vector<int>& cpatch) {
  const int npp = nc * nc;
  const int N = P * npp;
  const int D = t.D;
  const HostLevel& L = t.lv[D];
  // per target: every candidate patch's nodes, plus the neighbour-box points on other patches
  const int64_t kChunk = 4096;
  const int64_t nchunk = ((int64_t)N + kChunk - 1) / kChunk;
  std::vector<int64_t> part(nchunk, 0);
  std::vector<std::vector<uint8_t>> marks(dynamic_workers(nchunk));
  parallel_dynamic(nchunk, 1, [&](int w, int64_t c0, int64_t c1) {
    std::vector<uint8_t>& mark = marks[w];
    if (mark.empty()) mark.assign(P, 0);
    for (int64_t ch = c0; ch < c1; ++ch) {
      int64_t n = 0;
      const int l0 = (int)(ch * kChunk), l1 = (int)std::min<int64_t>(N, (ch + 1) * kChunk);
      for (int l = l0; l < l1; ++l) {
        for (int64_t e = cptr[l]; e < cptr[l + 1]; ++e) mark[cpatch[e]] = 1;
        n += (cptr[l + 1] - cptr[l]) * (int64_t)npp;
        const int A = t.box_of[D][t.iperm[l]];
        for (int B : L.nbr[A])
          for (int s = L.pt_begin[B]; s < L.pt_end[B]; ++s) n += mark[t.perm[s] / npp] ? 0 : 1;
        for (int64_t e = cptr[l]; e < cptr[l + 1]; ++e) mark[cpatch[e]] = 0;
      }
      part[ch] = n;
    }
  });
  int64_t total = 0;
  for (int64_t v : part) total += v;
  return total;
}

void near_structure(const HostTree& t, int P, int nc, const std::vector<int64_t>& cptr,
                    const std::vector<int>& cpatch, const std::vector<uint8_t>& singular,
                    std::vector<int64_t>& row_ptr, host_array<int>& col, host_array<int>& pair) {
  const int npp = nc * nc;
  const int N = P * npp;
  const int D = t.D;
  const HostLevel& L = t.lv[D];
  // Row l: all nodes of the singular patches of x_l (Eq. patch_sing), in candidate order, then
  // the neighbour points on regular patches (reading R12: IFGF leaves them out), in sorted
  // order.  Two passes over host threads (count, then fill), each thread with its own patch
  // marks; the result does not depend on the thread count.
  auto row = [&](int l, std::vector<int>& mark, int* c, int* q) -> int64_t {
    int64_t n = 0;
    for (int64_t e = cptr[l]; e < cptr[l + 1]; ++e)
      if (singular[e]) mark[cpatch[e]] = (int)e;
    for (int64_t e = cptr[l]; e < cptr[l + 1]; ++e)
      if (singular[e]) {
        const int p = cpatch[e];
        if (c)
          for (int m = 0; m < npp; ++m) {
            c[n + m] = p * npp + m;
            q[n + m] = (int)e;
          }
        n += npp;
      }
    const int A = t.box_of[D][t.iperm[l]];
    for (int B : L.nbr[A])
      for (int s = L.pt_begin[B]; s < L.pt_end[B]; ++s) {
        const int m = t.perm[s];
        if (mark[m / npp] >= 0) continue;
        if (c) {
          c[n] = m;
          q[n] = -1;
        }
        ++n;
      }
    for (int64_t e = cptr[l]; e < cptr[l + 1]; ++e) mark[cpatch[e]] = -1;
    return n;
  };
  row_ptr.assign(N + 1, 0);
  parallel_for(N, [&](int64_t l0, int64_t l1) {
    std::vector<int> mark(P, -1);
    for (int64_t l = l0; l < l1; ++l) row_ptr[l + 1] = row((int)l, mark, nullptr, nullptr);
  });
  for (int l = 0; l < N; ++l) row_ptr[l + 1] += row_ptr[l];
  col.resize(row_ptr[N]);
  pair.resize(row_ptr[N]);
  parallel_for(N, [&](int64_t l0, int64_t l1) {
    std::vector<int> mark(P, -1);
    for (int64_t l = l0; l < l1; ++l) row((int)l, mark, col.data() + row_ptr[l], pair.data() + row_ptr[l]);
  });
}

}  // namespace ifgf
