// IFGF far-field kernels (Sec. III-E to III-G, vectorised over 8 densities x
// 2 wavenumbers as in Eq. ifgf_sum_em):
//   (a) k_leaf:   F^D_k at the interpolation points of every relevant cone
//                 segment of every leaf box by direct summation of Eq.
//                 bkd_contr_ana_fac (algorithm step 2), then values ->
//                 Chebyshev coefficients per cone (Sec. III-E interpolation).
//   (b) k_up:     F^{d-1}_j at the parent's interpolation points: interpolate
//                 each child's F^d_k, multiply by G(x,x_k)/G(x,x_j) and sum
//                 over the children (algorithm step 3, second item).
//   (c) k_target: I^d_k at the cousin points: interpolate F^d_k and multiply by
//                 the centred factor G(x, x_k) (algorithm step 3, first item),
//                 plus the normal derivative of the same product (Sec. III-I).
// Coefficients are stored per cone segment as [75][32] reals: Chebyshev index
// (i_s*5 + i_theta)*5 + i_phi, then 16 complex fields (kernel*8 + density).
#include <type_traits>

#include "kernels.h"

namespace ifgf {

namespace {

// Inner-loop helpers of the leaf step: in FP32 the hardware approximations
// (__fdividef, __sincosf; the phase argument there is bounded by k h_leaf,
// a few radians, where __sincosf is accurate to ~4e-7); in FP64 the exact ones.
template <typename T>
__device__ inline T leaf_div(T a, T b) { return a / b; }
template <>
__device__ inline float leaf_div<float>(float a, float b) { return __fdividef(a, b); }
template <typename T>
__device__ inline void leaf_sincos(T x, T* s, T* c) { sincos_t(x, s, c); }
template <>
__device__ inline void leaf_sincos<float>(float x, float* s, float* c) { __sincosf(x, s, c); }

// 1D values -> coefficients maps for 3 and 5 open Chebyshev nodes, and the nodes.
template <typename T>
struct SmallMaps {
  T A3[9], A5[25];
  T x3[3], x5[5];
};

template <typename T>
__device__ void init_maps(SmallMaps<T>& M) {
  int t = threadIdx.x;
  // in the kernel's own precision (cos(pi x) of exact arguments)
  if (t < 9) {
    int i = t / 3, j = t % 3;
    M.A3[t] = (i == 0 ? T(1) : T(2)) / T(3) * cospi_t<T>(T(i * (2 * j + 1)) / T(6));
  }
  if (t < 25) {
    int i = t / 5, j = t % 5;
    M.A5[t] = (i == 0 ? T(1) : T(2)) / T(5) * cospi_t<T>(T(i * (2 * j + 1)) / T(10));
  }
  if (t < 3) M.x3[t] = cospi_t<T>(T(2 * t + 1) / T(6));
  if (t < 5) M.x5[t] = cospi_t<T>(T(2 * t + 1) / T(10));
}

// Interpolation point q of cone `cone` relative to the box centre.
template <typename T>
__device__ inline void cone_point(const SmallMaps<T>& M, const ConeGeomT<T>& cg, cone_key cone, int q, T* X) {
  int g1, g2, g3;
  cone_decode(cone, &g1, &g2, &g3);
  int is = q / 25, it = (q / 5) % 5, ip = q % 5;
  const T ds = cg.ds, dth = cg.dth;
  T s = ((T)g1 + T(0.5) * (T(1) + M.x3[is])) * ds;
  T th = ((T)g2 + T(0.5) * (T(1) + M.x5[it])) * dth;
  T ph = ((T)g3 + T(0.5) * (T(1) + M.x5[ip])) * dth;
  T r = cg.h / s;
  T st, ct, sp, cp;
  sincos_t(th, &st, &ct);
  sincos_t(ph, &sp, &cp);
  X[0] = r * st * cp;
  X[1] = r * st * sp;
  X[2] = r * ct;
}

// Local coordinates in [-1, 1]^3 of a point (relative to the box centre) inside cone `cone`.
template <typename T>
__device__ inline void local_coords(const ConeGeomT<T>& cg, cone_key cone, T x, T y, T z, T* ts, T* tt, T* tp,
                                    T* rr, T* sth, T* cth, T* sph, T* cph) {
  int g1, g2, g3;
  cone_decode(cone, &g1, &g2, &g3);
  T rho = sqrt_t(x * x + y * y);
  T r = sqrt_t(rho * rho + z * z);
  T s = cg.h / r;
  T th = atan2_t(rho, z);
  T ph = atan2_t(y, x);
  T php = ph - (T)g3 * cg.dth;
  if (php < T(-kPi)) php += T(2 * kPi);   // phi wraps: measure from the cell start
  if (php > T(kPi)) php -= T(2 * kPi);
  *ts = T(2) * (s * cg.ids - (T)g1) - T(1);
  *tt = T(2) * (th * cg.idth - (T)g2) - T(1);
  *tp = T(2) * php * cg.idth - T(1);
  *rr = r;
  *sth = rho / r;
  *cth = z / r;
  T irho = rho > T(0) ? T(1) / rho : T(0);
  *cph = rho > T(0) ? x * irho : T(1);
  *sph = rho > T(0) ? y * irho : T(0);
}

// In-place 3D values -> coefficients transform of one real column (stride `st`) of 75 values.
template <typename T>
__device__ void vals_to_coefs_col(const SmallMaps<T>& M, T* v, int st) {
  T t5[5];
  // phi (innermost)
  for (int a = 0; a < 15; ++a) {
    for (int k = 0; k < 5; ++k) t5[k] = v[(a * 5 + k) * st];
    for (int k = 0; k < 5; ++k) {
      T acc = 0;
      for (int kk = 0; kk < 5; ++kk) acc += M.A5[k * 5 + kk] * t5[kk];
      v[(a * 5 + k) * st] = acc;
    }
  }
  // theta
  for (int is = 0; is < 3; ++is)
    for (int k = 0; k < 5; ++k) {
      for (int j = 0; j < 5; ++j) t5[j] = v[((is * 5 + j) * 5 + k) * st];
      for (int j = 0; j < 5; ++j) {
        T acc = 0;
        for (int jj = 0; jj < 5; ++jj) acc += M.A5[j * 5 + jj] * t5[jj];
        v[((is * 5 + j) * 5 + k) * st] = acc;
      }
    }
  // s
  for (int jk = 0; jk < 25; ++jk) {
    for (int i = 0; i < 3; ++i) t5[i] = v[(i * 25 + jk) * st];
    for (int i = 0; i < 3; ++i) {
      T acc = 0;
      for (int ii = 0; ii < 3; ++ii) acc += M.A3[i * 3 + ii] * t5[ii];
      v[(i * 25 + jk) * st] = acc;
    }
  }
}

constexpr int kVS = 33;   // padded row stride of the value buffers

// The same transform for all 32 columns of `ns` consecutive [75][kStride] value
// buffers by the whole block (one (buffer, line, column) task per thread and pass,
// consecutive threads on consecutive columns), followed by a coalesced store of the
// 75 x 32 coefficients of buffer i to out + i * 75 * 32.  Every thread of the block
// must call it.
template <typename T, int kStride>
__device__ void vals_to_coefs_block(const SmallMaps<T>& M, T* vb, T* out, int ns = 1) {
  const int nt = blockDim.x;
  constexpr int kBuf = kQ * kStride;
  for (int e = threadIdx.x; e < ns * 15 * 32; e += nt) {   // phi lines
    const int b = e / (15 * 32), r = e - b * 15 * 32, a = r >> 5, col = r & 31;
    T* v = vb + b * kBuf;
    T t5[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) t5[k] = v[(a * 5 + k) * kStride + col];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      T acc = 0;
#pragma unroll
      for (int kk = 0; kk < 5; ++kk) acc += M.A5[k * 5 + kk] * t5[kk];
      v[(a * 5 + k) * kStride + col] = acc;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < ns * 15 * 32; e += nt) {   // theta lines
    const int b = e / (15 * 32), r = e - b * 15 * 32, ik = r >> 5, col = r & 31, is = ik / 5, k = ik % 5;
    T* v = vb + b * kBuf;
    T t5[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) t5[j] = v[((is * 5 + j) * 5 + k) * kStride + col];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      T acc = 0;
#pragma unroll
      for (int jj = 0; jj < 5; ++jj) acc += M.A5[j * 5 + jj] * t5[jj];
      v[((is * 5 + j) * 5 + k) * kStride + col] = acc;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < ns * 25 * 32; e += nt) {   // s lines
    const int b = e / (25 * 32), r = e - b * 25 * 32, jk = r >> 5, col = r & 31;
    T* v = vb + b * kBuf;
    T t3[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) t3[i] = v[(i * 25 + jk) * kStride + col];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      T acc = 0;
#pragma unroll
      for (int ii = 0; ii < 3; ++ii) acc += M.A3[i * 3 + ii] * t3[ii];
      v[(i * 25 + jk) * kStride + col] = acc;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < ns * kQ * 32; e += nt) {
    const int b = e / (kQ * 32), r = e - b * kQ * 32;
    out[e] = vb[b * kBuf + (r >> 5) * kStride + (r & 31)];
  }
}

// ------------------------------------------------------------------ (a) leaf direct
constexpr int kLeafThreads = 160;   // two cone segments (2 x 75 points) per pass
constexpr int kLeafChunk = 256;     // sources staged per pass
constexpr int kLeafSlots = 8;       // cone segments of one box per block (grid.y splits a box)

template <typename T>
struct LeafArgs {
  const int* box_pt_ptr;
  const int* box_slot_ptr;
  const cone_key* slot_cone;
  const double* box_center;
  ConeGeomT<T> cg;
  const double* x_sorted;
  const T* a_sorted;
  T* coefs;
  T ke, ki;
  size_t astride, cstride;   // per right-hand side: densities, cone coefficients
};

template <typename T>
__global__ void __launch_bounds__(kLeafThreads) k_leaf(LeafArgs<T> A) {
  __shared__ SmallMaps<T> M;
  // FP32: the staged sources and the value buffer have separate space, so a box's
  // sources are staged once; FP64 (which would need more than 48 KB) aliases them and
  // restages per pass.
  constexpr bool kSep = sizeof(T) == 4;
  constexpr int kSrcWords = kLeafChunk * 20, kValWords = 2 * kQ * kVS;
  __shared__ T pool[kSep ? kSrcWords + kValWords : (kSrcWords > kValWords ? kSrcWords : kValWords)];
  T (*src)[4] = reinterpret_cast<T (*)[4]>(pool);
  T (*sa)[16] = reinterpret_cast<T (*)[16]>(pool + kLeafChunk * 4);
  T* vbuf = pool + (kSep ? kSrcWords : 0);
  const int box = blockIdx.x;
  const int t = threadIdx.x;
  A.a_sorted += blockIdx.z * A.astride;   // right-hand side of a batched call
  A.coefs += blockIdx.z * A.cstride;
  const int sb = A.box_slot_ptr[box] + blockIdx.y * kLeafSlots;
  const int se = min(A.box_slot_ptr[box + 1], sb + kLeafSlots);
  if (sb >= se) return;   // the box has fewer segments than this block's range (uniform per block)
  init_maps(M);
  const double c0 = A.box_center[3 * box], c1 = A.box_center[3 * box + 1], c2 = A.box_center[3 * box + 2];
  const int pb = A.box_pt_ptr[box], pe = A.box_pt_ptr[box + 1];
  const int nsrc = pe - pb;
  const bool staged_once = kSep && nsrc <= kLeafChunk;   // the usual case for FP32
  const T kk[2] = {A.ke, A.ki};
  auto stage = [&](int cb, int nchunk) {
    for (int e = t; e < nchunk; e += blockDim.x) {
      const int m = pb + cb + e;
      T y0 = (T)(A.x_sorted[3 * (size_t)m] - c0);
      T y1 = (T)(A.x_sorted[3 * (size_t)m + 1] - c1);
      T y2 = (T)(A.x_sorted[3 * (size_t)m + 2] - c2);
      src[e][0] = y0; src[e][1] = y1; src[e][2] = y2;
      src[e][3] = y0 * y0 + y1 * y1 + y2 * y2;
      for (int k = 0; k < 16; ++k) sa[e][k] = A.a_sorted[16 * (size_t)m + k];
    }
  };
  if (staged_once) stage(0, nsrc);
  for (int s0 = sb; s0 < se; s0 += 2) {
    const int sl = t / kQ, q = t % kQ;
    const int slot = s0 + sl;
    const bool act = (t < 2 * kQ) && (slot < se);
    T X[3] = {0, 0, 0}, r = 1;
    __syncthreads();
    if (act) {
      cone_point(M, A.cg, A.slot_cone[slot], q, X);
      r = sqrt_t(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
    }
    T acc[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) acc[k] = 0;
    for (int cb = 0; cb < nsrc; cb += kLeafChunk) {
      const int nchunk = min(kLeafChunk, nsrc - cb);
      if (!staged_once) {
        __syncthreads();
        stage(cb, nchunk);
        __syncthreads();
      }
      if (act) {
        for (int e = 0; e < nchunk; ++e) {
          // g_S(X, y) = (r/|X-y|) exp(i k (|X-y| - r)), |X-y| - r = (|y|^2 - 2 X.y)/(|X-y| + r)
          T dxy = src[e][3] - T(2) * (X[0] * src[e][0] + X[1] * src[e][1] + X[2] * src[e][2]);
          T d = sqrt_t(r * r + dxy);
          T rd = leaf_div(r, d);
          T dd = leaf_div(dxy, d + r);
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            T sn, cs;
            leaf_sincos(kk[ks] * dd, &sn, &cs);
            T gr = rd * cs, gi = rd * sn;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              T ar = sa[e][2 * k], ai = sa[e][2 * k + 1];
              acc[2 * (8 * ks + k)] += ar * gr - ai * gi;
              acc[2 * (8 * ks + k) + 1] += ar * gi + ai * gr;
            }
          }
        }
      }
    }
    if (!kSep) __syncthreads();   // the value buffer overlays the staged sources
    if (act)
      for (int k = 0; k < 32; ++k) vbuf[(sl * kQ + q) * kVS + k] = acc[k];
    __syncthreads();
    vals_to_coefs_block<T, kVS>(M, vbuf, A.coefs + (size_t)s0 * kQ * 32, min(2, se - s0));
  }
}

// ------------------------------------------------------------------ (b) upward pass
constexpr int kUpThreads = 128;

template <typename T>
struct UpArgs {
  // parent level d-1
  const int* slot_box;
  const cone_key* slot_cone;
  const int* slot_upidx;
  const int* child;        // [nboxes_p][8]
  ConeGeomT<T> cgp;
  // child level d
  const int* cmap_c;       // [nboxes_c][ncomp_c] -> slot
  int ncomp_c;
  const cone_key* ckeys_c; // [ncomp_c]
  ConeGeomT<T> cgc;
  double Hc;
  const int* up_cc;        // [ncompact_p][8][75] child cone, compact index of level d
  const T* coefs_c;
  T* coefs_p;
  T ke, ki;
  size_t cstride_c, cstride_p;   // per right-hand side
};

template <typename T>
struct PtInfo {
  int cslot;
  T ts, tt, tp;
  T fr[2], fi[2];
};

template <typename T>
__global__ void __launch_bounds__(kUpThreads) k_up(UpArgs<T> A) {
  __shared__ SmallMaps<T> M;
  __shared__ T Xp[kQ][3];
  __shared__ PtInfo<T> info[kQ];
  __shared__ T vals[kQ * kVS];
  const int pslot = blockIdx.x;
  const int t = threadIdx.x, warp = t / 32, lane = t % 32;
  A.coefs_c += blockIdx.y * A.cstride_c;   // right-hand side of a batched call
  A.coefs_p += blockIdx.y * A.cstride_p;
  init_maps(M);
  const int P = A.slot_box[pslot], ci = A.slot_upidx[pslot];
  const cone_key pcone = A.slot_cone[pslot];
  __syncthreads();
  if (t < kQ) cone_point(M, A.cgp, pcone, t, Xp[t]);
  for (int e = t; e < kQ * kVS; e += blockDim.x) vals[e] = 0;
  const T off = (T)(0.5 * A.Hc);
  const T kk[2] = {A.ke, A.ki};
  for (int o = 0; o < 8; ++o) {
    const int cb = A.child[8 * P + o];
    if (cb < 0) continue;
    __syncthreads();
    if (t < kQ) {
      const T ox = (o & 1) ? off : -off, oy = (o & 2) ? off : -off, oz = (o & 4) ? off : -off;
      const T x = Xp[t][0] - ox, y = Xp[t][1] - oy, z = Xp[t][2] - oz;
      const int ccx = A.up_cc[((size_t)ci * 8 + o) * kQ + t];
      const cone_key cc = A.ckeys_c[ccx];
      info[t].cslot = A.cmap_c[(size_t)cb * A.ncomp_c + ccx];
      T rc, sth, cth, sph, cph;
      local_coords(A.cgc, cc, x, y, z, &info[t].ts, &info[t].tt, &info[t].tp, &rc, &sth, &cth, &sph, &cph);
      // re-centring factor G(x, x_child)/G(x, x_parent) = (r_p/r_c) e^{i k (r_c - r_p)}
      const T rp = sqrt_t(Xp[t][0] * Xp[t][0] + Xp[t][1] * Xp[t][1] + Xp[t][2] * Xp[t][2]);
      const T dr = (T(3) * off * off - T(2) * (Xp[t][0] * ox + Xp[t][1] * oy + Xp[t][2] * oz)) / (rc + rp);
      for (int ks = 0; ks < 2; ++ks) {
        T sn, cs;
        sincos_t(kk[ks] * dr, &sn, &cs);
        info[t].fr[ks] = rp / rc * cs;
        info[t].fi[ks] = rp / rc * sn;
      }
    }
    __syncthreads();
    for (int q = warp; q < kQ; q += kUpThreads / 32) {
      const PtInfo<T>& I = info[q];
      if (I.cslot < 0) continue;   // cannot happen: the host marked every such cone relevant
      T Ts[3], Tt[5], Tp[5];
      cheb_vals<T, 3>(I.ts, Ts);
      cheb_vals<T, 5>(I.tt, Tt);
      cheb_vals<T, 5>(I.tp, Tp);
      const T* C = A.coefs_c + (size_t)I.cslot * kQ * 32 + lane;
      T v = 0;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 5; ++j) {
          const T b = Ts[i] * Tt[j];
#pragma unroll
          for (int k = 0; k < 5; ++k) v += b * Tp[k] * __ldg(C + ((i * 5 + j) * 5 + k) * 32);
        }
      const T w = __shfl_xor_sync(0xffffffffu, v, 1);
      const int ks = lane >> 4;
      const T re = (lane & 1) ? w : v, im = (lane & 1) ? v : w;
      const T fr = I.fr[ks], fi = I.fi[ks];
      vals[q * kVS + lane] += (lane & 1) ? (re * fi + im * fr) : (re * fr - im * fi);
    }
  }
  __syncthreads();
  if (t < 32) {
    vals_to_coefs_col(M, vals + t, kVS);
    T* out = A.coefs_p + (size_t)pslot * kQ * 32 + t;
    for (int q = 0; q < kQ; ++q) out[q * 32] = vals[q * kVS + t];
  }
}

// (b), FP32 variant.  The parent points are processed in runs of up to
// kUpRunMax points that fall in the same child cone (box-independent tables
// built with the octree), one warp per run and one lane per real column.  The
// warp loads the child cone's 75 x 32 coefficients once into registers (75
// per lane) and then sweeps the run: per point the Chebyshev values and the
// re-centring factor, formed once per (octant, point) in the prologue, are read
// from shared memory with vector loads, and the 3D Chebyshev sum is contracted
// separably (over phi, then theta, then s: 74 FMA per lane).  The parent points
// are split into kUpGroups fixed groups, one per warp, so each warp adds into
// its own points' values with plain shared-memory adds.
struct RunTabs {
  const int* order;      // [ncompact][8][75] points ranked by (group, child cone)
  const int* task;       // runs per (compact cone, group), longest first: start | len << 8 | octant << 16
  const int* task_ptr;   // [ncompact * kUpGroups + 1]
};

// Per (octant, parent point) data of the FP32 upward pass, formed once in the prologue and
// read by every lane: the Chebyshev values T_1..T_4 of the local phi and theta coordinates and
// T_1, T_2 of the radial one (T_0 = 1 is implicit), 16-byte aligned for vector loads.
struct __align__(16) UpCheb {
  float tp[4];
  float tt[4];
  float ts[2];
  float pad[2];
};

constexpr int kUpRunWarps = kUpGroups;   // warp w adds only into the parent points of group w

// dynamic shared memory of k_up_runs (above the 48 KB static limit)
constexpr size_t kUpRunSmem = sizeof(UpCheb) * 8 * kQ      // Chebyshev values per (octant, point)
                              + sizeof(float4) * 8 * kQ    // re-centring factors (re, im) x 2 kernels
                              + sizeof(int) * 8 * kQ       // child slot per (octant, point)
                              + sizeof(float) * kQ * kVS   // parent values
                              + sizeof(float) * kQ * 3;    // parent points

__global__ void __launch_bounds__(32 * kUpRunWarps, 4) k_up_runs(UpArgs<float> A, RunTabs RT) {
  using T = float;
  __shared__ SmallMaps<T> M;
  extern __shared__ float4 up_smem[];
  UpCheb (*cheb)[kQ] = reinterpret_cast<UpCheb (*)[kQ]>(up_smem);
  float4 (*fac)[kQ] = reinterpret_cast<float4 (*)[kQ]>(cheb + 8);
  int (*cslot)[kQ] = reinterpret_cast<int (*)[kQ]>(fac + 8);
  T* vals = reinterpret_cast<T*>(cslot + 8);
  T (*Xp)[3] = reinterpret_cast<T (*)[3]>(vals + kQ * kVS);
  const int pslot = blockIdx.x;
  const int t = threadIdx.x, warp = t / 32, lane = t % 32;
  A.coefs_c += blockIdx.y * A.cstride_c;   // right-hand side of a batched call
  A.coefs_p += blockIdx.y * A.cstride_p;
  init_maps(M);
  const int P = A.slot_box[pslot], ci = A.slot_upidx[pslot];
  const cone_key pcone = A.slot_cone[pslot];
  __syncthreads();
  if (t < kQ) cone_point(M, A.cgp, pcone, t, Xp[t]);
  for (int e = t; e < kQ * kVS; e += blockDim.x) vals[e] = T(0);
  __syncthreads();
  const T off = (T)(0.5 * A.Hc);
  const T kk[2] = {A.ke, A.ki};
  // prologue: per (octant, parent point) the child slot, the Chebyshev values of the point's
  // local coordinates in its child cone, and the re-centring factor of both kernels
  for (int e = t; e < 8 * kQ; e += blockDim.x) {
    const int o = e / kQ, q = e % kQ;
    const int cb = A.child[8 * P + o];
    if (cb < 0) continue;
    const T ox = (o & 1) ? off : -off, oy = (o & 2) ? off : -off, oz = (o & 4) ? off : -off;
    const T x = Xp[q][0] - ox, y = Xp[q][1] - oy, z = Xp[q][2] - oz;
    const int ccx = A.up_cc[((size_t)ci * 8 + o) * kQ + q];
    const cone_key cc = A.ckeys_c[ccx];
    cslot[o][q] = A.cmap_c[(size_t)cb * A.ncomp_c + ccx];
    T ts, tt, tp, rc, sth, cth, sph, cph;
    local_coords(A.cgc, cc, x, y, z, &ts, &tt, &tp, &rc, &sth, &cth, &sph, &cph);
    T v5[5], v3[3];
    UpCheb& C = cheb[o][q];
    cheb_vals<T, 5>(tp, v5);
    C.tp[0] = v5[1]; C.tp[1] = v5[2]; C.tp[2] = v5[3]; C.tp[3] = v5[4];
    cheb_vals<T, 5>(tt, v5);
    C.tt[0] = v5[1]; C.tt[1] = v5[2]; C.tt[2] = v5[3]; C.tt[3] = v5[4];
    cheb_vals<T, 3>(ts, v3);
    C.ts[0] = v3[1]; C.ts[1] = v3[2];
    // re-centring factor G(x, x_child)/G(x, x_parent) = (r_p/r_c) e^{i k (r_c - r_p)}
    const T rp = sqrt_t(Xp[q][0] * Xp[q][0] + Xp[q][1] * Xp[q][1] + Xp[q][2] * Xp[q][2]);
    const T dr = (T(3) * off * off - T(2) * (Xp[q][0] * ox + Xp[q][1] * oy + Xp[q][2] * oz)) / (rc + rp);
    T sn0, cs0, sn1, cs1;
    sincos_t(kk[0] * dr, &sn0, &cs0);
    sincos_t(kk[1] * dr, &sn1, &cs1);
    const T a = rp / rc;
    fac[o][q] = make_float4(a * cs0, a * sn0, a * cs1, a * sn1);
  }
  __syncthreads();
  const int ks = lane >> 4;   // columns 0..15 belong to kernel e, 16..31 to kernel i
  // complex re-centring on interleaved (re, im) lanes: with w the partner lane's value,
  // re' = v fr - w fi (even lanes), im' = v fr + w fi (odd lanes)
  const T sgn = (lane & 1) ? T(1) : T(-1);
  // the warp's own runs (its group of parent points, all octants); runs of absent children
  // are skipped.  Only this warp adds into these points' values: plain shared-memory adds.
  const int w1 = __ldg(RT.task_ptr + (size_t)ci * kUpGroups + warp + 1);
  for (int w = __ldg(RT.task_ptr + (size_t)ci * kUpGroups + warp); w < w1; ++w) {
    const int tk = __ldg(RT.task + w);
    const int r0 = tk & 255, len = (tk >> 8) & 255, o = (tk >> 16) & 7;
    if (A.child[8 * P + o] < 0) continue;
    const size_t g = (size_t)ci * 8 + o;
    const int myq = lane < len ? __ldg(RT.order + g * kQ + r0 + lane) : 0;
    // one child slot per run: the host marked every such cone relevant
    const T* Cg = A.coefs_c + (size_t)cslot[o][__shfl_sync(0xffffffffu, myq, 0)] * kQ * 32 + lane;
    T c[kQ];
#pragma unroll
    for (int k = 0; k < kQ; ++k) c[k] = __ldg(Cg + k * 32);
    for (int a = 0; a < len; ++a) {
      const int q = __shfl_sync(0xffffffffu, myq, a);
      const float4* cp = reinterpret_cast<const float4*>(&cheb[o][q]);
      const float4 P4 = cp[0], T4 = cp[1], S4 = cp[2];
      const float4 F4 = fac[o][q];
      const T Tp[4] = {P4.x, P4.y, P4.z, P4.w};
      const T Tt[4] = {T4.x, T4.y, T4.z, T4.w};
      // separable contraction (phi, then theta, then s), T_0 = 1 folded in
      T E[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        T e = T(0);
#pragma unroll
        for (int j = 0; j < 5; ++j) {
          const T* cij = c + (i * 5 + j) * 5;
          T d = cij[0];
#pragma unroll
          for (int k = 0; k < 4; ++k) d = fmaf(Tp[k], cij[k + 1], d);
          e = j == 0 ? d : fmaf(Tt[j - 1], d, e);
        }
        E[i] = e;
      }
      const T v = fmaf(S4.y, E[2], fmaf(S4.x, E[1], E[0]));
      const T wv = __shfl_xor_sync(0xffffffffu, v, 1);
      const T fr = ks ? F4.z : F4.x, fi = ks ? F4.w : F4.y;
      vals[q * kVS + lane] += fmaf(v, fr, sgn * fi * wv);
    }
  }
  __syncthreads();
  vals_to_coefs_block<T, kVS>(M, vals, A.coefs_p + (size_t)pslot * kQ * 32);
}

// ------------------------------------------------------------------ (c) target evaluation
template <typename T>
struct TgtArgs {
  int N;
  const int64_t* tgt_ptr;
  const int* tgt_slot;
  const int* slot_box;
  const cone_key* slot_cone;
  const double* box_center;
  ConeGeomT<T> cg;
  const T* coefs;
  const double* x_sorted;
  const double* n_sorted;
  const int* perm;
  T* f28;
  T ke, ki;
  size_t cstride;   // cone coefficients per right-hand side (fields: 56 N)
};

// Per (target, cone) scalars, computed one cone per lane and read back by the
// whole warp: Chebyshev values and derivatives in (s, theta, phi), the
// directional-derivative weights and the centred factors of both kernels.
template <typename T>
struct TgtScal {
  T Ts[3], dTs[3], Tt[5], dTt[5], Tp[5], dTp[5];
  T as, at, ap;
  T G[2][4];   // per kernel: Re G, Im G, Re dG/dn, Im dG/dn
  int slot;
};

template <typename T>
__host__ __device__ constexpr int tgt_warps() { return sizeof(T) == 4 ? 8 : 4; }   // keeps the scalars under 48 KB

template <typename T>
__global__ void __launch_bounds__(32 * tgt_warps<T>(), 2) k_target(TgtArgs<T> A) {
  __shared__ TgtScal<T> sc[tgt_warps<T>()][32];
  const int warp = threadIdx.x >> 5;
  const int t = blockIdx.x * tgt_warps<T>() + warp;
  const int lane = threadIdx.x & 31;
  if (t >= A.N) return;
  A.coefs += blockIdx.y * A.cstride;   // right-hand side of a batched call
  A.f28 += blockIdx.y * 56 * (size_t)A.N;
  const int64_t e0 = A.tgt_ptr[t], e1 = A.tgt_ptr[t + 1];
  if (e0 == e1) return;
  const double x0 = A.x_sorted[3 * (size_t)t], x1 = A.x_sorted[3 * (size_t)t + 1], x2 = A.x_sorted[3 * (size_t)t + 2];
  const T n0 = (T)A.n_sorted[3 * (size_t)t], n1 = (T)A.n_sorted[3 * (size_t)t + 1], n2 = (T)A.n_sorted[3 * (size_t)t + 2];
  const int ks = lane >> 4;
  const T two_ids = T(2) * A.cg.ids, two_idth = T(2) * A.cg.idth, h = A.cg.h;
  TgtScal<T>* S = sc[warp];
  T accS = 0, accD = 0;
  for (int64_t c0 = e0; c0 < e1; c0 += 32) {
    const int nc = (int)min((int64_t)32, e1 - c0);
    if (lane < nc) {
      TgtScal<T>& Q = S[lane];
      const int slot = A.tgt_slot[c0 + lane];
      const int box = A.slot_box[slot];
      const cone_key cone = A.slot_cone[slot];
      const T xr = (T)(x0 - A.box_center[3 * box]);
      const T yr = (T)(x1 - A.box_center[3 * box + 1]);
      const T zr = (T)(x2 - A.box_center[3 * box + 2]);
      T ts, tt, tp, r, sth, cth, sph, cph;
      local_coords(A.cg, cone, xr, yr, zr, &ts, &tt, &tp, &r, &sth, &cth, &sph, &cph);
      cheb_vals<T, 3>(ts, Q.Ts);
      cheb_vals<T, 5>(tt, Q.Tt);
      cheb_vals<T, 5>(tp, Q.Tp);
      cheb_dvals<T, 3>(ts, Q.dTs);
      cheb_dvals<T, 5>(tt, Q.dTt);
      cheb_dvals<T, 5>(tp, Q.dTp);
      // n . grad of (s, theta, phi): grad s = -(h/r^2) r_hat, grad theta = theta_hat / r,
      // grad phi = phi_hat / (r sin theta)   (analytic derivative of the interpolant, reading R1)
      const T ir = T(1) / r;
      const T nr = (n0 * xr + n1 * yr + n2 * zr) * ir;
      const T nth = n0 * cth * cph + n1 * cth * sph - n2 * sth;
      const T nph = -n0 * sph + n1 * cph;
      Q.as = -(h * ir * ir) * nr * two_ids;
      Q.at = nth * ir * two_idth;
      const T sthg = sth > T(1e-7) ? sth : T(1e-7);
      Q.ap = nph * ir / sthg * two_idth;
      // centred factor G = e^{i k r}/(4 pi r) and its normal derivative (n.r_hat)(i k - 1/r) G
      const T g = T(1.0 / (4.0 * kPi)) * ir;
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        const T kap = kk ? A.ki : A.ke;
        T sn, cs;
        sincos_t(kap * r, &sn, &cs);
        const T Gr = g * cs, Gi = g * sn;
        Q.G[kk][0] = Gr;
        Q.G[kk][1] = Gi;
        Q.G[kk][2] = nr * (-ir * Gr - kap * Gi);
        Q.G[kk][3] = nr * (-ir * Gi + kap * Gr);
      }
      Q.slot = slot;
    }
    __syncwarp();
    for (int cI = 0; cI < nc; ++cI) {
      const TgtScal<T>& Q = S[cI];
      const T* C = A.coefs + (size_t)Q.slot * kQ * 32 + lane;
      // separable contraction: the phi sums with T and T' are shared by F and its three
      // partial derivatives, dF = a_s F_s + a_theta F_theta + a_phi F_phi
      T Tp[5], dTp[5], Tt[5], dTt[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        Tp[k] = Q.Tp[k]; dTp[k] = Q.dTp[k]; Tt[k] = Q.Tt[k]; dTt[k] = Q.dTt[k];
      }
      // all 75 coefficient loads are issued before the arithmetic: one round trip per pair
      T cc[kQ];
#pragma unroll
      for (int k = 0; k < kQ; ++k) cc[k] = __ldg(C + k * 32);
      T Fs[3], Ft[3], Fp[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        Fs[i] = Ft[i] = Fp[i] = T(0);
#pragma unroll
        for (int j = 0; j < 5; ++j) {
          const T* c = cc + (i * 5 + j) * 5;
          T d = Tp[0] * c[0], e = dTp[0] * c[0];
#pragma unroll
          for (int k = 1; k < 5; ++k) {
            d += Tp[k] * c[k];
            e += dTp[k] * c[k];
          }
          Fs[i] += Tt[j] * d;    // -> F and dF/d(ts)
          Ft[i] += dTt[j] * d;   // -> dF/d(tt)
          Fp[i] += Tt[j] * e;    // -> dF/d(tp)
        }
      }
      const T F = Q.Ts[0] * Fs[0] + Q.Ts[1] * Fs[1] + Q.Ts[2] * Fs[2];
      const T dF = Q.as * (Q.dTs[0] * Fs[0] + Q.dTs[1] * Fs[1] + Q.dTs[2] * Fs[2]) +
                   Q.at * (Q.Ts[0] * Ft[0] + Q.Ts[1] * Ft[1] + Q.Ts[2] * Ft[2]) +
                   Q.ap * (Q.Ts[0] * Fp[0] + Q.Ts[1] * Fp[1] + Q.Ts[2] * Fp[2]);
      const T Gr = Q.G[ks][0], Gi = Q.G[ks][1], dGr = Q.G[ks][2], dGi = Q.G[ks][3];
      const T Fw = __shfl_xor_sync(0xffffffffu, F, 1);
      const T dFw = __shfl_xor_sync(0xffffffffu, dF, 1);
      const bool odd = lane & 1;
      const T Fr = odd ? Fw : F, Fi = odd ? F : Fw;
      const T dFr = odd ? dFw : dF, dFi = odd ? dF : dFw;
      accS += odd ? (Gr * Fi + Gi * Fr) : (Gr * Fr - Gi * Fi);
      const T Dr = dGr * Fr - dGi * Fi + Gr * dFr - Gi * dFi;
      const T Di = dGr * Fi + dGi * Fr + Gr * dFi + Gi * dFr;
      accD += odd ? Di : Dr;
    }
    __syncwarp();
  }
  T* out = A.f28 + 56 * (size_t)A.perm[t];
  out[lane] += accS;
  const int dens = (lane >> 1) & 7;
  if (dens < 6) out[2 * (16 + 6 * ks + dens) + (lane & 1)] += accD;
}

template <typename T>
cudaError_t run_ifgf(ifgf_plan_t* p, cudaStream_t s, int nrhs) {
  const int D = p->tree.D;
  const T ke = (T)p->desc.k_ext, ki = (T)p->desc.k_int;
  {
    const DevLevel& L = p->dl[D];
    LeafArgs<T> A{L.box_pt_ptr, L.box_slot_ptr, L.slot_cone, L.box_center, cone_geom_t<T>(L.cg),
                  p->x_sorted, (const T*)p->a_sorted, (T*)L.coefs, ke, ki, 16 * (size_t)p->N, L.cstride};
    int rec = timer_begin(p, TK_LEAF, s);
    if (L.nboxes > 0 && L.max_box_slots > 0) {
      const dim3 grid((unsigned)L.nboxes, (unsigned)((L.max_box_slots + kLeafSlots - 1) / kLeafSlots),
                      (unsigned)nrhs);
      k_leaf<T><<<grid, kLeafThreads, 0, s>>>(A);
    }
    timer_end(p, rec, s);
    ++p->launches;
  }
  for (int d = D; d >= 3; --d) {
    const DevLevel& L = p->dl[d];
    TgtArgs<T> B{p->N, L.tgt_ptr, L.tgt_slot, L.slot_box, L.slot_cone, L.box_center, cone_geom_t<T>(L.cg),
                 (const T*)L.coefs, p->x_sorted, p->n_sorted, p->perm, (T*)p->f28, ke, ki, L.cstride};
    int rec = timer_begin(p, TK_TARGET, s);
    k_target<T><<<dim3((unsigned)((p->N + tgt_warps<T>() - 1) / tgt_warps<T>()), nrhs), 32 * tgt_warps<T>(), 0,
                  s>>>(B);
    timer_end(p, rec, s);
    ++p->launches;
    if (d > 3) {
      const DevLevel& Pp = p->dl[d - 1];
      UpArgs<T> U{Pp.slot_box, Pp.slot_cone, Pp.slot_upidx, Pp.child, cone_geom_t<T>(Pp.cg),
                  L.cmap, L.ncomp, L.ckeys, cone_geom_t<T>(L.cg), L.H, Pp.up_cc, (const T*)L.coefs, (T*)Pp.coefs, ke, ki,
                  L.cstride, Pp.cstride};
      rec = timer_begin(p, TK_UP, s);
      if (Pp.nslots > 0) {
        if constexpr (std::is_same<T, float>::value)
          k_up_runs<<<dim3(Pp.nslots, nrhs), 32 * kUpRunWarps, kUpRunSmem, s>>>(
              U, RunTabs{Pp.up_order, Pp.up_task, Pp.up_task_ptr});
        else
          k_up<T><<<dim3(Pp.nslots, nrhs), kUpThreads, 0, s>>>(U);
      }
      timer_end(p, rec, s);
      ++p->launches;
    }
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t setup_ifgf_kernels() {
  return cudaFuncSetAttribute(k_up_runs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUpRunSmem);
}

cudaError_t launch_far_ifgf(ifgf_plan_t* p, cudaStream_t s, int nrhs) {
  if (p->desc.precision == IFGF_FP64) return run_ifgf<double>(p, s, nrhs);
  return run_ifgf<float>(p, s, nrhs);
}

}  // namespace ifgf
