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
#include "ifgf_dev.cuh"

namespace ifgf {

namespace {

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
  if (A.img) A.img += blockIdx.z * A.istride;
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
    vals_to_coefs_block<T, kVS>(M, vbuf, A.coefs + (size_t)s0 * kQ * 32, min(2, se - s0),
                                A.img ? A.img + (size_t)s0 * kImgFloats : nullptr);
  }
}

// (a), FP32 on the tensor pipe: the same sums as k_leaf with the density products as warp-level
// TF32 matrix multiply-accumulates (mma.sync m16n8k8, three-term hi/lo split for FP32 accuracy,
// FP32 accumulation).  Per kernel kappa, with g_pj = (r / |X_p - y_j|) e^{i kappa (|X_p - y_j| - r)}
// and the 8 complex densities a_jd, the values V_pd = sum_j g_pj a_jd are one real product
//   V[p][(d, part)] = sum_{(j, s)} A[p][(j, s)] B[(j, s)][(d, part)],
//   A[p][(j, 0)] = Re g_pj, A[p][(j, 1)] = Im g_pj,
//   B[(j, 0)][(d, re)] = Re a_jd, B[(j, 1)][(d, re)] = -Im a_jd,
//   B[(j, 0)][(d, im)] = Im a_jd, B[(j, 1)][(d, im)] = Re a_jd,
// 16 points x 8 (4 sources x 2) per step.  Each lane evaluates g for exactly the entries of the A
// fragment it holds (points groupID and groupID + 8 of the tile, source threadID_in_group), both
// kernels from one distance, so the kernel values never leave registers; B comes from the staged
// densities.  A block takes the 2 x 75 points of two cone segments as 10 tiles of 16, two per warp
// (5 warps), then the values -> coefficients map and stores of k_leaf.
constexpr int kLeafMmaWarps = 5;

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(32 * kLeafMmaWarps, 4) k_leaf_mma(LeafArgs<float> A) {
  using T = float;
  __shared__ SmallMaps<T> M;
  __shared__ T pool[kLeafChunk * 20 + 2 * kQ * kVS];
  T (*src)[4] = reinterpret_cast<T (*)[4]>(pool);
  T (*sa)[16] = reinterpret_cast<T (*)[16]>(pool + kLeafChunk * 4);
  T* vbuf = pool + kLeafChunk * 20;
  const int box = blockIdx.x;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int gid = lane >> 2, tig = lane & 3;
  A.a_sorted += blockIdx.z * A.astride;   // right-hand side of a batched call
  A.coefs += blockIdx.z * A.cstride;
  if (A.img) A.img += blockIdx.z * A.istride;
  const int sb = A.box_slot_ptr[box] + blockIdx.y * kLeafSlots;
  const int se = min(A.box_slot_ptr[box + 1], sb + kLeafSlots);
  if (sb >= se) return;   // uniform per block
  init_maps(M);
  const double c0 = A.box_center[3 * box], c1 = A.box_center[3 * box + 1], c2 = A.box_center[3 * box + 2];
  const int pb = A.box_pt_ptr[box], pe = A.box_pt_ptr[box + 1];
  const int nsrc = pe - pb;
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
  const bool staged_once = nsrc <= kLeafChunk;
  if (staged_once) stage(0, nsrc);
  for (int s0 = sb; s0 < se; s0 += 2) {
    __syncthreads();
    // tiles 2 warp and 2 warp + 1 of the pass: tile u covers points 16 (u % 5) .. of slot s0 + u / 5
    float acc[2][2][2][4];   // [tile][kernel][n-tile][fragment]
    T X[2][2][3], R[2][2];   // [tile][row half] point and its distance to the box centre
    bool tile_on[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int u = 2 * warp + h, sl = u / 5, q0 = 16 * (u % 5);
      tile_on[h] = s0 + sl < se;
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int q = min(q0 + gid + 8 * r, kQ - 1);   // rows beyond 75 repeat the last point
        X[h][r][0] = X[h][r][1] = X[h][r][2] = T(0);
        if (tile_on[h]) cone_point(M, A.cg, A.slot_cone[s0 + sl], q, X[h][r]);
        R[h][r] = sqrt_t(X[h][r][0] * X[h][r][0] + X[h][r][1] * X[h][r][1] + X[h][r][2] * X[h][r][2]);
      }
#pragma unroll
      for (int ks = 0; ks < 2; ++ks)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
          for (int i = 0; i < 4; ++i) acc[h][ks][nt][i] = 0.f;
    }
    for (int cb = 0; cb < nsrc; cb += kLeafChunk) {
      const int nchunk = min(kLeafChunk, nsrc - cb);
      if (!staged_once) {
        __syncthreads();
        stage(cb, nchunk);
        __syncthreads();
      }
      for (int j0 = 0; j0 < nchunk; j0 += 4) {
        const int j = j0 + tig;
        const bool jon = j < nchunk;
        // B fragments (shared by both tiles and both kernels): rows (s, j) = (0, tig), (1, tig),
        // column 8 nt + gid = (density, part)
        uint32_t bh[2][2], bl[2][2];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          const int c = 8 * nt + gid, dd = c >> 1, im = c & 1;
          const T ar = jon ? sa[j][2 * dd] : T(0), ai = jon ? sa[j][2 * dd + 1] : T(0);
          const T b0 = im ? ai : ar, b1 = im ? ar : -ai;
          const T h0 = tf32_hi(b0), h1 = tf32_hi(b1);
          bh[nt][0] = __float_as_uint(h0);
          bh[nt][1] = __float_as_uint(h1);
          bl[nt][0] = __float_as_uint(b0 - h0);
          bl[nt][1] = __float_as_uint(b1 - h1);
        }
        const T sy0 = jon ? src[j][0] : T(0), sy1 = jon ? src[j][1] : T(0), sy2 = jon ? src[j][2] : T(0);
        const T sy3 = jon ? src[j][3] : T(0);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (!tile_on[h]) continue;   // warp-uniform
          // A fragments: a0 (row gid, Re), a1 (row gid + 8, Re), a2 (row gid, Im), a3 (row gid + 8, Im)
          uint32_t ah[2][4], al[2][4];
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            // g_S(X, y) = (r/|X-y|) exp(i k (|X-y| - r)), |X-y| - r = (|y|^2 - 2 X.y)/(|X-y| + r)
            const T rr = R[h][r];
            const T dxy = sy3 - T(2) * (X[h][r][0] * sy0 + X[h][r][1] * sy1 + X[h][r][2] * sy2);
            const T d = sqrt_t(rr * rr + dxy);
            const T rd = jon ? leaf_div(rr, d) : T(0);
            const T dd = leaf_div(dxy, d + rr);
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
              T sn, cs;
              leaf_sincos(kk[ks] * dd, &sn, &cs);
              const T gr = rd * cs, gi = rd * sn;
              const T hr = tf32_hi(gr), hi = tf32_hi(gi);
              ah[ks][r] = __float_as_uint(hr);
              ah[ks][r + 2] = __float_as_uint(hi);
              al[ks][r] = __float_as_uint(gr - hr);
              al[ks][r + 2] = __float_as_uint(gi - hi);
            }
          }
          // the three split terms of the four (kernel, n-tile) accumulators, term-major: four
          // independent products between two that share an accumulator
#pragma unroll
          for (int ks = 0; ks < 2; ++ks)
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) mma_tf32(acc[h][ks][nt], ah[ks], bh[nt]);
#pragma unroll
          for (int ks = 0; ks < 2; ++ks)
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) mma_tf32(acc[h][ks][nt], ah[ks], bl[nt]);
#pragma unroll
          for (int ks = 0; ks < 2; ++ks)
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) mma_tf32(acc[h][ks][nt], al[ks], bh[nt]);
        }
      }
    }
    // D fragments -> values: c0 (row gid, column 2 tig), c1 (+1), c2 / c3 (row gid + 8)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (!tile_on[h]) continue;
      const int u = 2 * warp + h, sl = u / 5, q0 = 16 * (u % 5);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int q = q0 + gid + 8 * (i >> 1);
        if (q >= kQ) continue;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks)
#pragma unroll
          for (int nt = 0; nt < 2; ++nt)
            vbuf[(sl * kQ + q) * kVS + 16 * ks + 8 * nt + 2 * tig + (i & 1)] = acc[h][ks][nt][i];
      }
    }
    __syncthreads();
    vals_to_coefs_block<T, kVS>(M, vbuf, A.coefs + (size_t)s0 * kQ * 32, min(2, se - s0),
                                A.img ? A.img + (size_t)s0 * kImgFloats : nullptr);
  }
}

// ------------------------------------------------------------------ (b) upward pass
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
// separably (over phi, then theta, then s: 74 FMA per lane), two points at a time
// (two independent FMA streams per warp).  The right-hand sides of a batched call are taken
// one after the other by the same block, so the prologue serves all of them.  The parent points
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

// The 3D Chebyshev sum of one lane's 75 coefficients c at NP points, contracted separably (phi,
// then theta, then s; T_0 = 1 folded in): 74 FMA per point.  The points' sums are independent,
// so evaluating two at once gives the scheduler two FMA streams that share each coefficient.
template <int NP>
__device__ __forceinline__ void up_contract(const float (&c)[kQ], const float4 (&P4)[NP], const float4 (&T4)[NP],
                                            const float4 (&S4)[NP], float (&v)[NP]) {
  float E[NP][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float e[NP];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      const float* cij = c + (i * 5 + j) * 5;
#pragma unroll
      for (int n = 0; n < NP; ++n) {
        float d = cij[0];
        d = fmaf(P4[n].x, cij[1], d);
        d = fmaf(P4[n].y, cij[2], d);
        d = fmaf(P4[n].z, cij[3], d);
        d = fmaf(P4[n].w, cij[4], d);
        const float tt = j == 1 ? T4[n].x : j == 2 ? T4[n].y : j == 3 ? T4[n].z : T4[n].w;
        e[n] = j == 0 ? d : fmaf(tt, d, e[n]);
      }
    }
#pragma unroll
    for (int n = 0; n < NP; ++n) E[n][i] = e[n];
  }
#pragma unroll
  for (int n = 0; n < NP; ++n) v[n] = fmaf(S4[n].y, E[n][2], fmaf(S4[n].x, E[n][1], E[n][0]));
}

constexpr int kUpRunWarps = kUpGroups;   // warp w adds only into the parent points of group w

// dynamic shared memory of k_up_runs (above the 48 KB static limit)
constexpr size_t kUpRunSmem = sizeof(UpCheb) * 8 * kQ      // Chebyshev values per (octant, point)
                              + sizeof(float4) * 8 * kQ    // re-centring factors (re, im) x 2 kernels
                              + sizeof(int) * 8 * kQ       // child slot per (octant, point) of the current slot
                              + sizeof(float) * kQ * kVS   // parent values
                              + sizeof(float) * kQ * 3;    // parent points

__global__ void __launch_bounds__(32 * kUpRunWarps, 4) k_up_runs(UpArgs<float> A, RunTabs RT, int nrhs,
                                                                   const int* __restrict__ items) {
  using T = float;
  __shared__ SmallMaps<T> M;
  extern __shared__ float4 up_smem[];
  UpCheb (*cheb)[kQ] = reinterpret_cast<UpCheb (*)[kQ]>(up_smem);
  float4 (*fac)[kQ] = reinterpret_cast<float4 (*)[kQ]>(cheb + 8);
  int (*cslot)[kQ] = reinterpret_cast<int (*)[kQ]>(fac + 8);
  T* vals = reinterpret_cast<T*>(cslot + 8);
  T (*Xp)[3] = reinterpret_cast<T (*)[3]>(vals + kQ * kVS);
  const int t = threadIdx.x, warp = t / 32, lane = t % 32;
  // the block's parent slots: one, or (items) up to kTcBoxes slots of one parent cone in other
  // boxes, whose geometry (child cones, local coordinates, re-centring factors) is the same
  int slots[kTcBoxes], nsl = 1, omask = 0;
  slots[0] = items ? __ldg(items + (size_t)blockIdx.x * kTcBoxes) : (int)blockIdx.x;
#pragma unroll
  for (int b = 1; b < kTcBoxes; ++b) {
    slots[b] = items ? __ldg(items + (size_t)blockIdx.x * kTcBoxes + b) : -1;
    nsl += slots[b] >= 0;
  }
#pragma unroll
  for (int b = 0; b < kTcBoxes; ++b)
    if (slots[b] >= 0)
      for (int o = 0; o < 8; ++o) omask |= (__ldg(A.child + 8 * __ldg(A.slot_box + slots[b]) + o) >= 0) << o;
  init_maps(M);
  const int ci = A.slot_upidx[slots[0]];
  const cone_key pcone = A.slot_cone[slots[0]];
  __syncthreads();
  if (t < kQ) cone_point(M, A.cgp, pcone, t, Xp[t]);
  __syncthreads();
  const T off = (T)(0.5 * A.Hc);
  const T kk[2] = {A.ke, A.ki};
  // prologue: per (octant, parent point) the Chebyshev values of the point's local coordinates in
  // its child cone and the re-centring factor of both kernels (octants with a child in some box)
  for (int e = t; e < 8 * kQ; e += blockDim.x) {
    const int o = e / kQ, q = e % kQ;
    if (!((omask >> o) & 1)) continue;
    const T ox = (o & 1) ? off : -off, oy = (o & 2) ? off : -off, oz = (o & 4) ? off : -off;
    const T x = Xp[q][0] - ox, y = Xp[q][1] - oy, z = Xp[q][2] - oz;
    const int ccx = A.up_cc[((size_t)ci * 8 + o) * kQ + q];
    const cone_key cc = A.ckeys_c[ccx];
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
  const int w0 = __ldg(RT.task_ptr + (size_t)ci * kUpGroups + warp);
  const int w1 = __ldg(RT.task_ptr + (size_t)ci * kUpGroups + warp + 1);
  // the slots, and the right-hand sides of a batched call, one after the other: the prologue's
  // geometry serves all of them
  for (int b = 0; b < nsl; ++b) {
    const int pslot = slots[b], P = __ldg(A.slot_box + pslot);
    // the child slot of every (octant, parent point) of this slot, so that a run finds its child
    // coefficients with one shared-memory read (the barrier after the clearing of vals below
    // publishes it; the barrier that ends the previous slot's last right-hand side retired the
    // previous table's readers)
    for (int e = t; e < 8 * kQ; e += blockDim.x) {
      const int o = e / kQ, q = e % kQ;
      const int cb = __ldg(A.child + 8 * P + o);
      if (cb >= 0) cslot[o][q] = __ldg(A.cmap_c + (size_t)cb * A.ncomp_c + __ldg(A.up_cc + ((size_t)ci * 8 + o) * kQ + q));
    }
    for (int rb = 0; rb < nrhs; ++rb) {
      const T* coefs_c = A.coefs_c + rb * A.cstride_c;
      for (int e = t; e < kQ * kVS; e += blockDim.x) vals[e] = T(0);
      __syncthreads();
      // the warp's own runs (its group of parent points, all octants); runs of absent children
      // are skipped.  Only this warp adds into these points' values: plain shared-memory adds.
      for (int w = w0; w < w1; ++w) {
        const int tk = __ldg(RT.task + w);
        const int r0 = tk & 255, len = (tk >> 8) & 255, o = (tk >> 16) & 7;
        if (A.child[8 * P + o] < 0) continue;
        const size_t g = (size_t)ci * 8 + o;
        const int myq = lane < len ? __ldg(RT.order + g * kQ + r0 + lane) : 0;
        // one child slot per run (the host marked every such cone relevant)
        const int q0 = __shfl_sync(0xffffffffu, myq, 0);
        const T* Cg = coefs_c + (size_t)cslot[o][q0] * kQ * 32 + lane;
        T c[kQ];
#pragma unroll
        for (int k = 0; k < kQ; ++k) c[k] = __ldg(Cg + k * 32);
        int a = 0;
        for (; a + 1 < len; a += 2) {   // two points at a time (independent sums, distinct points)
          int q[2];
          float4 P4[2], T4[2], S4[2];
          float2 F2[2];
          float v[2];
#pragma unroll
          for (int n = 0; n < 2; ++n) {
            q[n] = __shfl_sync(0xffffffffu, myq, a + n);
            const float4* cp = reinterpret_cast<const float4*>(&cheb[o][q[n]]);
            P4[n] = cp[0]; T4[n] = cp[1]; S4[n] = cp[2];
            F2[n] = reinterpret_cast<const float2*>(&fac[o][q[n]])[ks];   // this lane's kernel: (re, im)
          }
          up_contract<2>(c, P4, T4, S4, v);
#pragma unroll
          for (int n = 0; n < 2; ++n) {
            const T wv = __shfl_xor_sync(0xffffffffu, v[n], 1);
            vals[q[n] * kVS + lane] += fmaf(v[n], F2[n].x, sgn * F2[n].y * wv);
          }
        }
        if (a < len) {
          const int q = __shfl_sync(0xffffffffu, myq, a);
          const float4* cp = reinterpret_cast<const float4*>(&cheb[o][q]);
          const float4 P4[1] = {cp[0]}, T4[1] = {cp[1]}, S4[1] = {cp[2]};
          const float2 F2 = reinterpret_cast<const float2*>(&fac[o][q])[ks];
          float v[1];
          up_contract<1>(c, P4, T4, S4, v);
          const T wv = __shfl_xor_sync(0xffffffffu, v[0], 1);
          vals[q * kVS + lane] += fmaf(v[0], F2.x, sgn * F2.y * wv);
        }
      }
      __syncthreads();
      vals_to_coefs_block<T, kVS>(M, vals, A.coefs_p + rb * A.cstride_p + (size_t)pslot * kQ * 32, 1,
                                  A.img_p ? A.img_p + rb * A.istride_p + (size_t)pslot * kImgFloats : nullptr);
      __syncthreads();   // vals is cleared for the next right-hand side
    }
  }
}

// (b), FP32 variant with a warp per parent slot.  The warp walks the slot's units (the points of
// one octant that fall in one child cone, at most kUpRunMax of them, from the unit tables): it
// loads the child cone's 75 x 32 coefficients once per unit into registers (75 per lane) and
// sweeps the unit's points with the separable contraction of k_up_runs.  Owning the whole slot,
// the warp adds every octant's contributions into its own parent values with plain shared-memory
// adds, so the units need no split by point groups (about 3.2 units per octant against 8.2 runs
// per octant in k_up_runs, at 23 points per unit on average) and no block barrier follows the
// prologue: per octant the warp forms the Chebyshev values and re-centring factors of its points
// itself, and at the end transforms its values to coefficients column by column (lane = column).
// Measured on GB300 it is 1.1-1.3x slower than k_up_runs on the sphere workloads despite 12 %
// fewer instructions (14 warps per SM, the per-octant prologue and each unit's coefficient loads
// are not overlapped: issue 41 % against 57 %), so it is an autotuner candidate, not the default.
struct UnitTabs {
  const int* order;      // [ncompact][8][75] points ranked by child cone
  const int* unit;       // units per compact cone, in octant order: start | len << 8 | octant << 16
  const int* unit_ptr;   // [ncompact + 1]
};

struct __align__(16) UpPoint {   // per parent point of the current octant
  float tp[4];
  float tt[4];
  float ts[2];
  float pad[2];
  float4 fac;                    // re-centring factors (re, im) of kernels e and i
};

constexpr int kUpWarpW = 2;   // warps (parent slots) per block
constexpr size_t kUpWarpBytes = sizeof(float) * kQ * 32 + sizeof(UpPoint) * kQ + sizeof(float) * kQ * 4;
constexpr size_t kUpWarpSmem = kUpWarpW * kUpWarpBytes;

__global__ void __launch_bounds__(32 * kUpWarpW, 7) k_up_warp(UpArgs<float> A, UnitTabs UT, int nslots) {
  using T = float;
  __shared__ SmallMaps<T> M;
  extern __shared__ float4 upw_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* base = reinterpret_cast<unsigned char*>(upw_smem) + warp * kUpWarpBytes;
  T* vals = reinterpret_cast<T*>(base);                                        // [75][32]
  UpPoint* pt = reinterpret_cast<UpPoint*>(base + sizeof(float) * kQ * 32);   // [75]
  T (*Xp)[4] = reinterpret_cast<T (*)[4]>(pt + kQ);                           // [75] parent points
  A.coefs_c += blockIdx.y * A.cstride_c;   // right-hand side of a batched call
  A.coefs_p += blockIdx.y * A.cstride_p;
  init_maps(M);
  __syncthreads();
  const int pslot = blockIdx.x * kUpWarpW + warp;
  if (pslot >= nslots) return;   // no block barrier follows
  const int P = __ldg(A.slot_box + pslot), ci = __ldg(A.slot_upidx + pslot);
  const cone_key pcone = A.slot_cone[pslot];
  for (int q = lane; q < kQ; q += 32) {
    cone_point(M, A.cgp, pcone, q, Xp[q]);
    Xp[q][3] = sqrt_t(Xp[q][0] * Xp[q][0] + Xp[q][1] * Xp[q][1] + Xp[q][2] * Xp[q][2]);
  }
  for (int e = lane; e < kQ * 32; e += 32) vals[e] = T(0);
  __syncwarp();
  const T off = (T)(0.5 * A.Hc);
  const T kk[2] = {A.ke, A.ki};
  const int ks = lane >> 4;
  const T sgn = (lane & 1) ? T(1) : T(-1);
  const int u1 = __ldg(UT.unit_ptr + ci + 1);
  int u = __ldg(UT.unit_ptr + ci);
  for (int o = 0; o < 8 && u < u1; ++o) {
    int ue = u;   // units of octant o: [u, ue)
    while (ue < u1 && ((__ldg(UT.unit + ue) >> 16) & 7) == o) ++ue;
    const int cb = __ldg(A.child + 8 * P + o);
    if (cb < 0 || ue == u) {
      u = ue;
      continue;
    }
    const size_t g = (size_t)ci * 8 + o;
    // the octant's points: Chebyshev values in their child cone and the re-centring factor
    const T ox = (o & 1) ? off : -off, oy = (o & 2) ? off : -off, oz = (o & 4) ? off : -off;
    for (int q = lane; q < kQ; q += 32) {
      const int ccx = __ldg(A.up_cc + g * kQ + q);
      if (ccx < 0) continue;
      const T x = Xp[q][0] - ox, y = Xp[q][1] - oy, z = Xp[q][2] - oz;
      T ts, tt, tp, rc, sth, cth, sph, cph;
      local_coords(A.cgc, A.ckeys_c[ccx], x, y, z, &ts, &tt, &tp, &rc, &sth, &cth, &sph, &cph);
      T v5[5], v3[3];
      UpPoint& C = pt[q];
      cheb_vals<T, 5>(tp, v5);
      C.tp[0] = v5[1]; C.tp[1] = v5[2]; C.tp[2] = v5[3]; C.tp[3] = v5[4];
      cheb_vals<T, 5>(tt, v5);
      C.tt[0] = v5[1]; C.tt[1] = v5[2]; C.tt[2] = v5[3]; C.tt[3] = v5[4];
      cheb_vals<T, 3>(ts, v3);
      C.ts[0] = v3[1]; C.ts[1] = v3[2];
      // re-centring factor G(x, x_child)/G(x, x_parent) = (r_p/r_c) e^{i k (r_c - r_p)}
      const T rp = Xp[q][3];
      const T dr = (T(3) * off * off - T(2) * (Xp[q][0] * ox + Xp[q][1] * oy + Xp[q][2] * oz)) / (rc + rp);
      T sn0, cs0, sn1, cs1;
      sincos_t(kk[0] * dr, &sn0, &cs0);
      sincos_t(kk[1] * dr, &sn1, &cs1);
      const T a = rp / rc;
      C.fac = make_float4(a * cs0, a * sn0, a * cs1, a * sn1);
    }
    __syncwarp();
    for (; u < ue; ++u) {
      const int tk = __ldg(UT.unit + u);
      const int r0 = tk & 255, len = (tk >> 8) & 255;
      const int myq = lane < len ? __ldg(UT.order + g * kQ + r0 + lane) : 0;
      const int q0 = __shfl_sync(0xffffffffu, myq, 0);
      const int cslot = __ldg(A.cmap_c + (size_t)cb * A.ncomp_c + __ldg(A.up_cc + g * kQ + q0));
      if (cslot < 0) continue;   // cannot happen: the host marked every such cone relevant
      const T* Cg = A.coefs_c + (size_t)cslot * kQ * 32 + lane;
      T c[kQ];
#pragma unroll
      for (int k = 0; k < kQ; ++k) c[k] = __ldg(Cg + k * 32);
      for (int a = 0; a < len; ++a) {   // one point at a time (measured faster here than two)
        const int q = __shfl_sync(0xffffffffu, myq, a);
        const float4* cp = reinterpret_cast<const float4*>(&pt[q]);
        const float4 P4[1] = {cp[0]}, T4[1] = {cp[1]}, S4[1] = {cp[2]};
        const float4 F4 = cp[3];
        float v[1];
        up_contract<1>(c, P4, T4, S4, v);
        const T wv = __shfl_xor_sync(0xffffffffu, v[0], 1);
        const T fr = ks ? F4.z : F4.x, fi = ks ? F4.w : F4.y;
        vals[q * 32 + lane] += fmaf(v[0], fr, sgn * fi * wv);
      }
    }
    __syncwarp();   // the next octant's prologue overwrites pt
  }
  // values -> coefficients, lane = column, and a coalesced store
  vals_to_coefs_col(M, vals + lane, 32);
  T* out = A.coefs_p + (size_t)pslot * kQ * 32 + lane;
  for (int q = 0; q < kQ; ++q) out[q * 32] = vals[q * 32 + lane];
  if (A.img_p) {   // tensor-core operand image: lane = row m
    float* im = A.img_p + blockIdx.y * A.istride_p + (size_t)pslot * kImgFloats;
    for (int kc = 0; kc < 20; ++kc) {
      float x[4], h[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int k = 4 * kc + j;
        x[j] = k < kQ ? vals[k * 32 + lane] : 0.f;
        h[j] = tf32_hi(x[j]);
      }
      *reinterpret_cast<float4*>(im + img_off(lane, kc)) = make_float4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<float4*>(im + kImgFloats / 2 + img_off(lane, kc)) =
          make_float4(x[0] - h[0], x[1] - h[1], x[2] - h[2], x[3] - h[3]);
    }
  }
}

// ------------------------------------------------------------------ (b) on the tensor cores
// The upward step as dense contractions on the 5th-generation tensor cores (tcgen05, kind::tf32,
// FP32 accumulation in tensor memory).  A block takes kTcBoxes parent slots of one parent cone
// (their parent points, child cones and re-centring factors are box-independent) and sweeps the
// cone's units: the points of one octant that fall in one child cone (at most 32).  Per unit
//   D[(box, field) x point] = C^T[(box, field) x k] . B[k x point],  M = 128, N = 32, K = 80,
// with C the child cones' 75 x 32 coefficients (A operand) and B the Chebyshev basis
// T_i(s) T_j(theta) T_k(phi) of the unit's points, both K-major without swizzle (8-row x 16-byte
// core matrices), K padded from 75 to 80 with zeros.  FP32 accuracy comes from a three-term split
// x = hi + lo (hi = x with the 13 low mantissa bits cleared, exactly the TF32 operand):
// D = A_hi B_hi + A_hi B_lo + A_lo B_hi.
// The A operand needs no staging by threads: the kernel that produced the child coefficients
// also wrote them as operand images (img_off: hi and lo parts, the K-major core-matrix layout),
// and one bulk asynchronous copy per (box, part) moves an image into shared memory, completing on
// an mbarrier.  The copy for unit u+1 is issued as soon as the MMAs of unit u have read the A
// buffer, so it runs under unit u's epilogue and unit u+1's basis.  The parent values of the four
// slots accumulate in tensor memory (lane = (box, field), column = parent point), next to the
// unit's accumulator D; the epilogue (warp w = box w, the tensor-memory lanes it may access)
// re-centres D's columns and adds them into the parent columns, and at the end each thread
// transforms its own column of 75 values to coefficients in registers and writes them, and their
// operand images when the level above also runs on the tensor cores.
// Measured on GB300 it is 2.4-2.6x slower than the SIMT kernel k_up_runs (upward step 19.2 against
// 7.3 ms at 9,600 nodes, 150 against 63 ms at 153,600): the MMAs remove the 74 contraction FMAs of
// a (parent point, child) pair, but the pair's share of the basis, the re-centring of its 32
// columns and its scatter-add (~60 warp instructions) remain, since a coefficient block serves
// only ~20 points, and 8 warps per SM do not hide the serial chain of a unit.  Plan option, not
// the default.
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* ptr) { return (uint32_t)__cvta_generic_to_shared(ptr); }

// shared-memory matrix descriptor: start address, leading / stride byte offsets, layout
// (0: no swizzle), descriptor version 1
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t layout) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46) | ((uint64_t)(layout & 7) << 61);
}
// instruction descriptor, kind::tf32: D FP32, A and B TF32, both K-major
__host__ __device__ constexpr uint32_t idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma(uint32_t td, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(td),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// arm an mbarrier for `bytes` of bulk-copy transactions (one arrival)
__device__ __forceinline__ void expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// bulk asynchronous copy global -> shared of `bytes` (multiple of 16, both addresses 16-byte
// aligned), completing its transactions on `bar`
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// wait for phase `parity` of an mbarrier, giving up after `limit_ns` nanoseconds or kWaitPolls
// polls, whichever comes first; true when the phase completed
constexpr int kWaitPolls = 1 << 26;
__device__ __forceinline__ bool wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  uint32_t done = 0;
  const uint64_t t0 = now_ns();
  for (int it = 0; it < kWaitPolls && !done; ++it) {
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    if (!done && now_ns() - t0 > limit_ns) break;
  }
  return done != 0;
}
// tensor-memory loads and stores of this warp's 32 lanes (32x32b shapes)
__device__ __forceinline__ void ld_x32(uint32_t ta, float (&r)[32]) {
  uint32_t* u = reinterpret_cast<uint32_t*>(r);
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]), "=r"(u[8]),
        "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]), "=r"(u[16]),
        "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]), "=r"(u[24]),
        "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31])
      : "r"(ta));
}
__device__ __forceinline__ void ld_x16(uint32_t ta, float* r) {
  uint32_t* u = reinterpret_cast<uint32_t*>(r);
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]), "=r"(u[8]),
        "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
      : "r"(ta));
}
__device__ __forceinline__ void ld_x1(uint32_t ta, float& r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(*reinterpret_cast<uint32_t*>(&r)) : "r"(ta));
}
__device__ __forceinline__ void st_x1(uint32_t ta, float v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(ta), "r"(__float_as_uint(v)) : "memory");
}
__device__ __forceinline__ void st_x16_zero(uint32_t ta) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(ta),
      "r"(0u)
      : "memory");
}
// wait for this thread's single-column loads; the registers are operands, so no use of them is
// scheduled before the wait
__device__ __forceinline__ void wait_ld_regs(float (&r)[32]) {
  uint32_t* u = reinterpret_cast<uint32_t*>(r);
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(u[0]), "+r"(u[1]), "+r"(u[2]), "+r"(u[3]), "+r"(u[4]), "+r"(u[5]), "+r"(u[6]), "+r"(u[7]),
                 "+r"(u[8]), "+r"(u[9]), "+r"(u[10]), "+r"(u[11]), "+r"(u[12]), "+r"(u[13]), "+r"(u[14]), "+r"(u[15]),
                 "+r"(u[16]), "+r"(u[17]), "+r"(u[18]), "+r"(u[19]), "+r"(u[20]), "+r"(u[21]), "+r"(u[22]),
                 "+r"(u[23]), "+r"(u[24]), "+r"(u[25]), "+r"(u[26]), "+r"(u[27]), "+r"(u[28]), "+r"(u[29]),
                 "+r"(u[30]), "+r"(u[31])
               :
               : "memory");
}
__device__ __forceinline__ void wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

constexpr int kK = 80;                          // K: 75 Chebyshev terms padded to a multiple of 8
constexpr int kN = 32;                          // N: points of a unit
constexpr int kThreads = 128;                   // 4 warps: warp w is box w in the epilogue
constexpr int kImgBytes = 32 * kK * 4;          // one operand image part (hi or lo) of one slot
constexpr int kCols = 128;                      // tensor-memory columns: parent values 0..79, D 96..127
constexpr int kColD = 96;
// shared memory (1024-byte aligned base): A hi [4 boxes] | A lo [4 boxes] | B hi | B lo | unit
// point data | re-centring factors | parent points | child slots per (box, unit) | unit records
constexpr int kOffAlo = kTcBoxes * kImgBytes;                 // 40960
constexpr int kOffB = 2 * kTcBoxes * kImgBytes;               // 81920
constexpr int kOffBlo = kOffB + kImgBytes;                    // 92160
constexpr int kOffPts = kOffB + 2 * kImgBytes;                // [32] x 3 float4: T values and the point
constexpr int kOffFac = kOffPts + kN * 48;                    // [32] float4
constexpr int kOffXp = kOffFac + kN * 16;                     // [75][4] floats
constexpr int kOffCs = kOffXp + kQ * 16;                      // [kTcBoxes][kTcMaxUnits] ints
constexpr int kOffUnit = kOffCs + kTcBoxes * kTcMaxUnits * 4; // [kTcMaxUnits] ints
constexpr int kSmem = kOffUnit + kTcMaxUnits * 4 + 1024;      // + alignment of the base
static_assert(kOffPts % 16 == 0 && kOffFac % 16 == 0 && kOffXp % 16 == 0, "16-byte aligned regions");
static_assert(2 * (kSmem + 1024) <= 228 * 1024, "two blocks per SM");

// row m, 16-byte chunk kc of a K-major operand without swizzle (bytes): img_off in bytes
__device__ __forceinline__ int kmaj_off(int m, int kc) { return 4 * img_off(m, kc); }

}  // namespace tc

struct TcTabs {
  const int* order;      // [ncompact][8][75] points ranked by child cone
  const int* unit;       // units per compact cone: start | len << 8 | octant << 16
  const int* unit_ptr;   // [ncompact + 1]
  const int* item;       // [nitems][kTcBoxes] parent slots (-1 padded)
  const float* img_c;    // child coefficients' operand images [nslots_c][kImgFloats], per rhs istride_c
  size_t istride_c;
  int* err;              // device status word: bit 0 set when a wait on the tensor cores timed out
  uint64_t wait_ns;      // limit of each wait (1 s; 1 ms under fault injection)
  int inject;            // fault injection: the first unit's MMAs are not issued, so its wait expires
};

// Per unit u (one thread issues the copies and the MMAs; phases of both barriers flip per unit):
//   unit points' coordinates (warp 0) -> basis B(u) (all) -> wait A(u) -> MMA(u) -> wait ->
//   copy A(u+1) (in flight during the rest) -> epilogue(u) into the parent columns.
__global__ void __launch_bounds__(tc::kThreads, 2) k_up_tc(UpArgs<float> A, TcTabs TT) {
  using T = float;
  __shared__ SmallMaps<T> M;
  __shared__ __align__(8) uint64_t bar_a, bar_m;
  __shared__ uint32_t tmem_base;
  __shared__ int nact_s;
  __shared__ int slot[kTcBoxes];
  extern __shared__ __align__(16) unsigned char tc_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~uintptr_t(1023));
  float4* pts = reinterpret_cast<float4*>(sm + tc::kOffPts);   // [32][3]
  float4* fac = reinterpret_cast<float4*>(sm + tc::kOffFac);   // [32]
  T (*Xp)[4] = reinterpret_cast<T (*)[4]>(sm + tc::kOffXp);
  int (*cs)[kTcMaxUnits] = reinterpret_cast<int (*)[kTcMaxUnits]>(sm + tc::kOffCs);
  int* units = reinterpret_cast<int*>(sm + tc::kOffUnit);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  A.coefs_c += blockIdx.y * A.cstride_c;   // right-hand side of a batched call
  A.coefs_p += blockIdx.y * A.cstride_p;
  const float* imgc = TT.img_c + blockIdx.y * TT.istride_c;
  float* imgp = A.img_p ? A.img_p + blockIdx.y * A.istride_p : nullptr;
  if (t < kTcBoxes) slot[t] = __ldg(TT.item + (size_t)blockIdx.x * kTcBoxes + t);
  init_maps(M);
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(&bar_a)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(&bar_m)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&tmem_base)),
                 "r"(tc::kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tm = tmem_base;
  const uint32_t tlane = tm + ((uint32_t)(32 * warp) << 16);   // this warp's tensor-memory lanes
  const int ci = A.slot_upidx[slot[0]];   // every item holds at least one slot, first
  const cone_key pcone = A.slot_cone[slot[0]];
  const int u0 = __ldg(TT.unit_ptr + ci);
  int nunits = __ldg(TT.unit_ptr + ci + 1) - u0;
  for (int e = t; e < nunits; e += blockDim.x) units[e] = __ldg(TT.unit + u0 + e);
  if (t < kQ) {
    cone_point(M, A.cgp, pcone, t, Xp[t]);
    Xp[t][3] = sqrt_t(Xp[t][0] * Xp[t][0] + Xp[t][1] * Xp[t][1] + Xp[t][2] * Xp[t][2]);
  }
  // parent values start at zero (columns 0..79 of every lane)
#pragma unroll
  for (int c = 0; c < 80; c += 16) tc::st_x16_zero(tlane + c);
  tc::wait_st();
  __syncthreads();
  // child slot of every (box, unit): -1 where the box has no child in the unit's octant
  for (int e = t; e < kTcBoxes * nunits; e += blockDim.x) {
    const int b = e / nunits, u = e - b * nunits;
    const int tk = units[u], o = (tk >> 16) & 7;
    const size_t g = (size_t)ci * 8 + o;
    const int q0 = __ldg(TT.order + g * kQ + (tk & 255));
    const int P = slot[b] >= 0 ? __ldg(A.slot_box + slot[b]) : -1;
    const int cb = P >= 0 ? __ldg(A.child + 8 * P + o) : -1;
    cs[b][u] = cb >= 0 ? __ldg(A.cmap_c + (size_t)cb * A.ncomp_c + __ldg(A.up_cc + g * kQ + q0)) : -1;
  }
  __syncthreads();
  // keep the units in which some box of the item has a child (in place, order kept: one warp
  // reads a group of 32 units, then writes them to positions at or below the group's start)
  if (warp == 0) {
    int nact = 0;
    for (int g0 = 0; g0 < nunits; g0 += 32) {
      const int u = g0 + lane;
      int tk = 0, c[kTcBoxes];
      bool any = false;
      if (u < nunits) {
        tk = units[u];
#pragma unroll
        for (int b = 0; b < kTcBoxes; ++b) {
          c[b] = cs[b][u];
          any = any || c[b] >= 0;
        }
      }
      const unsigned msk = __ballot_sync(0xffffffffu, any);
      __syncwarp();
      if (any) {
        const int pos = nact + __popc(msk & ((1u << lane) - 1u));
        units[pos] = tk;
#pragma unroll
        for (int b = 0; b < kTcBoxes; ++b) cs[b][pos] = c[b];
      }
      nact += __popc(msk);
      __syncwarp();
    }
    if (lane == 0) nact_s = nact;
  }
  __syncthreads();
  nunits = nact_s;
  auto issue_a = [&](int u) {   // thread 0: the operand images of unit u's child cones
    uint32_t bytes = 0;
#pragma unroll
    for (int b = 0; b < kTcBoxes; ++b) bytes += cs[b][u] >= 0 ? 2u * tc::kImgBytes : 0u;
    tc::expect_tx(&bar_a, bytes);
#pragma unroll
    for (int b = 0; b < kTcBoxes; ++b) {
      if (cs[b][u] < 0) continue;
      const float* src = imgc + (size_t)cs[b][u] * kImgFloats;
      tc::bulk_g2s(sm + b * tc::kImgBytes, src, tc::kImgBytes, &bar_a);
      tc::bulk_g2s(sm + tc::kOffAlo + b * tc::kImgBytes, src + kImgFloats / 2, tc::kImgBytes, &bar_a);
    }
  };
  if (t == 0 && nunits > 0) issue_a(0);
  const T off = (T)(0.5 * A.Hc);
  const T kk[2] = {A.ke, A.ki};
  const T sgn = (lane & 1) ? T(1) : T(-1);
  const int ks = lane >> 4;
  const uint32_t id = tc::idesc(128, tc::kN);
  uint32_t ph = 0;
  bool ok = true, a_pending = nunits > 0, m_pending = false;
  for (int u = 0; u < nunits; ++u) {
    const int tk = units[u], r0 = tk & 255, len = (tk >> 8) & 255, o = (tk >> 16) & 7;
    const size_t g = (size_t)ci * 8 + o;
    // the unit's points: Chebyshev values in the child cone and re-centring factors (warp 0)
    if (warp == 0 && lane < len) {
      const int q = __ldg(TT.order + g * kQ + r0 + lane);
      const int ccx = __ldg(A.up_cc + g * kQ + q);
      const T ox = (o & 1) ? off : -off, oy = (o & 2) ? off : -off, oz = (o & 4) ? off : -off;
      const T x = Xp[q][0] - ox, y = Xp[q][1] - oy, z = Xp[q][2] - oz;
      T ts, tt, tp, rc, sth, cth, sph, cph;
      local_coords(A.cgc, A.ckeys_c[ccx], x, y, z, &ts, &tt, &tp, &rc, &sth, &cth, &sph, &cph);
      T v5[5], w5[5], v3[3];
      cheb_vals<T, 3>(ts, v3);
      cheb_vals<T, 5>(tt, v5);
      cheb_vals<T, 5>(tp, w5);
      pts[3 * lane] = make_float4(v3[1], v3[2], v5[1], v5[2]);
      pts[3 * lane + 1] = make_float4(v5[3], v5[4], w5[1], w5[2]);
      pts[3 * lane + 2] = make_float4(w5[3], w5[4], __int_as_float(q), 0.f);
      const T rp = Xp[q][3];
      const T dr = (T(3) * off * off - T(2) * (Xp[q][0] * ox + Xp[q][1] * oy + Xp[q][2] * oz)) / (rc + rp);
      T sn0, cs0, sn1, cs1;
      sincos_t(kk[0] * dr, &sn0, &cs0);
      sincos_t(kk[1] * dr, &sn1, &cs1);
      const T a = rp / rc;
      fac[lane] = make_float4(a * cs0, a * sn0, a * cs1, a * sn1);
    }
    __syncthreads();
    // basis B(u): (point n, chunk kc) tasks, hi and lo parts (rows n >= len are not read back)
    for (int e = t; e < len * 20; e += blockDim.x) {
      const int n = e / 20, kc = e - n * 20;
      const float4 p0 = pts[3 * n], p1 = pts[3 * n + 1], p2 = pts[3 * n + 2];
      const T TS[3] = {T(1), p0.x, p0.y};
      const T TV[5] = {T(1), p0.z, p0.w, p1.x, p1.y};
      const T TP[5] = {T(1), p1.z, p1.w, p2.x, p2.y};
      T v[4], h[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int k = 4 * kc + j;
        v[j] = k < kQ ? TS[k / 25] * TV[(k / 5) % 5] * TP[k % 5] : T(0);
        h[j] = tf32_hi(v[j]);
      }
      const int bo = tc::kmaj_off(n, kc);
      *reinterpret_cast<float4*>(sm + tc::kOffB + bo) = make_float4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<float4*>(sm + tc::kOffBlo + bo) = make_float4(v[0] - h[0], v[1] - h[1], v[2] - h[2], v[3] - h[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // B visible to the tensor cores
    ok = __syncthreads_and(tc::wait(&bar_a, ph, TT.wait_ns)) != 0;   // A(u) landed
    if (!ok) break;
    a_pending = false;
    tc::fence_after();
    if (t == 0 && !(TT.inject && u == 0)) {
      const uint32_t aH = tc::smem_u32(sm), aL = tc::smem_u32(sm + tc::kOffAlo);
      const uint32_t bH = tc::smem_u32(sm + tc::kOffB), bL = tc::smem_u32(sm + tc::kOffBlo);
#pragma unroll 1
      for (int pass = 0; pass < 3; ++pass) {
        const uint32_t ab = pass == 2 ? aL : aH, bb = pass == 1 ? bL : bH;
#pragma unroll
        for (int k8 = 0; k8 < tc::kK / 8; ++k8)
          tc::mma(tm + tc::kColD, tc::sdesc(ab + k8 * 256, 128, 2560, 0), tc::sdesc(bb + k8 * 256, 128, 2560, 0), id,
                  (pass | k8) ? 1u : 0u);
      }
      tc::commit(&bar_m);
    }
    m_pending = true;
    ok = __syncthreads_and(tc::wait(&bar_m, ph, TT.wait_ns)) != 0;   // MMA(u) done: D ready, A free
    if (!ok) break;
    m_pending = false;
    tc::fence_after();
    ph ^= 1u;
    if (t == 0 && u + 1 < nunits) issue_a(u + 1);
    a_pending = u + 1 < nunits;
    // epilogue: warp w re-centres box w's columns of D and adds them into the parent columns
    if (slot[warp] >= 0 && cs[warp][u] >= 0) {
      float r[32], pv[32];
      tc::ld_x32(tlane + tc::kColD, r);
      int qn[32];
#pragma unroll
      for (int n = 0; n < 32; ++n) {
        pv[n] = 0.f;
        if (n < len) {
          qn[n] = __float_as_int(pts[3 * n + 2].z);
          tc::ld_x1(tlane + (uint32_t)qn[n], pv[n]);
        }
      }
      tc::wait_ld_regs(pv);
#pragma unroll
      for (int n = 0; n < 32; ++n) {
        if (n < len) {
          const T wv = __shfl_xor_sync(0xffffffffu, r[n], 1);
          const float4 F = fac[n];
          const T fr = ks ? F.z : F.x, fi = ks ? F.w : F.y;
          tc::st_x1(tlane + (uint32_t)qn[n], pv[n] + fmaf(r[n], fr, sgn * fi * wv));
        }
      }
      tc::wait_st();
    }
    tc::fence_before();
    __syncthreads();
  }
  if (!ok) {
    // a wait timed out: record it, let the copies and MMAs in flight finish (bounded), release
    if (t == 0) atomicOr(TT.err, 1);
    if (a_pending) tc::wait(&bar_a, ph, TT.wait_ns);
    if (m_pending) tc::wait(&bar_m, ph, TT.wait_ns);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (ok && slot[warp] >= 0) {
    // this thread's column (box warp, field lane) of 75 parent values -> coefficients
    float v[80];
#pragma unroll
    for (int c = 0; c < 80; c += 16) tc::ld_x16(tlane + c, v + c);
    float t5[5];
#pragma unroll
    for (int a = 0; a < 15; ++a) {   // phi
#pragma unroll
      for (int k = 0; k < 5; ++k) t5[k] = v[a * 5 + k];
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        float acc = 0.f;
#pragma unroll
        for (int kk2 = 0; kk2 < 5; ++kk2) acc += M.A5[k * 5 + kk2] * t5[kk2];
        v[a * 5 + k] = acc;
      }
    }
#pragma unroll
    for (int is = 0; is < 3; ++is)   // theta
#pragma unroll
      for (int k = 0; k < 5; ++k) {
#pragma unroll
        for (int j = 0; j < 5; ++j) t5[j] = v[(is * 5 + j) * 5 + k];
#pragma unroll
        for (int j = 0; j < 5; ++j) {
          float acc = 0.f;
#pragma unroll
          for (int jj = 0; jj < 5; ++jj) acc += M.A5[j * 5 + jj] * t5[jj];
          v[(is * 5 + j) * 5 + k] = acc;
        }
      }
#pragma unroll
    for (int jk = 0; jk < 25; ++jk) {   // s
#pragma unroll
      for (int i = 0; i < 3; ++i) t5[i] = v[i * 25 + jk];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        float acc = 0.f;
#pragma unroll
        for (int ii = 0; ii < 3; ++ii) acc += M.A3[i * 3 + ii] * t5[ii];
        v[i * 25 + jk] = acc;
      }
    }
    T* out = A.coefs_p + (size_t)slot[warp] * kQ * 32 + lane;
#pragma unroll
    for (int k = 0; k < kQ; ++k) out[k * 32] = v[k];
    if (imgp) {   // operand images for the next upward step on the tensor cores
      float* im = imgp + (size_t)slot[warp] * kImgFloats;
#pragma unroll
      for (int kc = 0; kc < 20; ++kc) {
        float x[4], h[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          x[j] = 4 * kc + j < kQ ? v[4 * kc + j] : 0.f;
          h[j] = tf32_hi(x[j]);
        }
        *reinterpret_cast<float4*>(im + img_off(lane, kc)) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4*>(im + kImgFloats / 2 + img_off(lane, kc)) =
            make_float4(x[0] - h[0], x[1] - h[1], x[2] - h[2], x[3] - h[3]);
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(tc::kCols) : "memory");
}

// ------------------------------------------------------------------ (c) target evaluation
// T: arithmetic and coefficient type; TO: the fields' storage (FP64 in the mixed-precision plan)
// (c), warp per target: the target's pairs in groups of 32, scalars one per lane.
template <typename T, typename TO>
__global__ void __launch_bounds__(32 * tgt_warps<T>(), 2) k_target(TgtArgs<T, TO> A) {
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
  TgtScal<T>* S = sc[warp];
  T accS = 0, accD = 0;
  for (int64_t c0 = e0; c0 < e1; c0 += 32) {
    const int nc = (int)min((int64_t)32, e1 - c0);
    if (lane < nc) tgt_scalars(A, x0, x1, x2, n0, n1, n2, A.tgt_slot[c0 + lane], S[lane]);
    __syncwarp();
    for (int cI = 0; cI < nc; ++cI) {
      const TgtScal<T>& Q = S[cI];
      const T* C = A.coefs + (size_t)Q.slot * kQ * 32 + lane;
      // all 75 coefficient loads are issued before the arithmetic: one round trip per pair
      T cc[kQ];
#pragma unroll
      for (int k = 0; k < kQ; ++k) cc[k] = __ldg(C + k * 32);
      T oS, oD;
      tgt_contract(Q, cc, lane >> 4, (lane & 1) != 0, oS, oD);
      accS += oS;
      accD += oD;
    }
    __syncwarp();
  }
  TO* out = A.f28 + 56 * (size_t)A.perm[t];
  out[lane] += (TO)accS;
  const int dens = (lane >> 1) & 7;
  if (dens < 6) out[2 * (16 + 6 * ks + dens) + (lane & 1)] += (TO)accD;
}

// (c), FP32: warp per chunk of at most 32 targets of one box.  The targets of a box share their
// cousin boxes, and neighbouring targets mostly fall in the same cone segment of a cousin.  The
// chunk's (target, cousin) pairs are taken 32 at a time, cousin-major (one pair per lane for the
// scalars); the lanes whose pairs share a cone segment form a group that loads the segment's
// coefficients once.  Per-target fields accumulate in shared memory.
constexpr int kTgtBoxWarps = 4;
constexpr size_t kTgtBoxSmem = (size_t)kTgtBoxWarps * 32 * (sizeof(TgtScal<float>) + 56 * sizeof(float));

template <typename TO>
__global__ void __launch_bounds__(32 * kTgtBoxWarps) k_target_box(TgtArgs<float, TO> A, const int2* __restrict__ chunks,
                                                                  int nchunks) {
  using T = float;
  extern __shared__ float4 tb_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  TgtScal<T>* S = reinterpret_cast<TgtScal<T>*>(tb_smem) + warp * 32;
  T* acc = reinterpret_cast<T*>(reinterpret_cast<TgtScal<T>*>(tb_smem) + kTgtBoxWarps * 32) + warp * 32 * 56;
  const int chunk = blockIdx.x * kTgtBoxWarps + warp;
  if (chunk >= nchunks) return;   // no block-wide synchronisation below
  A.coefs += blockIdx.y * A.cstride;   // right-hand side of a batched call
  A.f28 += blockIdx.y * 56 * (size_t)A.N;
  const int2 ch = chunks[chunk];
  const int t0 = ch.x, n = ch.y;
  const int64_t base0 = A.tgt_ptr[t0];
  const int ncous = (int)(A.tgt_ptr[t0 + 1] - base0);   // every target of the box has one record per cousin
  for (int e = lane; e < 32 * 56; e += 32) acc[e] = T(0);
  const int dens = (lane >> 1) & 7, ks = lane >> 4;
  const int dcol = 2 * (16 + 6 * ks + dens) + (lane & 1);
  const int npairs = n * ncous;
  for (int p0 = 0; p0 < npairs; p0 += 32) {
    const int pp = p0 + lane;
    const bool act = pp < npairs;
    const int j = act ? pp / n : 0, i = act ? pp - j * n : 0;   // cousin j, target t0 + i
    int myslot = -1;
    if (act) {
      const int t = t0 + i;
      myslot = A.tgt_slot[base0 + (int64_t)i * ncous + j];
      tgt_scalars(A, A.x_sorted[3 * (size_t)t], A.x_sorted[3 * (size_t)t + 1], A.x_sorted[3 * (size_t)t + 2],
                  (T)A.n_sorted[3 * (size_t)t], (T)A.n_sorted[3 * (size_t)t + 1], (T)A.n_sorted[3 * (size_t)t + 2],
                  myslot, S[lane]);
    }
    const int mytgt = i;
    __syncwarp();
    unsigned rem = __ballot_sync(0xffffffffu, act);
    while (rem) {
      const int leader = __ffs(rem) - 1;
      const int s0 = __shfl_sync(0xffffffffu, myslot, leader);
      unsigned grp = __ballot_sync(0xffffffffu, myslot == s0) & rem;
      rem &= ~grp;
      const T* C = A.coefs + (size_t)s0 * kQ * 32 + lane;
      T cc[kQ];
#pragma unroll
      for (int k = 0; k < kQ; ++k) cc[k] = __ldg(C + k * 32);
      while (grp) {
        const int m = __ffs(grp) - 1;
        grp &= grp - 1;
        const int ti = __shfl_sync(0xffffffffu, mytgt, m);
        T oS, oD;
        tgt_contract(S[m], cc, lane >> 4, (lane & 1) != 0, oS, oD);
        acc[ti * 56 + lane] += oS;
        if (dens < 6) acc[ti * 56 + dcol] += oD;
      }
    }
    __syncwarp();
  }
  for (int i = 0; i < n; ++i) {
    TO* out = A.f28 + 56 * (size_t)A.perm[t0 + i];
    out[lane] += (TO)acc[i * 56 + lane];
    if (lane < 24) out[32 + lane] += (TO)acc[i * 56 + 32 + lane];
  }
}

// The FP32 SIMT upward step into the level below Pp: mode 0 runs per point group (a block per
// parent slot), 1 a warp per parent slot (unit tables), 2 runs per point group with a block per
// item of up to kTcBoxes slots of one parent cone (one prologue for the item).
void launch_up_simt(const UpArgs<float>& U, const DevLevel& Pp, int mode, int nrhs, cudaStream_t s) {
  if (mode == 1 && Pp.tc_unit_ptr)
    k_up_warp<<<dim3((unsigned)((Pp.nslots + kUpWarpW - 1) / kUpWarpW), nrhs), 32 * kUpWarpW, kUpWarpSmem, s>>>(
        U, UnitTabs{Pp.tc_order, Pp.tc_unit, Pp.tc_unit_ptr}, Pp.nslots);
  else if (mode == 2 && Pp.tc_item)
    k_up_runs<<<dim3((unsigned)Pp.ntc_items, 1), 32 * kUpRunWarps, kUpRunSmem, s>>>(
        U, RunTabs{Pp.up_order, Pp.up_task, Pp.up_task_ptr}, nrhs, Pp.tc_item);
  else
    k_up_runs<<<dim3(Pp.nslots, 1), 32 * kUpRunWarps, kUpRunSmem, s>>>(
        U, RunTabs{Pp.up_order, Pp.up_task, Pp.up_task_ptr}, nrhs, nullptr);
}

template <typename T, typename TO = T>
cudaError_t run_ifgf(ifgf_plan_t* p, cudaStream_t s, int nrhs) {
  const int D = p->tree.D;
  const T ke = (T)p->desc.k_ext, ki = (T)p->desc.k_int;
  {
    const DevLevel& L = p->dl[D];
    LeafArgs<T> A{L.box_pt_ptr, L.box_slot_ptr, L.slot_cone, L.box_center, cone_geom_t<T>(L.cg),
                  p->x_sorted, (const T*)p->a_sorted, (T*)L.coefs, ke, ki, 16 * (size_t)p->N, L.cstride,
                  L.img, L.istride};
    int rec = timer_begin(p, TK_LEAF, s);
    if (L.nboxes > 0 && L.max_box_slots > 0) {
      const dim3 grid((unsigned)L.nboxes, (unsigned)((L.max_box_slots + kLeafSlots - 1) / kLeafSlots),
                      (unsigned)nrhs);
      if constexpr (std::is_same<T, float>::value) {
        if (L.leaf_mode == 1)
          k_leaf_mma<<<grid, 32 * kLeafMmaWarps, 0, s>>>(A);
        else
          k_leaf<T><<<grid, kLeafThreads, 0, s>>>(A);
      } else {
        k_leaf<T><<<grid, kLeafThreads, 0, s>>>(A);
      }
    }
    timer_end(p, rec, s);
    ++p->launches;
  }
  for (int d = D; d >= 3; --d) {
    const DevLevel& L = p->dl[d];
    TgtArgs<T, TO> B{p->N, L.tgt_ptr, L.tgt_slot, L.slot_box, L.slot_cone, L.box_center, cone_geom_t<T>(L.cg),
                     (const T*)L.coefs, p->x_sorted, p->n_sorted, p->perm, (TO*)p->f28, ke, ki, L.cstride,
                     L.cg.h, 1.0 / L.cg.ds(), p->desc.k_ext, p->desc.k_int, L.trig_th, L.trig_ph};
    int rec = timer_begin(p, TK_TARGET, s);
    if constexpr (std::is_same<T, float>::value) {
      // a warp per box chunk or a warp per target: the level's tgt_mode (set at plan creation,
      // retuned by ifgf_plan_tune)
      if (L.tgt_mode == 1 && L.ntgt_chunks > 0)
        k_target_box<TO><<<dim3((unsigned)((L.ntgt_chunks + kTgtBoxWarps - 1) / kTgtBoxWarps), nrhs),
                           32 * kTgtBoxWarps, kTgtBoxSmem, s>>>(B, L.tgt_chunk, L.ntgt_chunks);
      else
        k_target<T, TO><<<dim3((unsigned)((p->N + tgt_warps<T>() - 1) / tgt_warps<T>()), nrhs), 32 * tgt_warps<T>(),
                          0, s>>>(B);
    } else {
      k_target<T, TO><<<dim3((unsigned)((p->N + tgt_warps<T>() - 1) / tgt_warps<T>()), nrhs), 32 * tgt_warps<T>(), 0,
                    s>>>(B);
    }
    timer_end(p, rec, s);
    ++p->launches;
    if (d > 3) {
      const DevLevel& Pp = p->dl[d - 1];
      UpArgs<T> U{Pp.slot_box, Pp.slot_cone, Pp.slot_upidx, Pp.child, cone_geom_t<T>(Pp.cg),
                  L.cmap, L.ncomp, L.ckeys, cone_geom_t<T>(L.cg), L.H, Pp.up_cc, (const T*)L.coefs, (T*)Pp.coefs, ke, ki,
                  L.cstride, Pp.cstride, Pp.img, Pp.istride};
      rec = timer_begin(p, TK_UP, s);
      if (Pp.nslots > 0) {
        if constexpr (std::is_same<T, float>::value) {
          if (Pp.tc)
            k_up_tc<<<dim3(Pp.ntc_items, nrhs), tc::kThreads, tc::kSmem, s>>>(
                U, TcTabs{Pp.tc_order, Pp.tc_unit, Pp.tc_unit_ptr, Pp.tc_item, L.img, L.istride, p->dev_err,
                          p->inject ? 1000000ull : 1000000000ull, p->inject});
          else
            launch_up_simt(U, Pp, Pp.up_mode, nrhs, s);
        } else
          k_up<T><<<dim3(Pp.nslots, nrhs), kUpThreads, 0, s>>>(U);
      }
      timer_end(p, rec, s);
      ++p->launches;
    }
  }
  return cudaGetLastError();
}

}  // namespace

// The FP32 target step of level d alone in `mode` (0 warp per target, 1 warp per box chunk), for
// the autotuner; accumulates into the plan's fields buffer like an apply.
cudaError_t launch_target_level(ifgf_plan_t* p, int d, int mode, cudaStream_t s) {
  if (ifgf64(p->desc)) return cudaErrorInvalidValue;
  const DevLevel& L = p->dl[d];
  TgtArgs<float, float> B32{p->N, L.tgt_ptr, L.tgt_slot, L.slot_box, L.slot_cone, L.box_center,
                            cone_geom_t<float>(L.cg), (const float*)L.coefs, p->x_sorted, p->n_sorted, p->perm,
                            (float*)p->f28, (float)p->desc.k_ext, (float)p->desc.k_int, L.cstride, L.cg.h,
                            1.0 / L.cg.ds(), p->desc.k_ext, p->desc.k_int, L.trig_th, L.trig_ph};
  TgtArgs<float, double> B64{p->N, L.tgt_ptr, L.tgt_slot, L.slot_box, L.slot_cone, L.box_center,
                             cone_geom_t<float>(L.cg), (const float*)L.coefs, p->x_sorted, p->n_sorted, p->perm,
                             (double*)p->f28, (float)p->desc.k_ext, (float)p->desc.k_int, L.cstride, L.cg.h,
                             1.0 / L.cg.ds(), p->desc.k_ext, p->desc.k_int, L.trig_th, L.trig_ph};
  const bool out64 = store64(p->desc);
  if (mode == 1 && L.ntgt_chunks > 0) {
    const dim3 g((unsigned)((L.ntgt_chunks + kTgtBoxWarps - 1) / kTgtBoxWarps), 1);
    if (out64)
      k_target_box<double><<<g, 32 * kTgtBoxWarps, kTgtBoxSmem, s>>>(B64, L.tgt_chunk, L.ntgt_chunks);
    else
      k_target_box<float><<<g, 32 * kTgtBoxWarps, kTgtBoxSmem, s>>>(B32, L.tgt_chunk, L.ntgt_chunks);
  } else {
    const dim3 g((unsigned)((p->N + tgt_warps<float>() - 1) / tgt_warps<float>()), 1);
    if (out64)
      k_target<float, double><<<g, 32 * tgt_warps<float>(), 0, s>>>(B64);
    else
      k_target<float, float><<<g, 32 * tgt_warps<float>(), 0, s>>>(B32);
  }
  return cudaGetLastError();
}

// The FP32 SIMT upward step from level d + 1 into level d alone in `mode` (0 runs per point
// group, 1 a warp per parent slot), for the autotuner; writes level d's coefficients like an apply.
cudaError_t launch_up_level(ifgf_plan_t* p, int d, int mode, cudaStream_t s) {
  if (ifgf64(p->desc) || d < 3 || d >= p->tree.D) return cudaErrorInvalidValue;
  const DevLevel& L = p->dl[d + 1];
  const DevLevel& Pp = p->dl[d];
  if (Pp.nslots == 0) return cudaSuccess;
  UpArgs<float> U{Pp.slot_box, Pp.slot_cone, Pp.slot_upidx, Pp.child, cone_geom_t<float>(Pp.cg),
                  L.cmap, L.ncomp, L.ckeys, cone_geom_t<float>(L.cg), L.H, Pp.up_cc, (const float*)L.coefs,
                  (float*)Pp.coefs, (float)p->desc.k_ext, (float)p->desc.k_int, L.cstride, Pp.cstride,
                  Pp.img, Pp.istride};
  launch_up_simt(U, Pp, mode, 1, s);
  return cudaGetLastError();
}

// The FP32 leaf step alone in `mode` (0 SIMT, 1 tensor-pipe products), for the autotuner; writes
// the leaf level's coefficients like an apply.
cudaError_t launch_leaf_level(ifgf_plan_t* p, int mode, cudaStream_t s) {
  if (ifgf64(p->desc)) return cudaErrorInvalidValue;
  const DevLevel& L = p->dl[p->tree.D];
  if (L.nboxes == 0 || L.max_box_slots == 0) return cudaSuccess;
  LeafArgs<float> A{L.box_pt_ptr, L.box_slot_ptr, L.slot_cone, L.box_center, cone_geom_t<float>(L.cg),
                    p->x_sorted, (const float*)p->a_sorted, (float*)L.coefs, (float)p->desc.k_ext,
                    (float)p->desc.k_int, 16 * (size_t)p->N, L.cstride, L.img, L.istride};
  const dim3 grid((unsigned)L.nboxes, (unsigned)((L.max_box_slots + kLeafSlots - 1) / kLeafSlots), 1);
  if (mode == 1)
    k_leaf_mma<<<grid, 32 * kLeafMmaWarps, 0, s>>>(A);
  else
    k_leaf<float><<<grid, kLeafThreads, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t setup_ifgf_kernels() {
  cudaError_t e = cudaFuncSetAttribute(k_up_runs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUpRunSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_up_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_target_box<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTgtBoxSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_target_box<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTgtBoxSmem);
  return e;
}

cudaError_t launch_far_ifgf(ifgf_plan_t* p, cudaStream_t s, int nrhs) {
  if (narrow_passes(p->desc)) return launch_far_ifgf_pass(p, s, nrhs);
  if (ifgf64(p->desc)) return run_ifgf<double>(p, s, nrhs);
  if (store64(p->desc)) return run_ifgf<float, double>(p, s, nrhs);
  return run_ifgf<float>(p, s, nrhs);
}

}  // namespace ifgf
