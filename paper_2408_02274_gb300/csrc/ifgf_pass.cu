// IFGF far-field kernels with fewer fields per octree traversal (Sec. III, "IFGF for Multiple
// Densities: Speed-vs-Memory Trade-off", and the Remark "On selection of IFGF approach").  The
// sums of Eq. ifgf_sum_em, I_{k,n} for 8 densities k and 2 kernels n, are taken in groups of
// F = fields_per_pass fields (one kernel n, densities d0 .. d0 + F - 1), one full traversal
// (leaf step, then per level target and upward steps) per group:
//   F = 8: one kernel per traversal, 2 traversals, coefficient rows of 16 reals (half the
//          interpolation memory of IFGF_Vec);
//   F = 1: IFGF_Seq, 16 traversals, rows of 2 reals (1/16 of the memory).
// Each traversal repeats the work that IFGF_Vec shares among all 16 fields: the source distances
// and kernel values at the leaves, the cone coordinates and re-centring factors of the upward
// step, and the target coordinates and centred factors.  The upward step runs by the host's runs
// (register-resident child coefficients) for F = 8 and by (point, column) tasks for F = 1.  Coefficients are stored per cone
// segment as [75][NC] reals, NC = 2F (Chebyshev index, then the group's fields, re/im interleaved).
// FP32 arithmetic (the FP32 and mixed plans), the same formulas as the all-fields kernels.
#include "ifgf_dev.cuh"

namespace ifgf {

namespace {

// (a): F^D at the 75 points of two cone segments per pass, a thread per point, for the group's
// NC / 2 densities and the one kernel ks; the staged densities are the group's columns only.
template <int NC>
__global__ void __launch_bounds__(kLeafThreads) k_leaf_pass(LeafArgs<float> A, int ks, int d0) {
  using T = float;
  constexpr int kS = NC + 1;   // padded row stride of the value buffer
  __shared__ SmallMaps<T> M;
  __shared__ T src[kLeafChunk][4];
  __shared__ T sa[kLeafChunk][NC];
  __shared__ T vbuf[2 * kQ * kS];
  const int box = blockIdx.x;
  const int t = threadIdx.x;
  const int sb = A.box_slot_ptr[box] + blockIdx.y * kLeafSlots;
  const int se = min(A.box_slot_ptr[box + 1], sb + kLeafSlots);
  if (sb >= se) return;   // uniform per block
  init_maps(M);
  const double c0 = A.box_center[3 * box], c1 = A.box_center[3 * box + 1], c2 = A.box_center[3 * box + 2];
  const int pb = A.box_pt_ptr[box], pe = A.box_pt_ptr[box + 1];
  const int nsrc = pe - pb;
  const T kap = ks ? A.ki : A.ke;
  auto stage = [&](int cb, int nchunk) {
    for (int e = t; e < nchunk; e += blockDim.x) {
      const int m = pb + cb + e;
      const T y0 = (T)(A.x_sorted[3 * (size_t)m] - c0);
      const T y1 = (T)(A.x_sorted[3 * (size_t)m + 1] - c1);
      const T y2 = (T)(A.x_sorted[3 * (size_t)m + 2] - c2);
      src[e][0] = y0; src[e][1] = y1; src[e][2] = y2;
      src[e][3] = y0 * y0 + y1 * y1 + y2 * y2;
#pragma unroll
      for (int k = 0; k < NC; ++k) sa[e][k] = A.a_sorted[16 * (size_t)m + 2 * d0 + k];
    }
  };
  const bool staged_once = nsrc <= kLeafChunk;
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
    T acc[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) acc[k] = 0;
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
          const T dxy = src[e][3] - T(2) * (X[0] * src[e][0] + X[1] * src[e][1] + X[2] * src[e][2]);
          const T d = sqrt_t(r * r + dxy);
          const T rd = leaf_div(r, d);
          const T dd = leaf_div(dxy, d + r);
          T sn, cs;
          leaf_sincos(kap * dd, &sn, &cs);
          const T gr = rd * cs, gi = rd * sn;
#pragma unroll
          for (int k = 0; k < NC / 2; ++k) {
            const T ar = sa[e][2 * k], ai = sa[e][2 * k + 1];
            acc[2 * k] += ar * gr - ai * gi;
            acc[2 * k + 1] += ar * gi + ai * gr;
          }
        }
      }
    }
    if (act)
#pragma unroll
      for (int k = 0; k < NC; ++k) vbuf[(sl * kQ + q) * kS + k] = acc[k];
    __syncthreads();
    vals_to_coefs_block<T, kS, NC>(M, vbuf, A.coefs + (size_t)s0 * kQ * NC, min(2, se - s0));
  }
}

// (b): a block per parent slot.  Per child octant the 75 parent points' child cone, Chebyshev
// values and re-centring factor (kernel ks) go to shared memory; then every (point, column) task
// contracts its child cone's 75 coefficients of that column (separably: phi, theta, s) and the
// lane pairs (re, im) of a point multiply by the factor.  Tasks of one octant are distinct, so the
// values accumulate with plain shared-memory adds.
template <int NC>
__global__ void __launch_bounds__(kUpThreads) k_up_pass(UpArgs<float> A, int ks) {
  using T = float;
  constexpr int kS = NC + 1;
  constexpr int kTasks = kQ * NC;   // even: the lanes of a (re, im) pair are both in range or both out
  __shared__ SmallMaps<T> M;
  __shared__ T Xp[kQ][3];
  __shared__ int cslot[kQ];
  __shared__ T pt[kQ][16];   // T_0..2(ts), T_0..4(tt), T_0..4(tp), Re f, Im f
  __shared__ T vals[kQ * kS];
  const int pslot = blockIdx.x;
  const int t = threadIdx.x;
  init_maps(M);
  const int P = A.slot_box[pslot], ci = A.slot_upidx[pslot];
  const cone_key pcone = A.slot_cone[pslot];
  __syncthreads();
  if (t < kQ) cone_point(M, A.cgp, pcone, t, Xp[t]);
  for (int e = t; e < kQ * kS; e += blockDim.x) vals[e] = 0;
  const T off = (T)(0.5 * A.Hc);
  const T kap = ks ? A.ki : A.ke;
  for (int o = 0; o < 8; ++o) {
    const int cb = A.child[8 * P + o];
    if (cb < 0) continue;   // uniform per block
    __syncthreads();
    if (t < kQ) {
      const T ox = (o & 1) ? off : -off, oy = (o & 2) ? off : -off, oz = (o & 4) ? off : -off;
      const T x = Xp[t][0] - ox, y = Xp[t][1] - oy, z = Xp[t][2] - oz;
      const int ccx = A.up_cc[((size_t)ci * 8 + o) * kQ + t];
      const cone_key cc = A.ckeys_c[ccx];
      cslot[t] = A.cmap_c[(size_t)cb * A.ncomp_c + ccx];
      T ts, tt, tp, rc, sth, cth, sph, cph;
      local_coords(A.cgc, cc, x, y, z, &ts, &tt, &tp, &rc, &sth, &cth, &sph, &cph);
      cheb_vals<T, 3>(ts, &pt[t][0]);
      cheb_vals<T, 5>(tt, &pt[t][3]);
      cheb_vals<T, 5>(tp, &pt[t][8]);
      // re-centring factor G(x, x_child)/G(x, x_parent) = (r_p/r_c) e^{i k (r_c - r_p)}
      const T rp = sqrt_t(Xp[t][0] * Xp[t][0] + Xp[t][1] * Xp[t][1] + Xp[t][2] * Xp[t][2]);
      const T dr = (T(3) * off * off - T(2) * (Xp[t][0] * ox + Xp[t][1] * oy + Xp[t][2] * oz)) / (rc + rp);
      T sn, cs;
      sincos_t(kap * dr, &sn, &cs);
      pt[t][13] = rp / rc * cs;
      pt[t][14] = rp / rc * sn;
    }
    __syncthreads();
    for (int base = 0; base < kTasks; base += kUpThreads) {
      const int e = base + t;
      const bool on = e < kTasks;
      const int q = on ? e / NC : 0, c = e % NC;
      const int cs = on ? cslot[q] : -1;
      T v = 0;
      if (cs >= 0) {   // cs < 0 cannot happen: the host marked every such cone relevant
        const T* C = A.coefs_c + (size_t)cs * kQ * NC + c;
        const T* Q = pt[q];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          T ei = 0;
#pragma unroll
          for (int j = 0; j < 5; ++j) {
            T dj = 0;
#pragma unroll
            for (int k = 0; k < 5; ++k) dj += Q[8 + k] * __ldg(C + ((i * 5 + j) * 5 + k) * NC);
            ei += Q[3 + j] * dj;
          }
          v += Q[i] * ei;
        }
      }
      const T w = __shfl_xor_sync(0xffffffffu, v, 1);
      if (cs >= 0) {
        const bool odd = c & 1;
        const T re = odd ? w : v, im = odd ? v : w;
        const T fr = pt[q][13], fi = pt[q][14];
        vals[q * kS + c] += odd ? (re * fi + im * fr) : (re * fr - im * fi);
      }
    }
  }
  __syncthreads();
  vals_to_coefs_block<T, kS, NC>(M, vals, A.coefs_p + (size_t)pslot * kQ * NC, 1);
}

// (b) by runs: the host's run tables (per parent cone, the points of one octant in one child
// cone, at most 32, in four fixed point groups, one per warp) let a warp load its child cone's
// coefficients once per run into registers, 75 per lane, lane = column (NC lanes per point, the
// 32 / NC lane groups holding the same column set), and sweep the run's points 32 / NC at a time.
// The prologue puts each (octant, parent point)'s child slot, Chebyshev values and re-centring
// factor (kernel ks) in shared memory.  A warp adds only into its own group's points.
template <int NC>
__global__ void __launch_bounds__(32 * kUpGroups, 4) k_up_pass_runs(UpArgs<float> A, const int* __restrict__ order,
                                                                     const int* __restrict__ task,
                                                                     const int* __restrict__ task_ptr, int ks) {
  using T = float;
  constexpr int kS = NC + 1;
  constexpr int kP = 32 / NC;   // points per warp step
  __shared__ SmallMaps<T> M;
  __shared__ T Xp[kQ][3];
  __shared__ int cslot[8][kQ];
  __shared__ __align__(16) T pt[8][kQ][16];   // T_0..2(ts), T_0..4(tt), T_0..4(tp), Re f, Im f
  __shared__ T vals[kQ * kS];
  const int pslot = blockIdx.x;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  init_maps(M);
  const int P = A.slot_box[pslot], ci = A.slot_upidx[pslot];
  const cone_key pcone = A.slot_cone[pslot];
  __syncthreads();
  if (t < kQ) cone_point(M, A.cgp, pcone, t, Xp[t]);
  for (int e = t; e < kQ * kS; e += blockDim.x) vals[e] = 0;
  __syncthreads();
  const T off = (T)(0.5 * A.Hc);
  const T kap = ks ? A.ki : A.ke;
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
    T* Q = pt[o][q];
    cheb_vals<T, 3>(ts, Q);
    cheb_vals<T, 5>(tt, Q + 3);
    cheb_vals<T, 5>(tp, Q + 8);
    // re-centring factor G(x, x_child)/G(x, x_parent) = (r_p/r_c) e^{i k (r_c - r_p)}
    const T rp = sqrt_t(Xp[q][0] * Xp[q][0] + Xp[q][1] * Xp[q][1] + Xp[q][2] * Xp[q][2]);
    const T dr = (T(3) * off * off - T(2) * (Xp[q][0] * ox + Xp[q][1] * oy + Xp[q][2] * oz)) / (rc + rp);
    T sn, cs;
    sincos_t(kap * dr, &sn, &cs);
    Q[13] = rp / rc * cs;
    Q[14] = rp / rc * sn;
  }
  __syncthreads();
  const int col = lane % NC, sub = lane / NC;
  const bool odd = col & 1;
  const int w0 = task_ptr[(size_t)ci * kUpGroups + warp], w1 = task_ptr[(size_t)ci * kUpGroups + warp + 1];
  for (int w = w0; w < w1; ++w) {
    const int tk = task[w];
    const int r0 = tk & 255, len = (tk >> 8) & 255, o = (tk >> 16) & 7;
    if (A.child[8 * P + o] < 0) continue;   // uniform per warp
    const size_t g = (size_t)ci * 8 + o;
    const int myq = lane < len ? order[g * kQ + r0 + lane] : 0;
    // one child slot per run (the host marked every such cone relevant)
    const T* C = A.coefs_c + (size_t)cslot[o][__shfl_sync(0xffffffffu, myq, 0)] * kQ * NC + col;
    T c[kQ];
#pragma unroll
    for (int k = 0; k < kQ; ++k) c[k] = __ldg(C + k * NC);
    for (int a = 0; a < len; a += kP) {
      const int pi = a + sub;
      const bool on = pi < len;   // equal for both lanes of a (re, im) pair
      const int q = __shfl_sync(0xffffffffu, myq, on ? pi : 0);
      const T* Q = pt[o][q];
      T v = 0;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        T ei = 0;
#pragma unroll
        for (int j = 0; j < 5; ++j) {
          T dj = 0;
#pragma unroll
          for (int k = 0; k < 5; ++k) dj += Q[8 + k] * c[(i * 5 + j) * 5 + k];
          ei += Q[3 + j] * dj;
        }
        v += Q[i] * ei;
      }
      const T wv = __shfl_xor_sync(0xffffffffu, v, 1);
      if (on) {
        const T re = odd ? wv : v, im = odd ? v : wv;
        const T fr = Q[13], fi = Q[14];
        vals[q * kS + col] += odd ? (re * fi + im * fr) : (re * fr - im * fi);
      }
    }
  }
  __syncthreads();
  vals_to_coefs_block<T, kS, NC>(M, vals, A.coefs_p + (size_t)pslot * kQ * NC, 1);
}

// (c): a warp per target; its (target, cone segment) pairs are taken 32 at a time for the
// scalars (one pair per lane, centred factor of kernel ks only) and 32 / NC at a time for the
// contraction (NC lanes per pair, one column each); the lanes of equal column sum at the end.
constexpr int kTgtPassWarps = 8;

template <int NC, typename TO>
__global__ void __launch_bounds__(32 * kTgtPassWarps, 2) k_target_pass(TgtArgs<float, TO> A, int ks, int d0) {
  using T = float;
  constexpr int kG = 32 / NC;   // pairs per contraction step
  __shared__ TgtScal<T> sc[kTgtPassWarps][32];
  const int warp = threadIdx.x >> 5;
  const int t = blockIdx.x * kTgtPassWarps + warp;
  const int lane = threadIdx.x & 31;
  if (t >= A.N) return;   // uniform per warp
  const int64_t e0 = A.tgt_ptr[t], e1 = A.tgt_ptr[t + 1];
  if (e0 == e1) return;
  const double x0 = A.x_sorted[3 * (size_t)t], x1 = A.x_sorted[3 * (size_t)t + 1], x2 = A.x_sorted[3 * (size_t)t + 2];
  const T n0 = (T)A.n_sorted[3 * (size_t)t], n1 = (T)A.n_sorted[3 * (size_t)t + 1], n2 = (T)A.n_sorted[3 * (size_t)t + 2];
  const int g = lane / NC, c = lane % NC;
  TgtScal<T>* S = sc[warp];
  T accS = 0, accD = 0;
  for (int64_t c0 = e0; c0 < e1; c0 += 32) {
    const int nc = (int)min((int64_t)32, e1 - c0);
    if (lane < nc) tgt_scalars(A, x0, x1, x2, n0, n1, n2, A.tgt_slot[c0 + lane], S[lane], 1 << ks);
    __syncwarp();
    for (int cI = 0; cI < nc; cI += kG) {
      const bool on = cI + g < nc;   // equal for both lanes of a (re, im) pair
      const TgtScal<T>& Q = S[on ? cI + g : cI];
      const T* C = A.coefs + (size_t)Q.slot * kQ * NC + c;
      T cc[kQ];
#pragma unroll
      for (int k = 0; k < kQ; ++k) cc[k] = __ldg(C + k * NC);
      T oS, oD;
      tgt_contract(Q, cc, ks, (c & 1) != 0, oS, oD);
      if (on) {
        accS += oS;
        accD += oD;
      }
    }
    __syncwarp();
  }
#pragma unroll
  for (int o = NC; o < 32; o <<= 1) {
    accS += __shfl_xor_sync(0xffffffffu, accS, o);
    accD += __shfl_xor_sync(0xffffffffu, accD, o);
  }
  if (lane < NC) {
    TO* out = A.f28 + 56 * (size_t)A.perm[t];
    const int dens = d0 + (c >> 1);
    out[2 * (8 * ks + dens) + (c & 1)] += (TO)accS;
    if (dens < 6) out[2 * (16 + 6 * ks + dens) + (c & 1)] += (TO)accD;
  }
}

// One traversal per group of fields and right-hand side: (a), then per level (c) and (b).
template <int NC, typename TO>
cudaError_t run_passes(ifgf_plan_t* p, cudaStream_t s, int nrhs) {
  constexpr int F = NC / 2;
  const int D = p->tree.D, N = p->N;
  const float ke = (float)p->desc.k_ext, ki = (float)p->desc.k_int;
  for (int rb = 0; rb < nrhs; ++rb) {
    const float* a_rhs = (const float*)p->a_sorted + 16 * (size_t)N * rb;
    TO* f_rhs = (TO*)p->f28 + 56 * (size_t)N * rb;
    for (int ks = 0; ks < 2; ++ks)
      for (int d0 = 0; d0 < 8; d0 += F) {
        {
          const DevLevel& L = p->dl[D];
          LeafArgs<float> A{L.box_pt_ptr, L.box_slot_ptr, L.slot_cone, L.box_center, cone_geom_t<float>(L.cg),
                            p->x_sorted, a_rhs, (float*)L.coefs, ke, ki, 0, 0, nullptr, 0};
          const int rec = timer_begin(p, TK_LEAF, s);
          if (L.nboxes > 0 && L.max_box_slots > 0)
            k_leaf_pass<NC><<<dim3((unsigned)L.nboxes, (unsigned)((L.max_box_slots + kLeafSlots - 1) / kLeafSlots)),
                              kLeafThreads, 0, s>>>(A, ks, d0);
          timer_end(p, rec, s);
          ++p->launches;
        }
        for (int d = D; d >= 3; --d) {
          const DevLevel& L = p->dl[d];
          TgtArgs<float, TO> B{N, L.tgt_ptr, L.tgt_slot, L.slot_box, L.slot_cone, L.box_center,
                               cone_geom_t<float>(L.cg), (const float*)L.coefs, p->x_sorted, p->n_sorted, p->perm,
                               f_rhs, ke, ki, 0, L.cg.h, 1.0 / L.cg.ds(), p->desc.k_ext, p->desc.k_int, L.trig_th,
                               L.trig_ph};
          int rec = timer_begin(p, TK_TARGET, s);
          k_target_pass<NC, TO><<<(unsigned)((N + kTgtPassWarps - 1) / kTgtPassWarps), 32 * kTgtPassWarps, 0, s>>>(
              B, ks, d0);
          timer_end(p, rec, s);
          ++p->launches;
          if (d > 3) {
            const DevLevel& Pp = p->dl[d - 1];
            UpArgs<float> U{Pp.slot_box, Pp.slot_cone, Pp.slot_upidx, Pp.child, cone_geom_t<float>(Pp.cg),
                            L.cmap, L.ncomp, L.ckeys, cone_geom_t<float>(L.cg), L.H, Pp.up_cc,
                            (const float*)L.coefs, (float*)Pp.coefs, ke, ki, 0, 0, nullptr, 0};
            rec = timer_begin(p, TK_UP, s);
            // 16 columns: by runs (1.5-1.6x the all-fields IFGF time per forward map, against 1.9-2.0x
            // with a task per (point, column)); 2 columns: by tasks (the runs' 16 points per warp step
            // left the upward step 1.5x slower there)
            if (Pp.nslots > 0) {
              bool runs = false;
              if constexpr (NC == 16) {
                runs = Pp.up_task_ptr != nullptr;
                if (runs)
                  k_up_pass_runs<NC><<<(unsigned)Pp.nslots, 32 * kUpGroups, 0, s>>>(U, Pp.up_order, Pp.up_task,
                                                                                   Pp.up_task_ptr, ks);
              }
              if (!runs) k_up_pass<NC><<<(unsigned)Pp.nslots, kUpThreads, 0, s>>>(U, ks);
            }
            timer_end(p, rec, s);
            ++p->launches;
          }
        }
      }
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_far_ifgf_pass(ifgf_plan_t* p, cudaStream_t s, int nrhs) {
  if (!narrow_passes(p->desc) || ifgf64(p->desc)) return cudaErrorInvalidValue;
  const bool out64 = store64(p->desc);
  if (p->desc.fields_per_pass == 8)
    return out64 ? run_passes<16, double>(p, s, nrhs) : run_passes<16, float>(p, s, nrhs);
  return out64 ? run_passes<2, double>(p, s, nrhs) : run_passes<2, float>(p, s, nrhs);
}

}  // namespace ifgf
