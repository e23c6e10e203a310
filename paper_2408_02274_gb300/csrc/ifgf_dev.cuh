// Device helpers and argument blocks shared by the IFGF far-field kernels: the vectorised
// kernels of all 16 (density, kernel) fields (ifgf.cu) and the per-pass variants that carry
// fewer fields per octree traversal (ifgf_pass.cu).  Everything here sits in an anonymous
// namespace, so each translation unit has its own copy.
#pragma once
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

// Tensor-core operand image of one cone segment's coefficients (the upward step on the tensor
// cores copies it to shared memory as is): the 32 real columns m as rows, K = 80 (k >= 75 zero),
// K-major without swizzle in 8-row x 16-byte core matrices (chunk kc = k / 4 of row m at float
// offset img_off(m, kc) + k % 4), first as TF32 hi parts (low 13 mantissa bits cleared), then the
// lo parts x - hi: 2 x 2560 floats per segment.
constexpr int kImgFloats = 2 * 32 * 80;
__device__ __forceinline__ int img_off(int m, int kc) { return (m >> 3) * 640 + kc * 32 + ((m & 7) << 2); }
__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xffffe000u); }

// The same transform for all kCols columns of `ns` consecutive [75][kStride] value
// buffers by the whole block (one (buffer, line, column) task per thread and pass,
// consecutive threads on consecutive columns), followed by a coalesced store of the
// 75 x kCols coefficients of buffer i to out + i * 75 * kCols (and, for the 32-column FP32
// buffers, their operand images when img is given).  Every thread of the block must call it.
template <typename T, int kStride, int kCols = 32>
__device__ void vals_to_coefs_block(const SmallMaps<T>& M, T* vb, T* out, int ns = 1, float* img = nullptr) {
  const int nt = blockDim.x;
  constexpr int kBuf = kQ * kStride;
  for (int e = threadIdx.x; e < ns * 15 * kCols; e += nt) {   // phi lines
    const int b = e / (15 * kCols), r = e - b * 15 * kCols, a = r / kCols, col = r % kCols;
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
  for (int e = threadIdx.x; e < ns * 15 * kCols; e += nt) {   // theta lines
    const int b = e / (15 * kCols), r = e - b * 15 * kCols, ik = r / kCols, col = r % kCols, is = ik / 5, k = ik % 5;
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
  for (int e = threadIdx.x; e < ns * 25 * kCols; e += nt) {   // s lines
    const int b = e / (25 * kCols), r = e - b * 25 * kCols, jk = r / kCols, col = r % kCols;
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
  for (int e = threadIdx.x; e < ns * kQ * kCols; e += nt) {
    const int b = e / (kQ * kCols), r = e - b * kQ * kCols;
    out[e] = vb[b * kBuf + (r / kCols) * kStride + (r % kCols)];
  }
  if constexpr (sizeof(T) == 4 && kCols == 32) {
    if (img) {   // tensor-core operand images of the same coefficients (see img_off)
      for (int e = threadIdx.x; e < ns * 32 * 20; e += nt) {
        const int b = e / (32 * 20), r = e - b * 32 * 20, m = r / 20, kc = r - m * 20;
        float x[4], h[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int k = 4 * kc + j;
          x[j] = k < kQ ? (float)vb[b * kBuf + k * kStride + m] : 0.f;
          h[j] = tf32_hi(x[j]);
        }
        float* im = img + (size_t)b * kImgFloats + img_off(m, kc);
        *reinterpret_cast<float4*>(im) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4*>(im + kImgFloats / 2) =
            make_float4(x[0] - h[0], x[1] - h[1], x[2] - h[2], x[3] - h[3]);
      }
    }
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
  float* img = nullptr;      // tensor-core operand images of the coefficients (FP32, when the upward
  size_t istride = 0;        // step into the level above runs on the tensor cores), per rhs stride
};

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
  float* img_p = nullptr;        // tensor-core operand images of the parent coefficients (or none)
  size_t istride_p = 0;          // per right-hand side
};


template <typename T, typename TO = T>
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
  TO* f28;
  T ke, ki;
  size_t cstride;   // cone coefficients per right-hand side (fields: 56 N)
  // FP64 geometry of the level for the FP32 kernel's target coordinates and centre phases
  double h64, ids64, ke64, ki64;
  const double2* th0;   // [na] (cos, sin) of the theta cells' lower edges g2 * pi / na
  const double2* ph0;   // [2 na] (cos, sin) of the phi cells' lower edges g3 * pi / na
};

// Target coordinates of the FP32 target step.  The target's local coordinates in its cone and
// the centre phases k |x - x_c| feed every interpolated value; rounded in FP32 they would carry
// ~1e-6 (local coordinates on fine cones, through a full-angle atan2) and ~k r 1e-7 (phases, k r
// up to ~1e2) of independent noise per target, which the N-Mueller combination's surface
// derivatives amplify.  So x - x_c, r, s = h / r and the phases are formed in FP64 (the phase
// reduced to [-pi, pi] before the FP32 sincos), and each angle is measured from its cell's lower
// edge by rotating the FP64 components (FP32 atan2 then resolves a small angle).
__device__ inline void target_coords(double h64, double ids64, float idth, const double2* th0, const double2* ph0,
                                     cone_key cone, double dx, double dy, double dz, double ke, double ki,
                                     float* ts, float* tt, float* tp, float* r, float* sth, float* cth, float* sph,
                                     float* cph, float* phase) {
  int g1, g2, g3;
  cone_decode(cone, &g1, &g2, &g3);
  const double rho2 = dx * dx + dy * dy;
  const double rho = sqrt(rho2), r64 = sqrt(rho2 + dz * dz);
  const double ir = 1.0 / r64;
  *ts = (float)(2.0 * (h64 * ir * ids64 - (double)g1) - 1.0);
  const double2 t0 = th0[g2], p0 = ph0[g3];
  *tt = 2.f * atan2f((float)(rho * t0.x - dz * t0.y), (float)(dz * t0.x + rho * t0.y)) * idth - 1.f;
  *tp = 2.f * atan2f((float)(dy * p0.x - dx * p0.y), (float)(dx * p0.x + dy * p0.y)) * idth - 1.f;
  *r = (float)r64;
  *sth = (float)(rho * ir);
  *cth = (float)(dz * ir);
  const double irho = rho > 0.0 ? 1.0 / rho : 0.0;
  *cph = rho > 0.0 ? (float)(dx * irho) : 1.f;
  *sph = rho > 0.0 ? (float)(dy * irho) : 0.f;
  constexpr double kInv2Pi = 1.0 / (2.0 * kPi);
  const double a = ke * r64, b = ki * r64;
  phase[0] = (float)fma(-2.0 * kPi, rint(a * kInv2Pi), a);
  phase[1] = (float)fma(-2.0 * kPi, rint(b * kInv2Pi), b);
}

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

// Per (target, cone segment) scalars: Chebyshev values and derivatives of the target's local
// coordinates, the directional-derivative weights of n . grad and the centred factors (of the
// kernels in kmask: bit 0 kappa_e, bit 1 kappa_i).
template <typename T, typename TO>
__device__ inline void tgt_scalars(const TgtArgs<T, TO>& A, double x0, double x1, double x2, T n0, T n1, T n2,
                                   int slot, TgtScal<T>& Q, int kmask = 3) {
  const T two_ids = T(2) * A.cg.ids, two_idth = T(2) * A.cg.idth, h = A.cg.h;
  const int box = A.slot_box[slot];
  const cone_key cone = A.slot_cone[slot];
  const double dx = x0 - A.box_center[3 * box], dy = x1 - A.box_center[3 * box + 1], dz = x2 - A.box_center[3 * box + 2];
  const T xr = (T)dx, yr = (T)dy, zr = (T)dz;
  T ts, tt, tp, r, sth, cth, sph, cph, phase[2];
  if constexpr (std::is_same<T, float>::value) {
    target_coords(A.h64, A.ids64, A.cg.idth, A.th0, A.ph0, cone, dx, dy, dz, A.ke64, A.ki64, &ts, &tt, &tp, &r, &sth,
                  &cth, &sph, &cph, phase);
  } else {
    local_coords(A.cg, cone, xr, yr, zr, &ts, &tt, &tp, &r, &sth, &cth, &sph, &cph);
    phase[0] = A.ke * r;
    phase[1] = A.ki * r;
  }
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
    if (!((kmask >> kk) & 1)) continue;   // the kernels whose factors are wanted (bit kk)
    const T kap = kk ? A.ki : A.ke;
    T sn, cs;
    sincos_t(phase[kk], &sn, &cs);
    const T Gr = g * cs, Gi = g * sn;
    Q.G[kk][0] = Gr;
    Q.G[kk][1] = Gi;
    Q.G[kk][2] = nr * (-ir * Gr - kap * Gi);
    Q.G[kk][3] = nr * (-ir * Gi + kap * Gr);
  }
  Q.slot = slot;
}


// The interpolated field of this lane's real column and its normal derivative at one (target,
// cone) pair, times the centred factor of kernel ks: the S part and the D part (used by the
// lanes of densities 0..5).  cc: the cone's 75 coefficients of this lane's column; odd: the
// lane holds the imaginary part (its partner, lane ^ 1, the real part of the same field).
template <typename T>
__device__ __forceinline__ void tgt_contract(const TgtScal<T>& Q, const T* cc, int ks, bool odd, T& outS, T& outD) {
  // separable contraction: the phi sums with T and T' are shared by F and its three
  // partial derivatives, dF = a_s F_s + a_theta F_theta + a_phi F_phi
  T Tp[5], dTp[5], Tt[5], dTt[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    Tp[k] = Q.Tp[k]; dTp[k] = Q.dTp[k]; Tt[k] = Q.Tt[k]; dTt[k] = Q.dTt[k];
  }
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
  const T Fr = odd ? Fw : F, Fi = odd ? F : Fw;
  const T dFr = odd ? dFw : dF, dFi = odd ? dF : dFw;
  outS = odd ? (Gr * Fi + Gi * Fr) : (Gr * Fr - Gi * Fi);
  const T Dr = dGr * Fr - dGi * Fi + Gr * dFr - Gi * dFi;
  const T Di = dGr * Fi + dGi * Fr + Gr * dFi + Gi * dFr;
  outD = odd ? Di : Dr;
}

}  // namespace

}  // namespace ifgf
