// Per-body 3x3 math of the PBD-R solver shared by the streaming and the
// scene-resident kernels: quaternion <-> matrix, symmetric 3x3 solves and
// the rotation of the shape-matching fit.  Every lane of a warp calls these
// with identical inputs and gets identical results.
#pragma once

#include <cuda_runtime.h>

namespace pbdr {
namespace {

__device__ __forceinline__ float3 m3add(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 m3scale(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float m3dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 m3cross(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ void quat_to_mat(float4 q, float *R) {
  // q = (x, y, z, w), unit
  const float x = q.x, y = q.y, z = q.z, w = q.w;
  R[0] = 1.f - 2.f * (y * y + z * z);
  R[1] = 2.f * (x * y - z * w);
  R[2] = 2.f * (x * z + y * w);
  R[3] = 2.f * (x * y + z * w);
  R[4] = 1.f - 2.f * (x * x + z * z);
  R[5] = 2.f * (y * z - x * w);
  R[6] = 2.f * (x * z - y * w);
  R[7] = 2.f * (y * z + x * w);
  R[8] = 1.f - 2.f * (x * x + y * y);
}

// solve the symmetric system S u = g (S = [s00 s01 s02; . s11 s12; . . s22]);
// returns false if S is not positive definite (leading minors) or singular
__device__ __forceinline__ bool solve_spd3(float s00, float s01, float s02, float s11, float s12,
                                           float s22, float3 g, float3 &u, float rel_tol) {
  const float c00 = s11 * s22 - s12 * s12;
  const float c01 = s02 * s12 - s01 * s22;
  const float c02 = s01 * s12 - s02 * s11;
  const float det = s00 * c00 + s01 * c01 + s02 * c02;
  const float tr = (s00 + s11 + s22) * (1.f / 3.f);
  if (!(s00 > 0.f) || !(s00 * s11 - s01 * s01 > 0.f) || !(det > rel_tol * tr * tr * tr)) {
    u = make_float3(0.f, 0.f, 0.f);
    return false;
  }
  const float c11 = s00 * s22 - s02 * s02;
  const float c12 = s01 * s02 - s00 * s12;
  const float c22 = s00 * s11 - s01 * s01;
  const float id = 1.f / det;
  u.x = (c00 * g.x + c01 * g.y + c02 * g.z) * id;
  u.y = (c01 * g.x + c11 * g.y + c12 * g.z) * id;
  u.z = (c02 * g.x + c12 * g.y + c22 * g.z) * id;
  return true;
}

// unit quaternion (x, y, z, w) of a rotation matrix (Shepperd's method:
// branch on the largest of the trace and the diagonal)
__device__ __forceinline__ float4 mat_to_quat(const float *R) {
  const float tr = R[0] + R[4] + R[8];
  float4 q;
  if (tr >= R[0] && tr >= R[4] && tr >= R[8]) {
    const float s = 2.f * sqrtf(fmaxf(1.f + tr, 1e-30f));
    q = make_float4((R[7] - R[5]) / s, (R[2] - R[6]) / s, (R[3] - R[1]) / s, 0.25f * s);
  } else if (R[0] >= R[4] && R[0] >= R[8]) {
    const float s = 2.f * sqrtf(fmaxf(1.f + R[0] - R[4] - R[8], 1e-30f));
    q = make_float4(0.25f * s, (R[1] + R[3]) / s, (R[2] + R[6]) / s, (R[7] - R[5]) / s);
  } else if (R[4] >= R[8]) {
    const float s = 2.f * sqrtf(fmaxf(1.f + R[4] - R[0] - R[8], 1e-30f));
    q = make_float4((R[1] + R[3]) / s, 0.25f * s, (R[5] + R[7]) / s, (R[2] - R[6]) / s);
  } else {
    const float s = 2.f * sqrtf(fmaxf(1.f + R[8] - R[0] - R[4], 1e-30f));
    q = make_float4((R[2] + R[6]) / s, (R[5] + R[7]) / s, 0.25f * s, (R[3] - R[1]) / s);
  }
  const float n = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
  return make_float4(q.x * n, q.y * n, q.z * n, q.w * n);
}

// Orthogonal polar factor of a nonsingular A by Higham's scaled Newton
// iteration X <- (g X + (g X)^-T)/2, g = (|X^-1|_F / |X|_F)^(1/2).
// Returns false if A is (nearly) singular or the factor is a reflection.
__device__ bool polar_higham(const float *A, float *U) {
  float X[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) X[k] = A[k];
  for (int it = 0; it < 24; ++it) {
    // cofactors C_ij: X^-T = C / det
    const float c0 = X[4] * X[8] - X[5] * X[7], c1 = X[5] * X[6] - X[3] * X[8],
                c2 = X[3] * X[7] - X[4] * X[6], c3 = X[2] * X[7] - X[1] * X[8],
                c4 = X[0] * X[8] - X[2] * X[6], c5 = X[1] * X[6] - X[0] * X[7],
                c6 = X[1] * X[5] - X[2] * X[4], c7 = X[2] * X[3] - X[0] * X[5],
                c8 = X[0] * X[4] - X[1] * X[3];
    const float det = X[0] * c0 + X[1] * c1 + X[2] * c2;
    float nx = 0.f, nc = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) nx += X[k] * X[k];
    const float C[9] = {c0, c1, c2, c3, c4, c5, c6, c7, c8};
#pragma unroll
    for (int k = 0; k < 9; ++k) nc += C[k] * C[k];
    if (!(fabsf(det) > 1e-30f) || !(nx > 0.f)) return false;
    const float ninv = sqrtf(nc) / fabsf(det);   // |X^-1|_F
    const float g = sqrtf(ninv / sqrtf(nx));
    const float a = 0.5f * g, b = 0.5f / (g * det);
    float diff = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float xn = a * X[k] + b * C[k];
      diff += (xn - X[k]) * (xn - X[k]);
      X[k] = xn;
    }
    if (diff < 1e-12f) break;
  }
  const float det = X[0] * (X[4] * X[8] - X[5] * X[7]) - X[1] * (X[3] * X[8] - X[5] * X[6]) +
                    X[2] * (X[3] * X[7] - X[4] * X[6]);
  if (!(det > 0.5f)) return false;
#pragma unroll
  for (int k = 0; k < 9; ++k) U[k] = X[k];
  return true;
}

// Rotation maximising tr(R^T A) over SO(3) (the rotation of the least-squares
// rigid fit of shape matching), by Newton steps on SO(3) from the warm start
// q: with r_i, a_i the columns of R and A, the objective near R is
// f(th) ~ f + g.th - th^T H th / 2 with g = sum r_i x a_i and
// H = (sum r_i.a_i) I3 - sym(sum r_i a_i^T), so th = H^-1 g.  If H is not
// positive definite at the warm start (the start is far from the optimum),
// the start is replaced by the polar factor from Higham's iteration; where
// that fails too (singular or inverted A) damped gradient steps are taken.
__device__ __forceinline__ float4 shape_rotation(const float *A, float4 q) {
  bool restarted = false;
  for (int it = 0; it < 8; ++it) {
    float R[9];
    quat_to_mat(q, R);
    float3 g = make_float3(0.f, 0.f, 0.f);
    float M[9];
    float t = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float3 r = make_float3(R[i], R[3 + i], R[6 + i]);
      const float3 av = make_float3(A[i], A[3 + i], A[6 + i]);
      g = m3add(g, m3cross(r, av));
      t += m3dot(r, av);
    }
    // sum_i r_i a_i^T = R A^T
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        M[3 * r + c] = R[3 * r + 0] * A[3 * c + 0] + R[3 * r + 1] * A[3 * c + 1] +
                       R[3 * r + 2] * A[3 * c + 2];
    float3 th;
    const bool ok = solve_spd3(t - M[0], -0.5f * (M[1] + M[3]), -0.5f * (M[2] + M[6]), t - M[4],
                               -0.5f * (M[5] + M[7]), t - M[8], g, th, 1e-6f);
    if (!ok) {
      float U[9];
      if (!restarted && polar_higham(A, U)) {
        restarted = true;
        q = mat_to_quat(U);
        continue;
      }
      const float gn = sqrtf(m3dot(g, g));
      const float den = fabsf(t) + gn + 1e-30f;
      th = m3scale(1.f / den, g);
    }
    const float thn2 = m3dot(th, th);
    // q <- normalize(q + (0, th/2) (x) q)
    const float4 dq = make_float4(0.5f * (th.x * q.w + th.y * q.z - th.z * q.y),
                                  0.5f * (th.y * q.w + th.z * q.x - th.x * q.z),
                                  0.5f * (th.z * q.w + th.x * q.y - th.y * q.x),
                                  -0.5f * (th.x * q.x + th.y * q.y + th.z * q.z));
    q = make_float4(q.x + dq.x, q.y + dq.y, q.z + dq.z, q.w + dq.w);
    const float qn = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    q = make_float4(q.x * qn, q.y * qn, q.z * qn, q.w * qn);
    // Newton converges quadratically: after a step below 3e-4 rad the
    // remaining error is ~1e-7 rad, the FP32 resolution of the rotation
    if (thn2 < 1e-7f) break;
  }
  return q;
}


// I u = g for the symmetric positive definite inertia-like matrix I; u = 0
// when I is singular (a one-particle or colinear body has no angular part)
__device__ __forceinline__ void solve_sym3(float s00, float s01, float s02, float s11, float s12,
                                           float s22, float3 g, float3 &u) {
  solve_spd3(s00, s01, s02, s11, s12, s22, g, u, 1e-6f);
}

// ---------------------------------------------------------------------------
// Compensated body sums.  The momentum constraint (Sec. III-C, Eqs.
// lin_momentum / ang_momentum) restores P and L from the difference of two
// body sums taken a pass apart, so FP32 rounding of those sums is what FP32
// leaves of the conservation.  The centroid, P and L sums are therefore carried
// as unevaluated pairs s + lo: every addition of two partial sums is split by
// Knuth's TwoSum into the rounded sum and its exact rounding error, which is
// kept in lo.  The intrinsics fix the operations (no contraction), and TwoSum's
// error term is unique, so both partners of a butterfly step get the same pair.
// ---------------------------------------------------------------------------

// a + b = s + e exactly (Knuth, The Art of Computer Programming vol. 2, 4.2.2)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (s, lo) <- (s, lo) + (s2, lo2)
__device__ __forceinline__ void cadd(float &s, float &lo, float s2, float lo2) {
  float e;
  two_sum(s, s2, s, e);
  lo = __fadd_rn(__fadd_rn(lo, lo2), e);
}

// butterfly warp sum of a compensated value; every lane ends with the same pair
__device__ __forceinline__ void warp_sum_c(float &s, float &lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, o), l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    cadd(s, lo, s2, l2);
  }
}

__device__ __forceinline__ float cval(float s, float lo) { return __fadd_rn(s, lo); }

// (a_s + a_l) - (b_s + b_l) with the two large parts subtracted first (exact
// when they are within a factor of two, as two sums a pass apart are)
__device__ __forceinline__ float cdiff(float as, float al, float bs, float bl) {
  return __fadd_rn(__fsub_rn(as, bs), __fsub_rn(al, bl));
}

__device__ __forceinline__ float3 cross_rn(float3 a, float3 b) {
  return make_float3(__fsub_rn(__fmul_rn(a.y, b.z), __fmul_rn(a.z, b.y)),
                     __fsub_rn(__fmul_rn(a.z, b.x), __fmul_rn(a.x, b.z)),
                     __fsub_rn(__fmul_rn(a.x, b.y), __fmul_rn(a.y, b.x)));
}

// First-pass (X_bsm, V_bsm) quantities of a body kept for the momentum step:
// P_bsm as a pair, the anchor-relative L sum's large part, and
// lo(L sum) - (c_bsm - a) x P_bsm, so that L_bsm = Ls + T.
struct BsmMoments {
  float3 Ps, Pl, Ls, T;
};

__device__ __forceinline__ BsmMoments bsm_moments(const float *Ps, const float *Pl, const float *Ls,
                                                  const float *Ll, float3 cA) {
  BsmMoments r;
  r.Ps = make_float3(Ps[0], Ps[1], Ps[2]);
  r.Pl = make_float3(Pl[0], Pl[1], Pl[2]);
  r.Ls = make_float3(Ls[0], Ls[1], Ls[2]);
  const float3 P = make_float3(cval(Ps[0], Pl[0]), cval(Ps[1], Pl[1]), cval(Ps[2], Pl[2]));
  const float3 cp = cross_rn(cA, P);
  r.T = make_float3(__fsub_rn(Ll[0], cp.x), __fsub_rn(Ll[1], cp.y), __fsub_rn(Ll[2], cp.z));
  return r;
}

__device__ __forceinline__ float3 bsm_P(const BsmMoments &b) {
  return make_float3(cval(b.Ps.x, b.Pl.x), cval(b.Ps.y, b.Pl.y), cval(b.Ps.z, b.Pl.z));
}

// P_bsm - P_asm from the pairs
__device__ __forceinline__ float3 momentum_dP(const BsmMoments &b, const float *Pas, const float *Pal) {
  return make_float3(cdiff(b.Ps.x, b.Pl.x, Pas[0], Pal[0]), cdiff(b.Ps.y, b.Pl.y, Pas[1], Pal[1]),
                     cdiff(b.Ps.z, b.Pl.z, Pas[2], Pal[2]));
}

// L_asm - L_bsm, both about their own centre of mass: L = (anchor-relative
// sum) - (c - a) x P; the large parts of the two sums are subtracted first
__device__ __forceinline__ float3 momentum_dL(const BsmMoments &b, const float *Las, const float *Lal,
                                              float3 cA2, float3 Pa) {
  const float3 cp = cross_rn(cA2, Pa);
  const float3 Ta = make_float3(__fsub_rn(Lal[0], cp.x), __fsub_rn(Lal[1], cp.y), __fsub_rn(Lal[2], cp.z));
  return make_float3(__fadd_rn(__fsub_rn(Las[0], b.Ls.x), __fsub_rn(Ta.x, b.T.x)),
                     __fadd_rn(__fsub_rn(Las[1], b.Ls.y), __fsub_rn(Ta.y, b.T.y)),
                     __fadd_rn(__fsub_rn(Las[2], b.Ls.z), __fsub_rn(Ta.z, b.T.z)));
}

}  // namespace
}  // namespace pbdr
