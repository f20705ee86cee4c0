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
// The momentum constraint (Sec. III-C, Eqs. lin_momentum / ang_momentum)
// needs P_bsm - P_asm and L_asm - L_bsm.  With dx = x_asm - x_bsm and
// dv = v_asm - v_bsm per particle (the differences of the stored FP32
// values, exact in FP32 where the two lie within a factor of two of each
// other) and dc = c_asm - c_bsm = sum m dx / M, exactly
//   P_bsm - P_asm = -sum m dv,
//   L_asm - L_bsm = sum m [ r_bsm x dv + dx x v_asm ] - dc x P_asm,
// with r_bsm = x_bsm - c_bsm.  The terms are of the size of the
// shape-matching correction, so these FP32 sums carry no cancellation,
// unlike the difference of two whole-body sums, and they see the rounding
// of the stored x_asm and v_asm.  The explicit intrinsics fix the rounding
// of the per-particle terms, so every kernel that forms them gets the same
// bits.
// ---------------------------------------------------------------------------

__device__ __forceinline__ float3 cross_rn(float3 a, float3 b) {
  return make_float3(__fsub_rn(__fmul_rn(a.y, b.z), __fmul_rn(a.z, b.y)),
                     __fsub_rn(__fmul_rn(a.z, b.x), __fmul_rn(a.x, b.z)),
                     __fsub_rn(__fmul_rn(a.x, b.y), __fmul_rn(a.y, b.x)));
}

// Adds one particle's terms to the 12 first sums of shape matching:
// s[0..2] sum m e, s[3..11] sum m e q^T (row major), e = x_bsm - anchor.
__device__ __forceinline__ void shape_terms(float *s, float m, float3 e, float4 q) {
  const float3 me = make_float3(__fmul_rn(m, e.x), __fmul_rn(m, e.y), __fmul_rn(m, e.z));
  s[0] = __fadd_rn(s[0], me.x);
  s[1] = __fadd_rn(s[1], me.y);
  s[2] = __fadd_rn(s[2], me.z);
  s[3] = __fmaf_rn(me.x, q.x, s[3]);
  s[4] = __fmaf_rn(me.x, q.y, s[4]);
  s[5] = __fmaf_rn(me.x, q.z, s[5]);
  s[6] = __fmaf_rn(me.y, q.x, s[6]);
  s[7] = __fmaf_rn(me.y, q.y, s[7]);
  s[8] = __fmaf_rn(me.y, q.z, s[8]);
  s[9] = __fmaf_rn(me.z, q.x, s[9]);
  s[10] = __fmaf_rn(me.z, q.y, s[10]);
  s[11] = __fmaf_rn(me.z, q.z, s[11]);
}

// From the 12 first sums: c_bsm - anchor (cA) and A = sum m (x - c) q^T =
// sum m (x - a) q^T - (c - a) (sum m q)^T
__device__ __forceinline__ float3 shape_matrix(const float *s, float iM, float qsx, float qsy, float qsz,
                                               float *A) {
  const float3 cA = make_float3(__fmul_rn(iM, s[0]), __fmul_rn(iM, s[1]), __fmul_rn(iM, s[2]));
  const float ca[3] = {cA.x, cA.y, cA.z}, qs[3] = {qsx, qsy, qsz};
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) A[3 * r + c] = __fsub_rn(s[3 + 3 * r + c], __fmul_rn(ca[r], qs[c]));
  return cA;
}

// Adds one particle's terms to the kMomentumSums sums of the momentum step:
// s[0..2] sum m dv, s[3..5] sum m dx, s[6..8] sum m (r_bsm x dv + dx x v_asm),
// s[9..11] sum m v_asm, s[12..17] sum m e e^T (upper triangle,
// e = x_asm - anchor) for the inertia.
constexpr int kMomentumSums = 18;
__device__ __forceinline__ void momentum_terms(float *s, float m, float3 rb, float3 xb, float3 vb, float3 xa,
                                               float3 va, float3 e) {
  const float3 dx = make_float3(__fsub_rn(xa.x, xb.x), __fsub_rn(xa.y, xb.y), __fsub_rn(xa.z, xb.z));
  const float3 dv = make_float3(__fsub_rn(va.x, vb.x), __fsub_rn(va.y, vb.y), __fsub_rn(va.z, vb.z));
  s[0] = __fmaf_rn(m, dv.x, s[0]);
  s[1] = __fmaf_rn(m, dv.y, s[1]);
  s[2] = __fmaf_rn(m, dv.z, s[2]);
  s[3] = __fmaf_rn(m, dx.x, s[3]);
  s[4] = __fmaf_rn(m, dx.y, s[4]);
  s[5] = __fmaf_rn(m, dx.z, s[5]);
  const float3 a = cross_rn(rb, dv), b = cross_rn(dx, va);
  s[6] = __fmaf_rn(m, __fadd_rn(a.x, b.x), s[6]);
  s[7] = __fmaf_rn(m, __fadd_rn(a.y, b.y), s[7]);
  s[8] = __fmaf_rn(m, __fadd_rn(a.z, b.z), s[8]);
  s[9] = __fmaf_rn(m, va.x, s[9]);
  s[10] = __fmaf_rn(m, va.y, s[10]);
  s[11] = __fmaf_rn(m, va.z, s[11]);
  const float3 me = make_float3(__fmul_rn(m, e.x), __fmul_rn(m, e.y), __fmul_rn(m, e.z));
  s[12] = __fmaf_rn(me.x, e.x, s[12]);
  s[13] = __fmaf_rn(me.x, e.y, s[13]);
  s[14] = __fmaf_rn(me.x, e.z, s[14]);
  s[15] = __fmaf_rn(me.y, e.y, s[15]);
  s[16] = __fmaf_rn(me.y, e.z, s[16]);
  s[17] = __fmaf_rn(me.z, e.z, s[17]);
}

// S = sum m r r^T about c_asm from the anchor-relative sums s[12..17]
// (upper triangle: s00 s01 s02 s11 s12 s22)
__device__ __forceinline__ void body_second_moment(const float *s, float3 cA2, float M, float *S) {
  const float3 Mc = make_float3(__fmul_rn(M, cA2.x), __fmul_rn(M, cA2.y), __fmul_rn(M, cA2.z));
  S[0] = __fsub_rn(s[12], __fmul_rn(Mc.x, cA2.x));
  S[1] = __fsub_rn(s[13], __fmul_rn(Mc.x, cA2.y));
  S[2] = __fsub_rn(s[14], __fmul_rn(Mc.x, cA2.z));
  S[3] = __fsub_rn(s[15], __fmul_rn(Mc.y, cA2.y));
  S[4] = __fsub_rn(s[16], __fmul_rn(Mc.y, cA2.z));
  S[5] = __fsub_rn(s[17], __fmul_rn(Mc.z, cA2.z));
}

// From the body totals of momentum_terms: c_asm - anchor (cA2),
// dv = (P_bsm - P_asm) / M and w = I^-1 (L_asm - L_bsm) with I about c_asm
// (either left 0 when its part of the constraint is switched off).
__device__ __forceinline__ void momentum_step(const float *s, float3 cA, float M, float iM, bool lin, bool ang,
                                              float3 &cA2, float3 &dv, float3 &om) {
  const float3 dc = make_float3(__fmul_rn(iM, s[3]), __fmul_rn(iM, s[4]), __fmul_rn(iM, s[5]));
  cA2 = make_float3(__fadd_rn(cA.x, dc.x), __fadd_rn(cA.y, dc.y), __fadd_rn(cA.z, dc.z));
  dv = lin ? make_float3(-__fmul_rn(iM, s[0]), -__fmul_rn(iM, s[1]), -__fmul_rn(iM, s[2])) : make_float3(0.f, 0.f, 0.f);
  om = make_float3(0.f, 0.f, 0.f);
  if (ang) {
    const float3 cp = cross_rn(dc, make_float3(s[9], s[10], s[11]));
    const float3 dL = make_float3(__fsub_rn(s[6], cp.x), __fsub_rn(s[7], cp.y), __fsub_rn(s[8], cp.z));
    float S[6];
    body_second_moment(s, cA2, M, S);
    const float tr = __fadd_rn(__fadd_rn(S[0], S[3]), S[5]);
    // I = tr(S) I3 - S
    solve_sym3(tr - S[0], -S[1], -S[2], tr - S[3], -S[4], tr - S[5], dL, om);
  }
}

// ---------------------------------------------------------------------------
// Exact culling of the neighbour search.  A particle p can only be within R_n
// of a particle of body B if it lies within R_n of B's bounding box.  Every
// test below carries a margin that covers the FP32 rounding of the frame
// change and of |R| != 1, so culling never drops a pair of the O(N^2)
// definition.
// ---------------------------------------------------------------------------

// the search reach R_n with its rounding margin
__device__ __forceinline__ float cull_reach(float Rn2) { return sqrtf(Rn2) * (1.f + 1e-5f) + 1e-6f; }

// grows the box half-extents e of a body (centre cen) for rounding; returns
// the radius of its bounding sphere
__device__ __forceinline__ float cull_box_grow(float3 &e, float3 cen) {
  const float g = 1e-5f * (e.x + e.y + e.z + fabsf(cen.x) + fabsf(cen.y) + fabsf(cen.z)) + 1e-6f;
  e.x += g;
  e.y += g;
  e.z += g;
  return sqrtf(e.x * e.x + e.y * e.y + e.z * e.z) * (1.f + 1e-5f) + 1e-6f;
}

// bodies a (sphere centre ca, radius ra) and b may hold a pair within R_n
__device__ __forceinline__ bool cull_spheres_near(float3 ca, float ra, float3 cb, float rb, float reach) {
  const float3 d = make_float3(ca.x - cb.x, ca.y - cb.y, ca.z - cb.z);
  const float lim = ra + rb + reach +
                    1e-5f * (fabsf(ca.x) + fabsf(ca.y) + fabsf(ca.z) + fabsf(cb.x) + fabsf(cb.y) + fabsf(cb.z) + ra + rb) +
                    1e-6f;
  return d.x * d.x + d.y * d.y + d.z * d.z <= lim * lim;
}

// particle x lies within R_n of the box (centre cen, half-extents e, axes the
// columns of R) of another body
__device__ __forceinline__ bool cull_near_box(float3 x, float3 cen, float3 e, const float *R, float reach) {
  const float3 d = make_float3(x.x - cen.x, x.y - cen.y, x.z - cen.z);
  const float ux = fmaxf(fabsf(R[0] * d.x + R[3] * d.y + R[6] * d.z) - e.x, 0.f);
  const float uy = fmaxf(fabsf(R[1] * d.x + R[4] * d.y + R[7] * d.z) - e.y, 0.f);
  const float uz = fmaxf(fabsf(R[2] * d.x + R[5] * d.y + R[8] * d.z) - e.z, 0.f);
  const float lim = reach + 1e-5f * (fabsf(d.x) + fabsf(d.y) + fabsf(d.z)) + 1e-6f;
  return ux * ux + uy * uy + uz * uz <= lim * lim;
}

}  // namespace
}  // namespace pbdr
