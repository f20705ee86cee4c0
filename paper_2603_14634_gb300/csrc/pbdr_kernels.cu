// PBD-R substep kernels for sm_103a.
//
// Data layout (all FP32, float4 SoA, one slot per particle in caller order):
//   X  = (x, y, z, w)        position and inverse mass w_p
//   V  = (vx, vy, vz, 0)     velocity
//   Q  = (qx, qy, qz, m)     rest offset q_p = x0_p - c0 and mass m_p
// Bodies are contiguous particle ranges; scenes are contiguous body ranges.
//
// Kernels of one substep (Algorithm 1):
//   k_predict   integration and the hashed-grid cell key of x~
//   (radix sort of (key, particle))
//   k_cells     bucket records ([start, end), body bounds) and positions in
//               sorted order
//   k_neighbors candidate lists N(p) with the exact FP32 predicate (ELL)
//   k_iterate   one solver iteration for one body per warp:
//               contacts -> X_bsm, V_bsm; shape matching -> X_asm, V_asm;
//               momentum enforcement -> X_{i+1}, V_{i+1}
#include <math.h>

#include <algorithm>

#include "pbdr_internal.cuh"
#include "pbdr_math.cuh"

namespace pbdr {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) {
  return make_float3(a.x + b.x, a.y + b.y, a.z + b.z);
}
__device__ __forceinline__ float3 operator-(float3 a, float3 b) {
  return make_float3(a.x - b.x, a.y - b.y, a.z - b.z);
}
__device__ __forceinline__ float3 operator*(float s, float3 a) {
  return make_float3(s * a.x, s * a.y, s * a.z);
}
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// ---- hashed uniform grid (FP32, round-to-nearest, no contraction) --------

__device__ __forceinline__ int32_t cell_coord(float x, float inv_h) {
  float u = floorf(__fmul_rn(x, inv_h));
  u = fminf(fmaxf(u, -1.0e9f), 1.0e9f);
  return (int32_t)u;
}

// Teschner et al. 2003 spatial hash of integer cell coordinates
__device__ __forceinline__ uint32_t cell_hash(int32_t ix, int32_t iy, int32_t iz) {
  return ((uint32_t)ix * 73856093u) ^ ((uint32_t)iy * 19349663u) ^ ((uint32_t)iz * 83492791u);
}

// squared distance, dx = x_q - x_p per axis, (dx^2 + dy^2) + dz^2, each op RN
__device__ __forceinline__ float d2_rn(float4 p, float4 q) {
  float dx = __fsub_rn(q.x, p.x), dy = __fsub_rn(q.y, p.y), dz = __fsub_rn(q.z, p.z);
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// ---------------------------------------------------------------------------
// integration step + cell keys
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_predict(PredictArgs a) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.np) return;
  const int32_t p = a.pmap ? a.pmap[i] : a.pbase + i;
  const int32_t b = a.pbody[p];
  const BodyRec br = a.bodies[b];
  const ScenePar sp = a.scenes[br.scene];
  float4 x = a.X0[p];
  if (a.predict) {
    const float4 v = a.V0[p];
    float3 acc = make_float3(sp.gx, sp.gy, sp.gz);
    if (br.has_wrench) {
      const BodyWrench wr = a.wrench[b];
      float3 r = f3(x) - f3(wr.com);
      acc = acc + f3(wr.aF) + cross(f3(wr.alpha), r);
    }
    // v~ = v + dt w f_ext ;  x~ = x_init + dt v~
    float3 vt = f3(v) + sp.dt * acc;
    float3 xt = f3(x) + sp.dt * vt;
    if (a.Xinit) a.Xinit[p] = x;
    x = make_float4(xt.x, xt.y, xt.z, x.w);
    a.Xp[p] = x;
    a.Vp[p] = make_float4(vt.x, vt.y, vt.z, 0.f);
  }
  const uint32_t h = cell_hash(cell_coord(x.x, sp.inv_h), cell_coord(x.y, sp.inv_h),
                               cell_coord(x.z, sp.inv_h));
  a.keys[i] = a.hbase[br.scene] + (h & (sp.T - 1u));
  a.vals[i] = (uint32_t)p;
}

// ---------------------------------------------------------------------------
// bucket ranges of the sorted keys + positions gathered in sorted order
// ---------------------------------------------------------------------------

// A bucket record holds [first, end) of the bucket in sorted order and the
// lowest and (bitwise NOT of the) highest body id among its particles; the
// records start as all ones (empty bucket, identities of both minima), so
// the body bounds come from integer minima and do not depend on the order
// of the updates.
__global__ void __launch_bounds__(256) k_cells(CellArgs a) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.np) return;
  const uint32_t key = a.skeys[i];
  uint32_t *rec = reinterpret_cast<uint32_t *>(a.cells + key);
  if (i == 0 || a.skeys[i - 1] != key) rec[0] = (uint32_t)i;
  if (i == a.np - 1 || a.skeys[i + 1] != key) rec[1] = (uint32_t)(i + 1);
  const uint32_t p = a.svals[i];
  const int32_t body = a.pbody[p];
  atomicMin(rec + 2, (uint32_t)body);
  atomicMin(rec + 3, ~(uint32_t)body);
  const float4 x = a.Xp[p];
  a.spos[i] = make_float4(x.x, x.y, x.z, __int_as_float(body));
}

// ---------------------------------------------------------------------------
// neighbour lists: N(p) = {q : body(q) != body(p), d2_rn(p, q) < Rn^2},
// ascending, stored column-major (slot j of particle p at j*stride + p)
// ---------------------------------------------------------------------------

constexpr int kNbrCapMax = 64;

// Bounding box of every body of the plan on its predicted positions, in the
// frame of its warm-start rotation, grown for rounding, and its bounding
// sphere (one warp per body).
__global__ void __launch_bounds__(128) k_body_bounds(BoundArgs a) {
  const int lane = threadIdx.x & 31;
  const int32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= a.nbodies) return;
  const int32_t b = a.bmap ? a.bmap[w] : a.bbase + w;
  const BodyRec br = a.bodies[b];
  const int32_t p0 = br.start, pe = br.start + br.count;
  const float3 o = f3(a.Xp[p0]);
  float sx = 0.f, sy = 0.f, sz = 0.f;
  for (int32_t p = p0 + lane; p < pe; p += 32) {
    const float4 x = a.Xp[p];
    sx += x.x - o.x;
    sy += x.y - o.y;
    sz += x.z - o.z;
  }
  sx = warp_sum(sx);
  sy = warp_sum(sy);
  sz = warp_sum(sz);
  const float inv = 1.f / (float)br.count;
  const float3 cen = make_float3(o.x + sx * inv, o.y + sy * inv, o.z + sz * inv);
  float R[9];
  quat_to_mat(a.quat[b], R);
  float ex = 0.f, ey = 0.f, ez = 0.f;
  for (int32_t p = p0 + lane; p < pe; p += 32) {
    const float4 x = a.Xp[p];
    const float dx = x.x - cen.x, dy = x.y - cen.y, dz = x.z - cen.z;
    ex = fmaxf(ex, fabsf(R[0] * dx + R[3] * dy + R[6] * dz));
    ey = fmaxf(ey, fabsf(R[1] * dx + R[4] * dy + R[7] * dz));
    ez = fmaxf(ez, fabsf(R[2] * dx + R[5] * dy + R[8] * dz));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    ex = fmaxf(ex, __shfl_xor_sync(kFull, ex, off));
    ey = fmaxf(ey, __shfl_xor_sync(kFull, ey, off));
    ez = fmaxf(ez, __shfl_xor_sync(kFull, ez, off));
  }
  if (lane == 0) {
    float3 e = make_float3(ex, ey, ez);
    const float rad = cull_box_grow(e, cen);
    a.bounds[2 * (int64_t)b] = make_float4(cen.x, cen.y, cen.z, rad);
    a.bounds[2 * (int64_t)b + 1] = make_float4(e.x, e.y, e.z, 0.f);
  }
}

// Near bodies of every body of the plan (bounding spheres within R_n of each
// other, same scene); the count goes to bounds[2 b + 1].w, the first
// kNearMax ids to near[kNearMax b ...].  One thread per body.
__global__ void __launch_bounds__(128) k_near_bodies(BoundArgs a) {
  const int32_t w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= a.nbodies) return;
  const int32_t b = a.bmap ? a.bmap[w] : a.bbase + w;
  const BodyRec br = a.bodies[b];
  const ScenePar sp = a.scenes[br.scene];
  const float reach = cull_reach(sp.Rn2);
  const float4 sa = a.bounds[2 * (int64_t)b];
  int nn = 0;
  for (int32_t bo = sp.b0; bo < sp.b0 + sp.nb; ++bo) {
    if (bo == b) continue;
    const float4 sb = a.bounds[2 * (int64_t)bo];
    if (cull_spheres_near(f3(sa), sa.w, f3(sb), sb.w, reach)) {
      if (nn < kNearMax) a.near[(int64_t)kNearMax * b + nn] = bo;
      ++nn;
    }
  }
  float4 e = a.bounds[2 * (int64_t)b + 1];
  e.w = __int_as_float(nn);
  a.bounds[2 * (int64_t)b + 1] = e;
}

// true when particle p (predicted position xp, body bp) lies within R_n of
// the box of a body near its own, or when its body has more near bodies
// than are listed: only such a particle can have a neighbour
__device__ __forceinline__ bool near_other_body(const NbrArgs &a, float4 xp, int32_t bp, const ScenePar &sp) {
  const int nn = __float_as_int(a.bounds[2 * (int64_t)bp + 1].w);
  if (nn > kNearMax) return true;
  const float reach = cull_reach(sp.Rn2);
  for (int k = 0; k < nn; ++k) {
    const int32_t bo = a.near[(int64_t)kNearMax * bp + k];
    const float4 c4 = a.bounds[2 * (int64_t)bo], e4 = a.bounds[2 * (int64_t)bo + 1];
    float R[9];
    quat_to_mat(a.quat[bo], R);
    if (cull_near_box(f3(xp), f3(c4), f3(e4), R, reach)) return true;
  }
  return false;
}

// the 27-cell search of particle p: its ascending list of particles of
// other bodies within R_n, into nbr / nbr_cnt
__device__ __forceinline__ void search_cells(const NbrArgs &a, int32_t p, float4 xp, int32_t bp, int32_t s,
                                             const ScenePar &sp) {
  const uint32_t hb = a.hbase[s], mask = sp.T - 1u;
  const int32_t ix = cell_coord(xp.x, sp.inv_h), iy = cell_coord(xp.y, sp.inv_h),
                iz = cell_coord(xp.z, sp.inv_h);
  int32_t list[kNbrCapMax];
  const int cap = a.cap;
  int cnt = 0;
  // each of the 27 cells once; a bucket shared by several cells (hash
  // collision) is scanned once per cell and only that cell's particles are
  // taken, so no candidate appears twice.  A bucket that holds particles of
  // the particle's own body only (most buckets around a body's interior) has
  // no candidate and is not scanned.
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int32_t cx = ix + dx, cy = iy + dy, cz = iz + dz;
        const uint4 rec = __ldg(a.cells + hb + (cell_hash(cx, cy, cz) & mask));
        if (rec.x == kEmptyCell) continue;
        if (rec.z == (uint32_t)bp && ~rec.w == (uint32_t)bp) continue;
        const uint32_t st = rec.x, en = rec.y;
        for (uint32_t j = st; j < en; ++j) {
          const float4 xq = a.spos[j];
          if (__float_as_int(xq.w) == bp) continue;
          if (cell_coord(xq.x, sp.inv_h) != cx || cell_coord(xq.y, sp.inv_h) != cy ||
              cell_coord(xq.z, sp.inv_h) != cz)
            continue;
          if (!(d2_rn(xp, xq) < sp.Rn2)) continue;
          const int32_t q = (int32_t)a.svals[j];
          if (cnt < cap) {
            int at = cnt;   // insertion into the ascending list
            while (at > 0 && list[at - 1] > q) {
              list[at] = list[at - 1];
              --at;
            }
            list[at] = q;
          }
          ++cnt;
        }
      }
  const int nw = cnt < cap ? cnt : cap;
  for (int k = 0; k < nw; ++k) a.nbr[(int64_t)k * a.nbr_stride + p] = list[k];
  a.nbr_cnt[p] = nw;
  if (cnt > cap) atomicOr(&a.scene_err[s], (uint32_t)PBDR_EBIT_NBR_OVERFLOW);
}

// With culling: every particle near another body's box is appended to
// ilist (one atomic per warp; lanes keep their order, so a warp's particles
// stay together), every other one gets an empty list.
__global__ void __launch_bounds__(128) k_interface(NbrArgs a) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  bool iface = false;
  int32_t p = 0;
  if (i < a.np) {
    p = a.pmap ? a.pmap[i] : a.pbase + i;
    const int32_t bp = a.pbody[p];
    const ScenePar sp = a.scenes[a.bodies[bp].scene];
    iface = near_other_body(a, a.Xp[p], bp, sp);
    if (!iface) a.nbr_cnt[p] = 0;
  }
  const unsigned m = __ballot_sync(0xffffffffu, iface);
  if (m == 0u) return;
  uint32_t base = 0;
  if (lane == __ffs(m) - 1) base = atomicAdd(a.icount, (uint32_t)__popc(m));
  base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
  if (iface) a.ilist[base + __popc(m & ((1u << lane) - 1u))] = p;
}

// The search: over the interface list (grid-stride, every lane busy) or,
// without culling, one thread per particle.
__global__ void __launch_bounds__(128) k_neighbors(NbrArgs a) {
  if (a.ilist) {
    const uint32_t n = *a.icount;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
      const int32_t p = a.ilist[k];
      const int32_t bp = a.pbody[p];
      const int32_t s = a.bodies[bp].scene;
      search_cells(a, p, a.Xp[p], bp, s, a.scenes[s]);
    }
    return;
  }
  // threads walk the particles in caller order: the particles of a body are
  // contiguous and close in space, so a warp's bucket lookups coincide
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.np) return;
  const int32_t p = a.pmap ? a.pmap[i] : a.pbase + i;
  const int32_t bp = a.pbody[p];
  const int32_t s = a.bodies[bp].scene;
  search_cells(a, p, a.Xp[p], bp, s, a.scenes[s]);
}


// ---------------------------------------------------------------------------
// contact corrections of one particle (Sec. III-A constraints (1), (2)):
// ground push-out by the penetration and pairwise push-out split by inverse
// mass, each with Coulomb friction removing the tangential displacement of
// this substep up to mu times the penetration.  The displacement since the
// start of the substep, x - x_init, equals v dt for every state of the solve
// (each change of x comes with the same change of v*dt), and is formed as
// v dt to avoid the cancellation of x - x_init in FP32.
// ---------------------------------------------------------------------------

__device__ __forceinline__ float3 friction_cut(float3 del, float3 n, float mu_pen) {
  const float dn = dot(del, n);
  const float3 dt_ = del - dn * n;
  const float lt = sqrtf(dot(dt_, dt_));
  if (!(lt > 0.f)) return make_float3(0.f, 0.f, 0.f);
  const float f = fminf(mu_pen / lt, 1.f);
  return f * dt_;
}

__device__ __forceinline__ float3 contact_dx_n(const IterArgs &a, const ScenePar &sp, int32_t p,
                                               float4 xp, float4 vp, int32_t cnt) {
  const float r = sp.radius, d_c = 2.f * r, mu = sp.friction, dt = sp.dt;
  const float3 n = make_float3(sp.nx, sp.ny, sp.nz);
  float3 dX = make_float3(0.f, 0.f, 0.f);
  // ground
  const float pen_g = r - (dot(n, f3(xp)) - sp.nd);
  if (pen_g > 0.f) {
    const float3 del = dt * f3(vp);
    dX = pen_g * n - friction_cut(del, n, mu * pen_g);
  }
  // particle-particle over the ascending candidate list
  float3 acc = make_float3(0.f, 0.f, 0.f);
  int active = 0;
  for (int32_t j = 0; j < cnt; ++j) {
    const int32_t q = a.nbr[(int64_t)j * a.nbr_stride + p];
    const float4 xq = a.Xin[q];
    const float3 diff = f3(xp) - f3(xq);
    const float dd = dot(diff, diff);
    if (dd > 0.f && dd < d_c * d_c) {
      const float d = sqrtf(dd);
      const float pen = d_c - d;
      const float3 nh = (1.f / d) * diff;
      const float4 vq = a.Vin[q];
      const float s = xp.w / (xp.w + xq.w);
      const float3 del = dt * (f3(vp) - f3(vq));
      acc = acc + s * (pen * nh - friction_cut(del, nh, mu * pen));
      ++active;
    }
  }
  if ((sp.flags & kContactAvg) && active > 0) acc = (1.f / (float)active) * acc;
  return dX + acc;
}

__device__ __forceinline__ float3 contact_dx(const IterArgs &a, const ScenePar &sp, int32_t p,
                                             float4 xp, float4 vp) {
  return contact_dx_n(a, sp, p, xp, vp, a.nbr_cnt[p]);
}

// ---------------------------------------------------------------------------
// one solver iteration, one body per warp
// ---------------------------------------------------------------------------

constexpr int kIterBatch = 4;   // particles per lane whose loads are issued together

__global__ void __launch_bounds__(128) k_iterate(IterArgs a) {
  const int lane = threadIdx.x & 31;
  const int32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= a.nbodies) return;
  const int32_t b = a.bmap ? a.bmap[w] : a.bbase + w;
  const BodyRec br = a.bodies[b];
  const ScenePar sp = a.scenes[br.scene];
  const int32_t p0 = br.start, pe = br.start + br.count;
  if (a.k >= sp.iterations) {   // scene needs fewer iterations: carry the state
    for (int32_t p = p0 + lane; p < pe; p += 32) {
      a.Xout[p] = a.Xin[p];
      a.Vout[p] = a.Vin[p];
    }
    return;
  }
  const float dt = sp.dt, idt = sp.inv_dt;
  const bool std_vel = (sp.flags & kStdVelocity) != 0;
  // anchor of the FP32 body sums: the body's centre of mass after the previous
  // iteration, so that x - anchor stays within the body's extent
  const float3 anc = f3(a.bcom[b]);

  // (1) contacts from X_i (Jacobi) -> X_bsm, V_bsm ; first body reduction
  float s1[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) s1[k] = 0.f;
  // Each lane takes particles p0 + lane + 32 j in order of j; the loads of
  // kIterBatch of them are issued together (X_in, V_in, Q and the list
  // lengths are read-only here), so one memory round trip covers a batch.
  for (int32_t pb = p0 + lane; pb < pe; pb += 32 * kIterBatch) {
    float4 xr[kIterBatch], vr[kIterBatch], qr[kIterBatch];
    int32_t cr[kIterBatch];
#pragma unroll
    for (int u = 0; u < kIterBatch; ++u) {
      const int32_t p = pb + 32 * u;
      if (p < pe) {
        xr[u] = __ldg(a.Xin + p);
        vr[u] = __ldg(a.Vin + p);
        qr[u] = __ldg(a.Q + p);
        cr[u] = __ldg(a.nbr_cnt + p);
      }
    }
#pragma unroll
    for (int u = 0; u < kIterBatch; ++u) {
      const int32_t p = pb + 32 * u;
      if (p >= pe) break;
      const float4 xp = xr[u], vp = vr[u];
      const float3 dX = contact_dx_n(a, sp, p, xp, vp, cr[u]);
      const float3 xb = f3(xp) + dX;
      float3 vb;
      if (std_vel)
        vb = idt * (xb - f3(a.Xinit[p]));
      else
        vb = f3(vp) + idt * dX;   // V_i + dX/dt (Sec. III-B)
      a.Xout[p] = make_float4(xb.x, xb.y, xb.z, xp.w);
      a.Vout[p] = make_float4(vb.x, vb.y, vb.z, 0.f);
      shape_terms(s1, qr[u].w, xb - anc, qr[u]);
    }
  }
#pragma unroll
  for (int k = 0; k < 12; ++k) s1[k] = warp_sum(s1[k]);

  const float iM = br.inv_mass, M = br.mass;
  float A[9];
  const float3 cA = shape_matrix(s1, iM, br.qsx, br.qsy, br.qsz, A);   // c_bsm - anchor
  const float4 qrot = shape_rotation(A, a.quat[b]);
  float R[9];
  quat_to_mat(qrot, R);

  // (2) shape-matching goals g = R q + c -> X_asm, V_asm ; the sums of the
  // momentum step (momentum_terms)
  float sm[kMomentumSums];
#pragma unroll
  for (int k = 0; k < kMomentumSums; ++k) sm[k] = 0.f;
  for (int32_t pb = p0 + lane; pb < pe; pb += 32 * kIterBatch) {
    float4 xr[kIterBatch], vr[kIterBatch], qr[kIterBatch];
#pragma unroll
    for (int u = 0; u < kIterBatch; ++u) {   // this thread's own pass-(1) results
      const int32_t p = pb + 32 * u;
      if (p < pe) {
        xr[u] = a.Xout[p];
        vr[u] = a.Vout[p];
        qr[u] = __ldg(a.Q + p);
      }
    }
#pragma unroll
    for (int u = 0; u < kIterBatch; ++u) {
      const int32_t p = pb + 32 * u;
      if (p >= pe) break;
      const float4 xb4 = xr[u], vb4 = vr[u];
      const float4 q = qr[u];
      const float m = q.w;
      const float3 grel = make_float3(R[0] * q.x + R[1] * q.y + R[2] * q.z,
                                      R[3] * q.x + R[4] * q.y + R[5] * q.z,
                                      R[6] * q.x + R[7] * q.y + R[8] * q.z) + cA;
      const float3 dsm = grel - (f3(xb4) - anc);
      const float3 xa = f3(xb4) + dsm;
      float3 va;
      if (std_vel)
        va = idt * (xa - f3(a.Xinit[p]));
      else
        va = f3(vb4) + idt * dsm;
      a.Xout[p] = make_float4(xa.x, xa.y, xa.z, xb4.w);
      a.Vout[p] = make_float4(va.x, va.y, va.z, 0.f);
      momentum_terms(sm, m, f3(xb4) - anc - cA, f3(xb4), f3(vb4), xa, va, xa - anc);
    }
  }
#pragma unroll
  for (int k = 0; k < kMomentumSums; ++k) sm[k] = warp_sum(sm[k]);

  // momentum enforcement (Sec. III-C): dv = (P_bsm - P_asm)/M,
  // w = I^-1 (L_asm - L_bsm) with I about c_asm
  float3 cA2, dv, om;
  momentum_step(sm, cA, M, iM, !(sp.flags & kNoLinMom), !(sp.flags & kNoAngMom), cA2, dv, om);

  // (3) apply the uniform corrections: v = v_asm + dv - w x r, x = x_asm + (dv - w x r) dt
  bool bad = false;
  for (int32_t pb = p0 + lane; pb < pe; pb += 32 * kIterBatch) {
    float4 xr[kIterBatch], vr[kIterBatch];
#pragma unroll
    for (int u = 0; u < kIterBatch; ++u) {
      const int32_t p = pb + 32 * u;
      if (p < pe) {
        xr[u] = a.Xout[p];
        vr[u] = a.Vout[p];
      }
    }
#pragma unroll
    for (int u = 0; u < kIterBatch; ++u) {
      const int32_t p = pb + 32 * u;
      if (p >= pe) break;
      const float4 xa4 = xr[u], va4 = vr[u];
      const float3 r = (f3(xa4) - anc) - cA2;
      const float3 corr = dv - cross(om, r);
      const float3 v = f3(va4) + corr;
      const float3 x = f3(xa4) + dt * corr;
      a.Xout[p] = make_float4(x.x, x.y, x.z, xa4.w);
      a.Vout[p] = make_float4(v.x, v.y, v.z, 0.f);
      bad |= !(isfinite(x.x) && isfinite(x.y) && isfinite(x.z));
    }
  }
  if (lane == 0) {
    a.quat[b] = qrot;
    const float3 cn = anc + cA2 + dt * dv;   // CoM after the correction
    a.bcom[b] = make_float4(cn.x, cn.y, cn.z, 0.f);
  }
  if (__any_sync(kFull, bad) && lane == 0) atomicOr(&a.scene_err[br.scene], (uint32_t)PBDR_EBIT_NONFINITE);
}

// ---------------------------------------------------------------------------
// Tangent-linear substep (forward-mode derivative of Algorithm 1).
//
// Beside the primal state (X, V) every particle carries a tangent (dX, dV):
// the derivative of its state along one direction of the initial state.
// The kernels below advance both; the primal arithmetic is k_iterate's.  The
// contact set, the neighbour lists and the sticking / sliding branch of
// every friction term are those of the primal state (their derivative is
// taken inside the branch).  The rotation's tangent follows from the polar
// decomposition A = R S: with dR = R [w]x,
//   (tr(S) I - S) w = axial(R^T dA - dA^T R)
// (S = R^T A symmetric).  The momentum correction's tangent differentiates
// dv = (P_bsm - P_asm)/M and w = I^-1 (L_asm - L_bsm), including dI.
// ---------------------------------------------------------------------------

// derivative of friction_cut(del, n, mp) along (del', n', mp')
__device__ __forceinline__ float3 friction_cut_d(float3 del, float3 del_d, float3 n, float3 n_d, float mp,
                                                 float mp_d) {
  const float dn = dot(del, n);
  const float dn_d = dot(del_d, n) + dot(del, n_d);
  const float3 t = del - dn * n;
  const float3 t_d = del_d - dn_d * n - dn * n_d;
  const float lt = sqrtf(dot(t, t));
  if (!(lt > 0.f)) return make_float3(0.f, 0.f, 0.f);
  const float f = mp / lt;
  if (!(f < 1.f)) return t_d;                     // sticking: the whole tangential step
  const float lt_d = dot(t, t_d) / lt;
  return (mp_d / lt - f * lt_d / lt) * t + f * t_d;   // sliding: mu pen along t/|t|
}

// dmu: tangent of the friction coefficient (mu pen -> mu' pen + mu pen')
__device__ __forceinline__ float3 contact_dx_d(const IterArgs &a, const TangentArgs &t, const ScenePar &sp,
                                               int32_t p, float4 xp, float4 vp, float3 xpd, float3 vpd,
                                               float dmu) {
  const float r = sp.radius, d_c = 2.f * r, mu = sp.friction, dt = sp.dt;
  const float3 n = make_float3(sp.nx, sp.ny, sp.nz);
  const float3 zero = make_float3(0.f, 0.f, 0.f);
  float3 dXd = zero;
  const float pen_g = r - (dot(n, f3(xp)) - sp.nd);
  if (pen_g > 0.f) {
    const float pen_d = -dot(n, xpd);
    dXd = pen_d * n - friction_cut_d(dt * f3(vp), dt * vpd, n, zero, mu * pen_g, mu * pen_d + dmu * pen_g);
  }
  const int32_t cnt = a.nbr_cnt[p];
  float3 acc = zero;
  int active = 0;
  for (int32_t j = 0; j < cnt; ++j) {
    const int32_t q = a.nbr[(int64_t)j * a.nbr_stride + p];
    const float4 xq = a.Xin[q];
    const float3 diff = f3(xp) - f3(xq);
    const float dd = dot(diff, diff);
    if (dd > 0.f && dd < d_c * d_c) {
      const float d = sqrtf(dd);
      const float pen = d_c - d;
      const float3 nh = (1.f / d) * diff;
      const float3 diff_d = xpd - f3(t.Xdin[q]);
      const float d_d = dot(nh, diff_d);
      const float3 nh_d = (1.f / d) * (diff_d - d_d * nh);
      const float4 vq = a.Vin[q];
      const float s = xp.w / (xp.w + xq.w);
      const float3 del = dt * (f3(vp) - f3(vq));
      const float3 del_d = dt * (vpd - f3(t.Vdin[q]));
      acc = acc + s * ((-d_d) * nh + pen * nh_d -
                       friction_cut_d(del, del_d, nh, nh_d, mu * pen, -mu * d_d + dmu * pen));
      ++active;
    }
  }
  if ((sp.flags & kContactAvg) && active > 0) acc = (1.f / (float)active) * acc;
  return dXd + acc;
}

__global__ void __launch_bounds__(256) k_predict_tangent(TangentPredictArgs a) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.np) return;
  const int32_t p = a.pmap ? a.pmap[i] : a.pbase + i;
  const ScenePar sp = a.scenes[a.bodies[a.pbody[p]].scene];
  // v~' = v' (constant external acceleration) ; x~' = x' + dt v~'
  const float3 vd = f3(a.Vd0[p]);
  const float3 xd = f3(a.Xd0[p]) + sp.dt * vd;
  a.Xdp[p] = make_float4(xd.x, xd.y, xd.z, 0.f);
  a.Vdp[p] = make_float4(vd.x, vd.y, vd.z, 0.f);
}

// one solver iteration with its tangent, one body per warp
__global__ void __launch_bounds__(128) k_iterate_tangent(IterArgs a, TangentArgs t) {
  const int lane = threadIdx.x & 31;
  const int32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= a.nbodies) return;
  const int32_t b = a.bmap ? a.bmap[w] : a.bbase + w;
  const BodyRec br = a.bodies[b];
  const ScenePar sp = a.scenes[br.scene];
  const int32_t p0 = br.start, pe = br.start + br.count;
  if (a.k >= sp.iterations) {
    for (int32_t p = p0 + lane; p < pe; p += 32) {
      a.Xout[p] = a.Xin[p];
      a.Vout[p] = a.Vin[p];
      t.Xdout[p] = t.Xdin[p];
      t.Vdout[p] = t.Vdin[p];
    }
    return;
  }
  const float dt = sp.dt, idt = sp.inv_dt;
  const float dmu = t.dmu ? t.dmu[br.scene] : 0.f;
  const float3 anc = f3(a.bcom[b]);   // a constant reference point: no tangent

  // (1) contacts -> X_bsm, V_bsm and tangents; first sums (as k_iterate),
  // P_bsm for the tangent terms, and the tangents of the sums
  float s1[12], sP[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < 12; ++k) s1[k] = 0.f;
  float tx[3] = {0.f, 0.f, 0.f}, tA[9] = {0.f}, tP[3] = {0.f, 0.f, 0.f}, tL[3] = {0.f, 0.f, 0.f};
  for (int32_t p = p0 + lane; p < pe; p += 32) {
    const float4 xp = a.Xin[p], vp = a.Vin[p];
    const float3 xpd = f3(t.Xdin[p]), vpd = f3(t.Vdin[p]);
    const float3 dX = contact_dx(a, sp, p, xp, vp);
    const float3 dXd = contact_dx_d(a, t, sp, p, xp, vp, xpd, vpd, dmu);
    const float3 xb = f3(xp) + dX;
    const float3 vb = f3(vp) + idt * dX;
    const float3 xbd = xpd + dXd;
    const float3 vbd = vpd + idt * dXd;
    a.Xout[p] = make_float4(xb.x, xb.y, xb.z, xp.w);
    a.Vout[p] = make_float4(vb.x, vb.y, vb.z, 0.f);
    t.Xdout[p] = make_float4(xbd.x, xbd.y, xbd.z, 0.f);
    t.Vdout[p] = make_float4(vbd.x, vbd.y, vbd.z, 0.f);
    const float4 q = a.Q[p];
    const float m = q.w;
    shape_terms(s1, m, xb - anc, q);
    const float3 me = m * (xb - anc);
    const float3 med = m * xbd;
    sP[0] += m * vb.x; sP[1] += m * vb.y; sP[2] += m * vb.z;
    tx[0] += med.x; tx[1] += med.y; tx[2] += med.z;
    tA[0] += med.x * q.x; tA[1] += med.x * q.y; tA[2] += med.x * q.z;
    tA[3] += med.y * q.x; tA[4] += med.y * q.y; tA[5] += med.y * q.z;
    tA[6] += med.z * q.x; tA[7] += med.z * q.y; tA[8] += med.z * q.z;
    tP[0] += m * vbd.x; tP[1] += m * vbd.y; tP[2] += m * vbd.z;
    const float3 ld = cross(med, vb) + cross(me, vbd);
    tL[0] += ld.x; tL[1] += ld.y; tL[2] += ld.z;
  }
#pragma unroll
  for (int k = 0; k < 12; ++k) s1[k] = warp_sum(s1[k]);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    sP[k] = warp_sum(sP[k]);
    tx[k] = warp_sum(tx[k]); tP[k] = warp_sum(tP[k]); tL[k] = warp_sum(tL[k]);
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) tA[k] = warp_sum(tA[k]);
  const float iM = br.inv_mass, M = br.mass;
  float A[9], Ad[9];
  const float3 cA = shape_matrix(s1, iM, br.qsx, br.qsy, br.qsz, A);
  const float3 Pb = make_float3(sP[0], sP[1], sP[2]);
  const float3 cAd = iM * make_float3(tx[0], tx[1], tx[2]);
  const float3 Pbd = make_float3(tP[0], tP[1], tP[2]);
  const float3 Lbd = make_float3(tL[0], tL[1], tL[2]) - cross(cAd, Pb) - cross(cA, Pbd);
  {
    const float qs[3] = {br.qsx, br.qsy, br.qsz};
    const float cad[3] = {cAd.x, cAd.y, cAd.z};
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) Ad[3 * r + c] = tA[3 * r + c] - cad[r] * qs[c];
  }
  const float4 qrot = shape_rotation(A, a.quat[b]);
  float R[9];
  quat_to_mat(qrot, R);
  // rotation tangent dR = R [wr]x from the polar decomposition
  float3 wr;
  {
    float S[9], W[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        S[3 * i + j] = R[i] * A[j] + R[3 + i] * A[3 + j] + R[6 + i] * A[6 + j];      // R^T A
        W[3 * i + j] = R[i] * Ad[j] + R[3 + i] * Ad[3 + j] + R[6 + i] * Ad[6 + j];   // R^T dA
      }
    const float3 ax = make_float3(W[7] - W[5], W[2] - W[6], W[3] - W[1]);   // axial(W - W^T)
    const float s01 = 0.5f * (S[1] + S[3]), s02 = 0.5f * (S[2] + S[6]), s12 = 0.5f * (S[5] + S[7]);
    const float tr = S[0] + S[4] + S[8];
    solve_sym3(tr - S[0], -s01, -s02, tr - S[4], -s12, tr - S[8], ax, wr);
  }

  // (2) goals and their tangents; the momentum sums (as k_iterate), P_asm for
  // the tangent terms, and the tangents of the second sums
  float sm[kMomentumSums], sP2[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < kMomentumSums; ++k) sm[k] = 0.f;
  float tx2[3] = {0.f, 0.f, 0.f}, tP2[3] = {0.f, 0.f, 0.f}, tL2[3] = {0.f, 0.f, 0.f}, tXX[6] = {0.f};
  for (int32_t p = p0 + lane; p < pe; p += 32) {
    const float4 xb4 = a.Xout[p], vb4 = a.Vout[p];
    const float3 xbd = f3(t.Xdout[p]), vbd = f3(t.Vdout[p]);
    const float4 q = a.Q[p];
    const float m = q.w;
    const float3 grel = make_float3(R[0] * q.x + R[1] * q.y + R[2] * q.z,
                                    R[3] * q.x + R[4] * q.y + R[5] * q.z,
                                    R[6] * q.x + R[7] * q.y + R[8] * q.z) + cA;
    const float3 dsm = grel - (f3(xb4) - anc);
    const float3 xa = f3(xb4) + dsm;
    const float3 va = f3(vb4) + idt * dsm;
    // g' = R (wr x q) + c'
    const float3 wq = cross(wr, make_float3(q.x, q.y, q.z));
    const float3 gd = make_float3(R[0] * wq.x + R[1] * wq.y + R[2] * wq.z,
                                  R[3] * wq.x + R[4] * wq.y + R[5] * wq.z,
                                  R[6] * wq.x + R[7] * wq.y + R[8] * wq.z) + cAd;
    const float3 xad = gd;
    const float3 vad = vbd + idt * (gd - xbd);
    a.Xout[p] = make_float4(xa.x, xa.y, xa.z, xb4.w);
    a.Vout[p] = make_float4(va.x, va.y, va.z, 0.f);
    t.Xdout[p] = make_float4(xad.x, xad.y, xad.z, 0.f);
    t.Vdout[p] = make_float4(vad.x, vad.y, vad.z, 0.f);
    momentum_terms(sm, m, f3(xb4) - anc - cA, f3(xb4), f3(vb4), xa, va, xa - anc);
    const float3 e = xa - anc;
    const float3 me = m * e;
    const float3 med = m * xad;
    sP2[0] += m * va.x; sP2[1] += m * va.y; sP2[2] += m * va.z;
    tx2[0] += med.x; tx2[1] += med.y; tx2[2] += med.z;
    tP2[0] += m * vad.x; tP2[1] += m * vad.y; tP2[2] += m * vad.z;
    const float3 ld = cross(med, va) + cross(me, vad);
    tL2[0] += ld.x; tL2[1] += ld.y; tL2[2] += ld.z;
    tXX[0] += 2.f * med.x * e.x; tXX[1] += med.x * e.y + me.x * xad.y; tXX[2] += med.x * e.z + me.x * xad.z;
    tXX[3] += 2.f * med.y * e.y; tXX[4] += med.y * e.z + me.y * xad.z; tXX[5] += 2.f * med.z * e.z;
  }
#pragma unroll
  for (int k = 0; k < kMomentumSums; ++k) sm[k] = warp_sum(sm[k]);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    sP2[k] = warp_sum(sP2[k]);
    tx2[k] = warp_sum(tx2[k]); tP2[k] = warp_sum(tP2[k]); tL2[k] = warp_sum(tL2[k]);
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) tXX[k] = warp_sum(tXX[k]);
  const bool linm = !(sp.flags & kNoLinMom), angm = !(sp.flags & kNoAngMom);
  float3 cA2, dv, om;
  momentum_step(sm, cA, M, iM, linm, angm, cA2, dv, om);
  const float3 Pa = make_float3(sP2[0], sP2[1], sP2[2]);
  const float3 cA2d = iM * make_float3(tx2[0], tx2[1], tx2[2]);
  const float3 Pad = make_float3(tP2[0], tP2[1], tP2[2]);
  const float3 Lad = make_float3(tL2[0], tL2[1], tL2[2]) - cross(cA2d, Pa) - cross(cA2, Pad);
  float3 dvd = make_float3(0.f, 0.f, 0.f), omd = dvd;
  if (linm) dvd = iM * (Pbd - Pad);
  if (angm) {
    float S[6];
    body_second_moment(sm, cA2, M, S);
    const float s00 = S[0], s01 = S[1], s02 = S[2], s11 = S[3], s12 = S[4], s22 = S[5];
    const float tr = __fadd_rn(__fadd_rn(s00, s11), s22);
    // dS = dSXX - M (c' c^T + c c'^T) ; dI = tr(dS) I3 - dS
    const float d00 = tXX[0] - 2.f * M * cA2d.x * cA2.x;
    const float d01 = tXX[1] - M * (cA2d.x * cA2.y + cA2.x * cA2d.y);
    const float d02 = tXX[2] - M * (cA2d.x * cA2.z + cA2.x * cA2d.z);
    const float d11 = tXX[3] - 2.f * M * cA2d.y * cA2.y;
    const float d12 = tXX[4] - M * (cA2d.y * cA2.z + cA2.y * cA2d.z);
    const float d22 = tXX[5] - 2.f * M * cA2d.z * cA2.z;
    const float dtr = d00 + d11 + d22;
    const float3 dIom = make_float3((dtr - d00) * om.x - d01 * om.y - d02 * om.z,
                                    -d01 * om.x + (dtr - d11) * om.y - d12 * om.z,
                                    -d02 * om.x - d12 * om.y + (dtr - d22) * om.z);
    solve_sym3(tr - s00, -s01, -s02, tr - s11, -s12, tr - s22, (Lad - Lbd) - dIom, omd);
  }

  // (3) corrections and their tangents
  bool bad = false;
  for (int32_t p = p0 + lane; p < pe; p += 32) {
    const float4 xa4 = a.Xout[p], va4 = a.Vout[p];
    const float3 xad = f3(t.Xdout[p]), vad = f3(t.Vdout[p]);
    const float3 r = (f3(xa4) - anc) - cA2;
    const float3 rd = xad - cA2d;
    const float3 corr = dv - cross(om, r);
    const float3 corrd = dvd - cross(omd, r) - cross(om, rd);
    const float3 v = f3(va4) + corr;
    const float3 x = f3(xa4) + dt * corr;
    const float3 vd = vad + corrd;
    const float3 xd = xad + dt * corrd;
    a.Xout[p] = make_float4(x.x, x.y, x.z, xa4.w);
    a.Vout[p] = make_float4(v.x, v.y, v.z, 0.f);
    t.Xdout[p] = make_float4(xd.x, xd.y, xd.z, 0.f);
    t.Vdout[p] = make_float4(vd.x, vd.y, vd.z, 0.f);
    bad |= !(isfinite(x.x) && isfinite(x.y) && isfinite(x.z) && isfinite(xd.x) && isfinite(xd.y) &&
             isfinite(xd.z));
  }
  if (lane == 0) {
    a.quat[b] = qrot;
    const float3 cn = anc + cA2 + dt * dv;
    a.bcom[b] = make_float4(cn.x, cn.y, cn.z, 0.f);
  }
  if (__any_sync(kFull, bad) && lane == 0) atomicOr(&a.scene_err[br.scene], (uint32_t)PBDR_EBIT_NONFINITE);
}

// ---------------------------------------------------------------------------
// Adjoint (reverse-mode derivative) of one solver iteration.
//
// k_iterate_adjoint_body (one body per warp) recomputes the iteration from
// the saved state at its start (same arithmetic as k_iterate) and takes the
// adjoint of X_{i+1}, V_{i+1} back through the momentum correction, the
// velocity update and shape matching to X_bsm, V_bsm:
//   corr = dv - w x r        ->  dv~ = sum c~,  w~ = -sum r x c~,  r~ = w x c~
//   w = I^-1 (L_asm - L_bsm) ->  y = I^-1 w~,  L~_asm = y, L~_bsm = -y,
//                                 I~ = -y w^T (through I = sum m (|r|^2 - r r^T))
//   dv = (P_bsm - P_asm)/M   ->  P~_bsm = dv~/M, P~_asm = -dv~/M
//   R = polar(A)             ->  A~ = R [z]x, (tr(S) I - S) z = axial(R^T R~ - R~^T R)
// and leaves, per particle, the direct parts of the adjoints of X_i, V_i and
// u = adjoint of the contact correction dX (X_bsm = X_i + dX, V_bsm = V_i + dX/dt).
// k_contact_adjoint (one particle per thread) adds the contact terms: for a
// pair term s_p T(x_p - x_q, v_p - v_q) of p and its mirror -s_q T(...) of q
// (T is odd), particle p gathers J^T (s_p u_p - s_q u_q) over its own
// (symmetric) list; no scatter, no atomics.  Jacobians of T and of the ground
// term are built column by column from the tangent functions above.
// ---------------------------------------------------------------------------

// weight of a particle's pair terms: 1, or 1 / (active pairs) with PBDR_CONTACT_AVG
__device__ __forceinline__ float contact_weight(const IterArgs &a, const ScenePar &sp, int32_t p, float4 xp) {
  if (!(sp.flags & kContactAvg)) return 1.f;
  const float d_c = 2.f * sp.radius;
  const int32_t cnt = a.nbr_cnt[p];
  int active = 0;
  for (int32_t j = 0; j < cnt; ++j) {
    const float3 diff = f3(xp) - f3(a.Xin[a.nbr[(int64_t)j * a.nbr_stride + p]]);
    const float dd = dot(diff, diff);
    active += (dd > 0.f && dd < d_c * d_c) ? 1 : 0;
  }
  return active > 0 ? 1.f / (float)active : 1.f;
}

__global__ void __launch_bounds__(128) k_iterate_adjoint_body(IterArgs a, AdjointArgs t) {
  const int lane = threadIdx.x & 31;
  const int32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= a.nbodies) return;
  const int32_t b = a.bmap ? a.bmap[w] : a.bbase + w;
  const BodyRec br = a.bodies[b];
  const ScenePar sp = a.scenes[br.scene];
  const int32_t p0 = br.start, pe = br.start + br.count;
  if (a.k >= sp.iterations) {   // the iteration carried the state: the adjoint passes through
    for (int32_t p = p0 + lane; p < pe; p += 32) {
      t.Xbout[p] = t.Xbin[p];
      t.Vbout[p] = t.Vbin[p];
      t.U[p] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    return;
  }
  const float dt = sp.dt, idt = sp.inv_dt;
  const float3 anc = f3(a.bcom[b]);
  const bool linm = !(sp.flags & kNoLinMom), angm = !(sp.flags & kNoAngMom);

  // ---- forward recomputation (as k_iterate) ----
  float s1[12], sP[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < 12; ++k) s1[k] = 0.f;
  for (int32_t p = p0 + lane; p < pe; p += 32) {
    const float4 xp = a.Xin[p], vp = a.Vin[p];
    const float3 dX = contact_dx(a, sp, p, xp, vp);
    const float3 xb = f3(xp) + dX;
    const float3 vb = f3(vp) + idt * dX;
    a.Xout[p] = make_float4(xb.x, xb.y, xb.z, xp.w);
    a.Vout[p] = make_float4(vb.x, vb.y, vb.z, 0.f);
    const float4 q = a.Q[p];
    const float m = q.w;
    shape_terms(s1, m, xb - anc, q);
    sP[0] += m * vb.x; sP[1] += m * vb.y; sP[2] += m * vb.z;
  }
#pragma unroll
  for (int k = 0; k < 12; ++k) s1[k] = warp_sum(s1[k]);
#pragma unroll
  for (int k = 0; k < 3; ++k) sP[k] = warp_sum(sP[k]);
  const float iM = br.inv_mass, M = br.mass;
  float A[9];
  const float3 cA = shape_matrix(s1, iM, br.qsx, br.qsy, br.qsz, A);
  const float3 Pb = make_float3(sP[0], sP[1], sP[2]);
  const float4 qrot = shape_rotation(A, a.quat[b]);
  float R[9];
  quat_to_mat(qrot, R);
  auto goal = [&](float4 q) {   // R q + c - anchor
    return make_float3(R[0] * q.x + R[1] * q.y + R[2] * q.z, R[3] * q.x + R[4] * q.y + R[5] * q.z,
                       R[6] * q.x + R[7] * q.y + R[8] * q.z) + cA;
  };
  float sm[kMomentumSums];
#pragma unroll
  for (int k = 0; k < kMomentumSums; ++k) sm[k] = 0.f;
  for (int32_t p = p0 + lane; p < pe; p += 32) {
    const float4 xb4 = a.Xout[p], vb4 = a.Vout[p];
    const float4 q = a.Q[p];
    const float m = q.w;
    const float3 grel = goal(q);
    const float3 dsm = grel - (f3(xb4) - anc);
    const float3 xa = f3(xb4) + dsm;
    const float3 va = f3(vb4) + idt * dsm;
    momentum_terms(sm, m, f3(xb4) - anc - cA, f3(xb4), f3(vb4), xa, va, xa - anc);
  }
#pragma unroll
  for (int k = 0; k < kMomentumSums; ++k) sm[k] = warp_sum(sm[k]);
  float3 cA2, dv_unused, om;
  momentum_step(sm, cA, M, iM, linm, angm, cA2, dv_unused, om);
  float S[6];
  body_second_moment(sm, cA2, M, S);
  const float s00 = S[0], s01 = S[1], s02 = S[2], s11 = S[3], s12 = S[4], s22 = S[5];
  const float trI = __fadd_rn(__fadd_rn(s00, s11), s22);

  // ---- backward: corrections -> dv~, w~ ----
  float sdv[3] = {0.f, 0.f, 0.f}, sw[3] = {0.f, 0.f, 0.f};
  for (int32_t p = p0 + lane; p < pe; p += 32) {
    const float4 xb4 = a.Xout[p];
    const float3 xa = f3(xb4) + (goal(a.Q[p]) - (f3(xb4) - anc));
    const float3 r = (xa - anc) - cA2;
    const float3 cb = f3(t.Vbin[p]) + dt * f3(t.Xbin[p]);
    sdv[0] += cb.x; sdv[1] += cb.y; sdv[2] += cb.z;
    const float3 rc = cross(r, cb);
    sw[0] -= rc.x; sw[1] -= rc.y; sw[2] -= rc.z;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    sdv[k] = warp_sum(sdv[k]);
    sw[k] = warp_sum(sw[k]);
  }
  const float3 dvb = linm ? make_float3(sdv[0], sdv[1], sdv[2]) : make_float3(0.f, 0.f, 0.f);
  float3 y = make_float3(0.f, 0.f, 0.f);
  if (angm) solve_sym3(trI - s00, -s01, -s02, trI - s11, -s12, trI - s22, make_float3(sw[0], sw[1], sw[2]), y);
  const float3 Lab = y, Lbb = make_float3(-y.x, -y.y, -y.z);
  const float yw = dot(y, om);
  // r~ of a particle (corrections, I, L_asm)
  auto rbar = [&](float3 r, float3 cb, float3 va, float m) {
    float3 rb = make_float3(0.f, 0.f, 0.f);
    if (angm) {
      rb = cross(om, cb) + m * ((-2.f * yw) * r + dot(om, r) * y + dot(y, r) * om) + m * cross(va, Lab);
    }
    return rb;
  };
  float srb[3] = {0.f, 0.f, 0.f};
  for (int32_t p = p0 + lane; p < pe; p += 32) {
    const float4 xb4 = a.Xout[p], vb4 = a.Vout[p];
    const float4 q = a.Q[p];
    const float3 dsm = goal(q) - (f3(xb4) - anc);
    const float3 xa = f3(xb4) + dsm;
    const float3 va = f3(vb4) + idt * dsm;
    const float3 r = (xa - anc) - cA2;
    const float3 cb = f3(t.Vbin[p]) + dt * f3(t.Xbin[p]);
    const float3 rb = rbar(r, cb, va, q.w);
    srb[0] += rb.x; srb[1] += rb.y; srb[2] += rb.z;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) srb[k] = warp_sum(srb[k]);
  const float3 cab = make_float3(-srb[0], -srb[1], -srb[2]);   // adjoint of c_asm
  // ---- backward: X_asm, V_asm -> goals -> R~, c~ ----
  float sRb[9] = {0.f}, scg[3] = {0.f, 0.f, 0.f};
  for (int32_t p = p0 + lane; p < pe; p += 32) {
    const float4 xb4 = a.Xout[p], vb4 = a.Vout[p];
    const float4 q = a.Q[p];
    const float m = q.w;
    const float3 dsm = goal(q) - (f3(xb4) - anc);
    const float3 xa = f3(xb4) + dsm;
    const float3 va = f3(vb4) + idt * dsm;
    const float3 r = (xa - anc) - cA2;
    const float3 xp1 = f3(t.Xbin[p]), vp1 = f3(t.Vbin[p]);
    const float3 cb = vp1 + dt * xp1;
    const float3 xab = xp1 + rbar(r, cb, va, m) + (m * iM) * cab;
    float3 vab = vp1 + (-m * iM) * dvb;
    if (angm) vab = vab + m * cross(Lab, r);
    const float3 gb = xab + idt * vab;
    sRb[0] += gb.x * q.x; sRb[1] += gb.x * q.y; sRb[2] += gb.x * q.z;
    sRb[3] += gb.y * q.x; sRb[4] += gb.y * q.y; sRb[5] += gb.y * q.z;
    sRb[6] += gb.z * q.x; sRb[7] += gb.z * q.y; sRb[8] += gb.z * q.z;
    scg[0] += gb.x; scg[1] += gb.y; scg[2] += gb.z;
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) sRb[k] = warp_sum(sRb[k]);
#pragma unroll
  for (int k = 0; k < 3; ++k) scg[k] = warp_sum(scg[k]);
  // A~ = R [z]x with (tr(S) I - S) z = axial(R^T R~ - R~^T R), S = R^T A
  float Ab[9];
  {
    float S[9], Bm[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        S[3 * i + j] = R[i] * A[j] + R[3 + i] * A[3 + j] + R[6 + i] * A[6 + j];
        Bm[3 * i + j] = R[i] * sRb[j] + R[3 + i] * sRb[3 + j] + R[6 + i] * sRb[6 + j];   // R^T R~
      }
    const float3 ax = make_float3(Bm[7] - Bm[5], Bm[2] - Bm[6], Bm[3] - Bm[1]);
    const float t01 = 0.5f * (S[1] + S[3]), t02 = 0.5f * (S[2] + S[6]), t12 = 0.5f * (S[5] + S[7]);
    const float tr = S[0] + S[4] + S[8];
    float3 z;
    solve_sym3(tr - S[0], -t01, -t02, tr - S[4], -t12, tr - S[8], ax, z);
    // [z]x = [[0,-z3,z2],[z3,0,-z1],[-z2,z1,0]] ; A~ = R [z]x
    const float Zx[9] = {0.f, -z.z, z.y, z.z, 0.f, -z.x, -z.y, z.x, 0.f};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        Ab[3 * i + j] = R[3 * i] * Zx[j] + R[3 * i + 1] * Zx[3 + j] + R[3 * i + 2] * Zx[6 + j];
  }
  // adjoint of c: from the goals and from L_bsm (through e = x_bsm - c)
  const float3 cb_tot = make_float3(scg[0], scg[1], scg[2]) - cross(Pb, Lbb);
  // ---- backward: X_bsm, V_bsm -> u = adjoint of dX; direct adjoints of X_i, V_i ----
  for (int32_t p = p0 + lane; p < pe; p += 32) {
    const float4 xb4 = a.Xout[p], vb4 = a.Vout[p];
    const float4 q = a.Q[p];
    const float m = q.w;
    const float3 dsm = goal(q) - (f3(xb4) - anc);
    const float3 xa = f3(xb4) + dsm;
    const float3 va = f3(vb4) + idt * dsm;
    const float3 r = (xa - anc) - cA2;
    const float3 xp1 = f3(t.Xbin[p]), vp1 = f3(t.Vbin[p]);
    const float3 cb = vp1 + dt * xp1;
    float3 vab = vp1 + (-m * iM) * dvb;
    if (angm) vab = vab + m * cross(Lab, r);
    const float3 e = (f3(xb4) - anc) - cA;
    const float3 Aq = make_float3(Ab[0] * q.x + Ab[1] * q.y + Ab[2] * q.z, Ab[3] * q.x + Ab[4] * q.y + Ab[5] * q.z,
                                  Ab[6] * q.x + Ab[7] * q.y + Ab[8] * q.z);
    float3 xbb = (-idt) * vab + m * Aq + (m * iM) * cb_tot;
    float3 vbb = vab + (m * iM) * dvb;
    if (angm) {
      xbb = xbb + m * cross(f3(vb4), Lbb);
      vbb = vbb + m * cross(Lbb, e);
    }
    (void)cb;
    t.Xbout[p] = make_float4(xbb.x, xbb.y, xbb.z, t.Xbin[p].w);   // w: friction adjoint, carried
    t.Vbout[p] = make_float4(vbb.x, vbb.y, vbb.z, 0.f);
    const float3 u = xbb + idt * vbb;
    t.U[p] = make_float4(u.x, u.y, u.z, contact_weight(a, sp, p, a.Xin[p]));
  }
}

// columns of the Jacobian of a pair term T(d, w) = pen n - f(dt w, n, mu pen)
// applied to a~: returns J_d^T a~ and J_w^T a~
__device__ __forceinline__ void pair_vjp(float3 diff, float3 vrel, float dc, float mu, float dt, float3 ab,
                                         float3 &gd, float3 &gw) {
  const float3 zero = make_float3(0.f, 0.f, 0.f);
  const float d = sqrtf(dot(diff, diff));
  const float pen = dc - d;
  const float3 nh = (1.f / d) * diff;
  const float3 del = dt * vrel;
  float out_d[3], out_w[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float3 ek = make_float3(k == 0 ? 1.f : 0.f, k == 1 ? 1.f : 0.f, k == 2 ? 1.f : 0.f);
    const float d_d = dot(nh, ek);
    const float3 nh_d = (1.f / d) * (ek - d_d * nh);
    const float3 Td = (-d_d) * nh + pen * nh_d - friction_cut_d(del, zero, nh, nh_d, mu * pen, -mu * d_d);
    const float3 Tw = zero - friction_cut_d(del, dt * ek, nh, zero, mu * pen, 0.f);
    out_d[k] = dot(ab, Td);
    out_w[k] = dot(ab, Tw);
  }
  gd = make_float3(out_d[0], out_d[1], out_d[2]);
  gw = make_float3(out_w[0], out_w[1], out_w[2]);
}

__global__ void __launch_bounds__(256) k_contact_adjoint(IterArgs a, AdjointArgs t, const int32_t *pbody,
                                                         const int32_t *pmap, int32_t pbase, int32_t np) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const int32_t p = pmap ? pmap[i] : pbase + i;
  const ScenePar sp = a.scenes[a.bodies[pbody[p]].scene];
  if (a.k >= sp.iterations) return;
  const float r = sp.radius, d_c = 2.f * r, mu = sp.friction, dt = sp.dt;
  const float3 n = make_float3(sp.nx, sp.ny, sp.nz);
  const float3 zero = make_float3(0.f, 0.f, 0.f);
  const float4 xp = a.Xin[p], vp = a.Vin[p];
  const float4 up4 = t.U[p];
  const float3 up = f3(up4);
  const float4 xbout = t.Xbout[p];
  float3 xb = f3(xbout), vb = f3(t.Vbout[p]);
  float mub = xbout.w;   // friction adjoint of this particle's own terms
  // ground term: J^T u column by column
  const float pen_g = r - (dot(n, f3(xp)) - sp.nd);
  if (pen_g > 0.f) {
    const float3 del = dt * f3(vp);
    float gx[3], gv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float3 ek = make_float3(k == 0 ? 1.f : 0.f, k == 1 ? 1.f : 0.f, k == 2 ? 1.f : 0.f);
      const float pen_d = -dot(n, ek);
      const float3 cx = pen_d * n - friction_cut_d(del, zero, n, zero, mu * pen_g, mu * pen_d);
      const float3 cv = zero - friction_cut_d(del, dt * ek, n, zero, mu * pen_g, 0.f);
      gx[k] = dot(up, cx);
      gv[k] = dot(up, cv);
    }
    xb = xb + make_float3(gx[0], gx[1], gx[2]);
    vb = vb + make_float3(gv[0], gv[1], gv[2]);
    // d(ground term)/d(mu) = -d f / d(mu pen) * pen
    mub += dot(up, zero - friction_cut_d(del, zero, n, zero, mu * pen_g, pen_g));
  }
  // pair terms over the symmetric list
  const int32_t cnt = a.nbr_cnt[p];
  for (int32_t j = 0; j < cnt; ++j) {
    const int32_t q = a.nbr[(int64_t)j * a.nbr_stride + p];
    const float4 xq = a.Xin[q];
    const float3 diff = f3(xp) - f3(xq);
    const float dd = dot(diff, diff);
    if (!(dd > 0.f && dd < d_c * d_c)) continue;
    const float4 uq4 = t.U[q];
    const float sw = xp.w + xq.w;
    const float3 ab = (xp.w / sw * up4.w) * up - (xq.w / sw * uq4.w) * f3(uq4);
    float3 gd, gw;
    pair_vjp(diff, f3(vp) - f3(a.Vin[q]), d_c, mu, dt, ab, gd, gw);
    xb = xb + gd;
    vb = vb + gw;
    {   // this particle's pair term s_p T: d T / d(mu) = -d f / d(mu pen) * pen
      const float d = sqrtf(dd);
      const float pen = d_c - d;
      const float3 nh = (1.f / d) * diff;
      const float3 del = dt * (f3(vp) - f3(a.Vin[q]));
      const float3 zero3 = make_float3(0.f, 0.f, 0.f);
      mub += (xp.w / sw * up4.w) * dot(up, zero3 - friction_cut_d(del, zero3, nh, zero3, mu * pen, pen));
    }
  }
  t.Xbout[p] = make_float4(xb.x, xb.y, xb.z, mub);
  t.Vbout[p] = make_float4(vb.x, vb.y, vb.z, 0.f);
}

// adjoint of the prediction: x~ = x + dt v~, v~ = v + dt g
__global__ void __launch_bounds__(256) k_predict_adjoint(TangentPredictArgs a) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.np) return;
  const int32_t p = a.pmap ? a.pmap[i] : a.pbase + i;
  const ScenePar sp = a.scenes[a.bodies[a.pbody[p]].scene];
  const float4 xb4 = a.Xd0[p];
  const float3 xb = f3(xb4);
  const float3 vb = f3(a.Vd0[p]) + sp.dt * xb;
  a.Xdp[p] = make_float4(xb.x, xb.y, xb.z, xb4.w);   // w: friction adjoint, carried
  a.Vdp[p] = make_float4(vb.x, vb.y, vb.z, 0.f);
}

// ---------------------------------------------------------------------------
// per-substep wrench accelerations: aF = F/M, alpha = I^-1 tau with c and I
// of the current positions (one body per warp, anchored FP32 sums)
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(128) k_wrench(WrenchArgs a) {
  const int lane = threadIdx.x & 31;
  const int32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= a.nb) return;
  const int32_t b = a.blist[w];
  const BodyRec br = a.bodies[b];
  const int32_t p0 = br.start, pe = br.start + br.count;
  const float3 anc = f3(a.X[p0]);
  float sx[3] = {0.f, 0.f, 0.f}, sXX[6] = {0.f};
  for (int32_t p = p0 + lane; p < pe; p += 32) {
    const float m = a.Q[p].w;
    const float3 e = f3(a.X[p]) - anc;
    const float3 me = m * e;
    sx[0] += me.x; sx[1] += me.y; sx[2] += me.z;
    sXX[0] += me.x * e.x; sXX[1] += me.x * e.y; sXX[2] += me.x * e.z;
    sXX[3] += me.y * e.y; sXX[4] += me.y * e.z; sXX[5] += me.z * e.z;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) sx[k] = warp_sum(sx[k]);
#pragma unroll
  for (int k = 0; k < 6; ++k) sXX[k] = warp_sum(sXX[k]);
  if (lane != 0) return;
  const float M = br.mass, iM = br.inv_mass;
  const float3 d = iM * make_float3(sx[0], sx[1], sx[2]);
  const float s00 = sXX[0] - M * d.x * d.x, s01 = sXX[1] - M * d.x * d.y,
              s02 = sXX[2] - M * d.x * d.z, s11 = sXX[3] - M * d.y * d.y,
              s12 = sXX[4] - M * d.y * d.z, s22 = sXX[5] - M * d.z * d.z;
  const float tr = s00 + s11 + s22;
  BodyWrench wr = a.wrench[b];
  float3 alpha;
  solve_sym3(tr - s00, -s01, -s02, tr - s11, -s12, tr - s22, f3(wr.torque), alpha);
  const float3 aF = iM * f3(wr.force);
  const float3 c = anc + d;
  wr.aF = make_float4(aF.x, aF.y, aF.z, 0.f);
  wr.alpha = make_float4(alpha.x, alpha.y, alpha.z, 0.f);
  wr.com = make_float4(c.x, c.y, c.z, 0.f);
  a.wrench[b] = wr;
}

// ---------------------------------------------------------------------------
// packing between the float4 state and caller xyz arrays (segments = scenes)
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_pack(PackArgs a, int unpack) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.total) return;
  int lo = 0, hi = a.nseg - 1;   // segment of packed index i
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.seg_off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  const int64_t p = a.seg_p0[lo] + (i - a.seg_off[lo]);
  if (!unpack) {
    if (a.hpos) {
      const float4 x = a.X[p];
      a.hpos[3 * i] = x.x; a.hpos[3 * i + 1] = x.y; a.hpos[3 * i + 2] = x.z;
    }
    if (a.hvel) {
      const float4 v = a.V[p];
      a.hvel[3 * i] = v.x; a.hvel[3 * i + 1] = v.y; a.hvel[3 * i + 2] = v.z;
    }
  } else {
    if (a.hpos) {
      float4 x = a.X[p];
      x.x = a.hpos[3 * i]; x.y = a.hpos[3 * i + 1]; x.z = a.hpos[3 * i + 2];
      a.X[p] = x;
    }
    if (a.hvel) a.V[p] = make_float4(a.hvel[3 * i], a.hvel[3 * i + 1], a.hvel[3 * i + 2], 0.f);
  }
}

// plan index -> global index over segments: map[seg_start[s] + j] = seg_base[s] + j
__global__ void __launch_bounds__(256) k_expand_map(const int32_t *seg_start, const int32_t *seg_base,
                                                    int32_t *map) {
  const int sg = blockIdx.x;
  const int32_t a = seg_start[sg], n = seg_start[sg + 1] - a, base = seg_base[sg];
  for (int32_t j = threadIdx.x; j < n; j += blockDim.x) map[a + j] = base + j;
}

inline int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

int launch_expand_map(const int32_t *seg_start, const int32_t *seg_base, int32_t nseg, int32_t *map,
                      cudaStream_t s) {
  if (nseg <= 0) return 0;
  k_expand_map<<<nseg, 256, 0, s>>>(seg_start, seg_base, map);
  return 1;
}

int launch_predict(const PredictArgs &a, cudaStream_t s) {
  if (a.np <= 0) return 0;
  k_predict<<<blocks_for(a.np, 256), 256, 0, s>>>(a);
  return 1;
}

int launch_cells(const CellArgs &a, cudaStream_t s) {
  if (a.np <= 0) return 0;
  k_cells<<<blocks_for(a.np, 256), 256, 0, s>>>(a);
  return 1;
}

int launch_body_bounds(const BoundArgs &a, cudaStream_t s) {
  if (a.nbodies <= 0) return 0;
  k_body_bounds<<<(a.nbodies + 3) / 4, 128, 0, s>>>(a);
  k_near_bodies<<<(a.nbodies + 127) / 128, 128, 0, s>>>(a);
  return 2;
}

int launch_neighbors(const NbrArgs &a, int num_sms, cudaStream_t s) {
  if (a.np <= 0) return 0;
  if (!a.ilist) {
    k_neighbors<<<blocks_for(a.np, 128), 128, 0, s>>>(a);
    return 1;
  }
  k_interface<<<blocks_for(a.np, 128), 128, 0, s>>>(a);
  // the list's length is known on the device only: a grid of 16 CTAs per SM
  // walks it
  const int grid = (int)std::min<int64_t>(blocks_for(a.np, 128), 16 * (int64_t)std::max(num_sms, 1));
  k_neighbors<<<grid, 128, 0, s>>>(a);
  return 2;
}

int launch_iterate(const IterArgs &a, int warps_per_block, cudaStream_t s) {
  if (a.nbodies <= 0) return 0;
  const int wpb = std::max(1, std::min(4, warps_per_block));
  k_iterate<<<blocks_for(a.nbodies, wpb), 32 * wpb, 0, s>>>(a);
  return 1;
}

int launch_iterate_tangent(const IterArgs &a, const TangentArgs &t, cudaStream_t s) {
  if (a.nbodies <= 0) return 0;
  k_iterate_tangent<<<blocks_for(a.nbodies, 4), 128, 0, s>>>(a, t);
  return 1;
}

int launch_iterate_adjoint(const IterArgs &a, const AdjointArgs &t, const int32_t *pbody, const int32_t *pmap,
                           int32_t pbase, int32_t np, cudaStream_t s) {
  if (a.nbodies <= 0) return 0;
  k_iterate_adjoint_body<<<blocks_for(a.nbodies, 4), 128, 0, s>>>(a, t);
  k_contact_adjoint<<<blocks_for(np, 256), 256, 0, s>>>(a, t, pbody, pmap, pbase, np);
  return 2;
}

int launch_predict_adjoint(const TangentPredictArgs &a, cudaStream_t s) {
  if (a.np <= 0) return 0;
  k_predict_adjoint<<<blocks_for(a.np, 256), 256, 0, s>>>(a);
  return 1;
}

int launch_predict_tangent(const TangentPredictArgs &a, cudaStream_t s) {
  if (a.np <= 0) return 0;
  k_predict_tangent<<<blocks_for(a.np, 256), 256, 0, s>>>(a);
  return 1;
}

int launch_wrench(const WrenchArgs &a, cudaStream_t s) {
  if (a.nb <= 0) return 0;
  k_wrench<<<blocks_for(a.nb, 4), 128, 0, s>>>(a);
  return 1;
}

int launch_pack(const PackArgs &a, int unpack, cudaStream_t s) {
  if (a.total <= 0) return 0;
  k_pack<<<blocks_for(a.total, 256), 256, 0, s>>>(a, unpack);
  return 1;
}

}  // namespace pbdr
