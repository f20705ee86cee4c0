// Scene-resident PBD-R substep: one CTA runs a whole substep of one scene
// (Algorithm 1: integration, neighbour build, K solver iterations) with the
// scene's positions held in shared memory, and loops over the scenes of a
// size class (persistent kernel, scenes handed out largest first).
//
// Shared memory per CTA (NCAP = particle capacity of the class):
//   Xs  float4[NCAP]  x (predicted, then X_i), w
//   DXs float4[NCAP]  contact correction dX_c, later x_asm   (or global scratch)
//   build area, aliased with DXs while the neighbour lists are built:
//     start u32[T'+1]  bucket counts -> starts (T' = smallest power of two >= N)
//     sidx  u16[N]     particle indices sorted by bucket
//     lbody u16[N]     body index of every particle within the scene
// Velocities, rest offsets and neighbour lists stay in global memory; within
// one CTA's processing of a scene they are L2 resident.
//
// The neighbour lists are the same sets as the streaming path's (every pair
// within R_n by the same FP32 predicate, ascending), so the contact sums run
// in the same order.  Inside a body, lane l owns particles l, l+32, ... and the
// body sums use the same shuffle tree, so a scene's result does not depend on
// which other scenes share the launch.
#include <math.h>

#include "pbdr_internal.cuh"
#include "pbdr_math.cuh"

namespace pbdr {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 add(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 sub(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 mul(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ int32_t cellc(float x, float inv_h) {
  float u = floorf(__fmul_rn(x, inv_h));
  u = fminf(fmaxf(u, -1.0e9f), 1.0e9f);
  return (int32_t)u;
}
__device__ __forceinline__ uint32_t chash(int32_t ix, int32_t iy, int32_t iz) {
  return ((uint32_t)ix * 73856093u) ^ ((uint32_t)iy * 19349663u) ^ ((uint32_t)iz * 83492791u);
}
__device__ __forceinline__ float d2rn(float3 p, float3 q) {
  float dx = __fsub_rn(q.x, p.x), dy = __fsub_rn(q.y, p.y), dz = __fsub_rn(q.z, p.z);
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ void quat_mat(float4 q, float *R) {
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

__device__ __forceinline__ float3 friction(float3 del, float3 n, float mu_pen) {
  const float dn = dot3(del, n);
  const float3 t = sub(del, mul(dn, n));
  const float lt = sqrtf(dot3(t, t));
  if (!(lt > 0.f)) return make_float3(0.f, 0.f, 0.f);
  return mul(fminf(mu_pen / lt, 1.f), t);
}

// block-wide exclusive scan of u32 a[0..m) in place (chunked per thread)
__device__ void block_scan_excl(uint32_t *a, int m, uint32_t *wsums) {
  const int nt = blockDim.x, t = threadIdx.x;
  const int chunk = (m + nt - 1) / nt;
  const int b0 = min(t * chunk, m), b1 = min(b0 + chunk, m);
  uint32_t s = 0;
  for (int i = b0; i < b1; ++i) s += a[i];
  // exclusive scan of the per-thread sums
  const int lane = t & 31, w = t >> 5, nw = nt >> 5;
  uint32_t x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsums[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t v = lane < nw ? wsums[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(kFull, v, o);
      if (lane >= o) v += y;
    }
    if (lane < nw) wsums[lane] = v;
  }
  __syncthreads();
  uint32_t run = (w > 0 ? wsums[w - 1] : 0u) + x - s;
  for (int i = b0; i < b1; ++i) {
    const uint32_t c = a[i];
    a[i] = run;
    run += c;
  }
  __syncthreads();
}

// body sums of phase A -> rotation of the shape-matching fit (Sec. III-C):
// red = [sum m e (3), sum m e q^T (9), P_bsm (3), sum m e x v (3)], e = x - a
__device__ __forceinline__ void body_rotation(const float *red, const BodyRec &br, float4 *bt,
                                              int lane) {
  const float3 cA = mul(br.inv_mass, make_float3(red[0], red[1], red[2]));
  const float3 Pb = make_float3(red[12], red[13], red[14]);
  const float3 Lb = sub(make_float3(red[15], red[16], red[17]), cross3(cA, Pb));
  float A[9];
  const float qs[3] = {br.qsx, br.qsy, br.qsz};
  const float ca[3] = {cA.x, cA.y, cA.z};
#pragma unroll
  for (int rr = 0; rr < 3; ++rr)
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) A[3 * rr + cc] = red[3 + 3 * rr + cc] - ca[rr] * qs[cc];
  const float4 qrot = shape_rotation(A, bt[0]);
  __syncwarp();
  if (lane == 0) {
    bt[0] = qrot;
    bt[1] = make_float4(cA.x, cA.y, cA.z, 0.f);
    bt[2] = make_float4(Pb.x, Pb.y, Pb.z, 0.f);
    bt[3] = make_float4(Lb.x, Lb.y, Lb.z, 0.f);
  }
}

// body sums of phase B -> momentum corrections (Eqs. lin_momentum,
// ang_momentum): red = [sum m e (3), P_asm (3), sum m e x v (3), sum m e e^T (6)]
__device__ __forceinline__ void body_momentum(const float *red, const BodyRec &br, float4 *bt,
                                              int aslot, int nslot, const ScenePar &sp, int lane) {
  const float M = br.mass, iM = br.inv_mass;
  const float3 cA2 = mul(iM, make_float3(red[0], red[1], red[2]));
  const float3 Pa = make_float3(red[3], red[4], red[5]);
  const float3 La = sub(make_float3(red[6], red[7], red[8]), cross3(cA2, Pa));
  const float3 Pb = f3(bt[2]), Lb = f3(bt[3]);
  float3 dv = make_float3(0.f, 0.f, 0.f), om = make_float3(0.f, 0.f, 0.f);
  if (!(sp.flags & kNoLinMom)) dv = mul(iM, sub(Pb, Pa));
  if (!(sp.flags & kNoAngMom)) {
    const float s00 = red[9] - M * cA2.x * cA2.x, s01 = red[10] - M * cA2.x * cA2.y,
                s02 = red[11] - M * cA2.x * cA2.z, s11 = red[12] - M * cA2.y * cA2.y,
                s12 = red[13] - M * cA2.y * cA2.z, s22 = red[14] - M * cA2.z * cA2.z;
    const float tr = s00 + s11 + s22;
    solve_sym3(tr - s00, -s01, -s02, tr - s11, -s12, tr - s22, sub(La, Lb), om);
  }
  const float3 anc = f3(bt[aslot]);
  __syncwarp();
  if (lane == 0) {
    bt[4] = make_float4(cA2.x, cA2.y, cA2.z, 0.f);
    bt[5] = make_float4(dv.x, dv.y, dv.z, 0.f);
    bt[8] = make_float4(om.x, om.y, om.z, 0.f);
    const float3 cn = add(add(anc, cA2), mul(sp.dt, dv));   // CoM after the correction
    bt[nslot] = make_float4(cn.x, cn.y, cn.z, 0.f);
  }
}

// totals of a body split over several chunks: lane j adds value j of the
// chunks' partial sums in chunk order, then every lane receives all totals
template <int NV>
__device__ __forceinline__ void sum_partials(const float *partials, const BodyRec &br, int lane,
                                             float *out) {
  float mine = 0.f;
  if (lane < NV)
    for (int k = 0; k < br.nk; ++k) mine += partials[(size_t)kPartialFloats * (br.slot0 + k) + lane];
#pragma unroll
  for (int j = 0; j < NV; ++j) out[j] = __shfl_sync(kFull, mine, j);
}

template <bool kDxShared, int kMaxThreads, int kMinBlocks>
__global__ void __launch_bounds__(kMaxThreads, kMinBlocks) k_scene_substep(FusedArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int32_t s_scene;
  __shared__ uint32_t s_wsums[32];
  float4 *Xs = reinterpret_cast<float4 *>(smem);
  float4 *DXs = kDxShared ? Xs + a.ncap : nullptr;
  unsigned char *build = reinterpret_cast<unsigned char *>(Xs + a.ncap);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;

  for (;;) {
    if (tid == 0) {
      const uint32_t i = atomicAdd(a.ticket, 1u);
      s_scene = i < (uint32_t)a.nscenes ? a.scene_list[i] : -1;
    }
    __syncthreads();
    const int32_t sid = s_scene;
    __syncthreads();
    if (sid < 0) return;
    const ScenePar sp = a.scenes[sid];
    const int32_t N = sp.np, p0 = sp.p0, B = sp.nb, b0 = sp.b0;
    if (N == 0) continue;
    const float dt = sp.dt, idt = sp.inv_dt;
    float4 *DX = kDxShared ? DXs : a.dx_scratch + p0;
    const bool std_vel = (sp.flags & kStdVelocity) != 0;

    // ---- wrench accelerations (aF = F/M, alpha = I^-1 tau about c) --------
    if (sp.flags & kSceneHasWrench) {
      for (int bl = warp; bl < B; bl += nwarps) {
        const int32_t b = b0 + bl;
        const BodyRec br = a.bodies[b];
        if (!br.has_wrench) continue;
        const float3 anc = f3(a.X[br.start]);
        float sx[3] = {0.f, 0.f, 0.f}, sXX[6] = {0.f};
        for (int32_t p = br.start + lane; p < br.start + br.count; p += 32) {
          const float m = a.Q[p].w;
          const float3 e = sub(f3(a.X[p]), anc);
          const float3 me = mul(m, e);
          sx[0] += me.x; sx[1] += me.y; sx[2] += me.z;
          sXX[0] += me.x * e.x; sXX[1] += me.x * e.y; sXX[2] += me.x * e.z;
          sXX[3] += me.y * e.y; sXX[4] += me.y * e.z; sXX[5] += me.z * e.z;
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) sx[k] = wsum(sx[k]);
#pragma unroll
        for (int k = 0; k < 6; ++k) sXX[k] = wsum(sXX[k]);
        if (lane == 0) {
          const float M = br.mass, iM = br.inv_mass;
          const float3 d = mul(iM, make_float3(sx[0], sx[1], sx[2]));
          const float s00 = sXX[0] - M * d.x * d.x, s01 = sXX[1] - M * d.x * d.y,
                      s02 = sXX[2] - M * d.x * d.z, s11 = sXX[3] - M * d.y * d.y,
                      s12 = sXX[4] - M * d.y * d.z, s22 = sXX[5] - M * d.z * d.z;
          const float tr = s00 + s11 + s22;
          BodyWrench wr = a.wrench[b];
          float3 alpha;
          solve_sym3(tr - s00, -s01, -s02, tr - s11, -s12, tr - s22, f3(wr.torque), alpha);
          const float3 aF = mul(iM, f3(wr.force));
          const float3 c = add(anc, d);
          wr.aF = make_float4(aF.x, aF.y, aF.z, 0.f);
          wr.alpha = make_float4(alpha.x, alpha.y, alpha.z, 0.f);
          wr.com = make_float4(c.x, c.y, c.z, 0.f);
          a.wrench[b] = wr;
        }
      }
      __syncthreads();
    }

    // ---- integration: x~ to shared memory, v~ to global, X keeps x_init ---
    for (int32_t i = tid; i < N; i += nt) {
      const int32_t p = p0 + i;
      const float4 x = a.X[p], v = a.V[p];
      float3 acc = make_float3(sp.gx, sp.gy, sp.gz);
      if (sp.flags & kSceneHasWrench) {
        const int32_t b = a.pbody[p];
        if (a.bodies[b].has_wrench) {
          const BodyWrench wr = a.wrench[b];
          acc = add(add(acc, f3(wr.aF)), cross3(f3(wr.alpha), sub(f3(x), f3(wr.com))));
        }
      }
      const float3 vt = add(f3(v), mul(dt, acc));
      const float3 xt = add(f3(x), mul(dt, vt));
      Xs[i] = make_float4(xt.x, xt.y, xt.z, x.w);
      a.V[p] = make_float4(vt.x, vt.y, vt.z, 0.f);
    }

    // ---- neighbour lists: counting sort of buckets in shared memory ------
    uint32_t T = 1;
    while (T < (uint32_t)N) T <<= 1;
    uint32_t *start = reinterpret_cast<uint32_t *>(build);
    uint16_t *sidx = reinterpret_cast<uint16_t *>(start + T + 1);
    uint16_t *lbody = sidx + N;
    for (uint32_t k = tid; k <= T; k += nt) start[k] = 0u;
    for (int bl = warp; bl < B; bl += nwarps) {
      const BodyRec br = a.bodies[b0 + bl];
      for (int32_t p = br.start + lane; p < br.start + br.count; p += 32)
        lbody[p - p0] = (uint16_t)bl;
    }
    // broad phase: bounding sphere of every body's x~ (slot 9 of the body
    // scratch: centre, radius grown to cover FP32 rounding)
    for (int bl = warp; bl < B; bl += nwarps) {
      const BodyRec br = a.bodies[b0 + bl];
      const int32_t l0 = br.start - p0, l1 = l0 + br.count;
      const float3 o = f3(Xs[l0]);
      float sx = 0.f, sy = 0.f, sz = 0.f;
      for (int32_t i = l0 + lane; i < l1; i += 32) {
        const float3 e = sub(f3(Xs[i]), o);
        sx += e.x; sy += e.y; sz += e.z;
      }
      sx = wsum(sx); sy = wsum(sy); sz = wsum(sz);
      const float inv = 1.f / (float)br.count;
      const float3 cen = add(o, make_float3(sx * inv, sy * inv, sz * inv));
      float r2 = 0.f;
      for (int32_t i = l0 + lane; i < l1; i += 32) {
        const float3 e = sub(f3(Xs[i]), cen);
        r2 = fmaxf(r2, dot3(e, e));
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) r2 = fmaxf(r2, __shfl_xor_sync(kFull, r2, off));
      if (lane == 0) {
        const float rad = sqrtf(r2) * (1.f + 1e-5f) + 1e-6f;
        a.biter[(size_t)kBodyScratch * (b0 + bl) + 9] = make_float4(cen.x, cen.y, cen.z, rad);
      }
    }
    __syncthreads();
    // a body needs the particle search only if another body's sphere comes
    // within the neighbour radius of its own (conservative margins)
    const float reach = sqrtf(sp.Rn2) * (1.f + 1e-5f) + 1e-6f;
    for (int bl = tid; bl < B; bl += nt) {
      const float4 sa = a.biter[(size_t)kBodyScratch * (b0 + bl) + 9];
      const float ma = fabsf(sa.x) + fabsf(sa.y) + fabsf(sa.z);
      int near = 0;
      for (int bo = 0; bo < B && !near; ++bo) {
        if (bo == bl) continue;
        const float4 sb = a.biter[(size_t)kBodyScratch * (b0 + bo) + 9];
        const float3 d = make_float3(sa.x - sb.x, sa.y - sb.y, sa.z - sb.z);
        const float lim = sa.w + sb.w + reach +
                          1e-5f * (ma + fabsf(sb.x) + fabsf(sb.y) + fabsf(sb.z) + sa.w + sb.w) + 1e-6f;
        near = dot3(d, d) <= lim * lim;
      }
      a.biter[(size_t)kBodyScratch * (b0 + bl) + 10] = make_float4(near ? 1.f : 0.f, 0.f, 0.f, 0.f);
    }
    for (int32_t i = tid; i < N; i += nt) {
      const float4 x = Xs[i];
      const uint32_t key = chash(cellc(x.x, sp.inv_h), cellc(x.y, sp.inv_h), cellc(x.z, sp.inv_h)) & (T - 1u);
      atomicAdd(&start[key], 1u);
    }
    __syncthreads();
    block_scan_excl(start, (int)T + 1, s_wsums);
    for (int32_t i = tid; i < N; i += nt) {
      const float4 x = Xs[i];
      const uint32_t key = chash(cellc(x.x, sp.inv_h), cellc(x.y, sp.inv_h), cellc(x.z, sp.inv_h)) & (T - 1u);
      const uint32_t at = atomicAdd(&start[key], 1u);
      sidx[at] = (uint16_t)i;
    }
    __syncthreads();
    // start[k] now holds the end of bucket k; bucket k = [start[k-1], start[k])
    const int cap = a.nbr_cap;
    for (int32_t i = tid; i < N; i += nt) {
      const float3 xp = f3(Xs[i]);
      const uint16_t bp = lbody[i];
      if (a.biter[(size_t)kBodyScratch * (b0 + bp) + 10].x == 0.f) {   // no other body in reach
        a.nbr_cnt[p0 + i] = 0;
        continue;
      }
      const int32_t ix = cellc(xp.x, sp.inv_h), iy = cellc(xp.y, sp.inv_h), iz = cellc(xp.z, sp.inv_h);
      int32_t list[kFusedNbrCap];
      int cnt = 0;
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            const int32_t cx = ix + dx, cy = iy + dy, cz = iz + dz;
            const uint32_t k = chash(cx, cy, cz) & (T - 1u);
            const uint32_t st = k ? start[k - 1] : 0u, en = start[k];
            for (uint32_t j = st; j < en; ++j) {
              const int32_t q = sidx[j];
              if (lbody[q] == bp) continue;
              const float3 xq = f3(Xs[q]);
              if (cellc(xq.x, sp.inv_h) != cx || cellc(xq.y, sp.inv_h) != cy || cellc(xq.z, sp.inv_h) != cz)
                continue;
              if (!(d2rn(xp, xq) < sp.Rn2)) continue;
              if (cnt < cap) {
                int at = cnt;
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
      for (int k = 0; k < nw; ++k) a.nbr[(int64_t)k * a.nbr_stride + p0 + i] = p0 + list[k];
      a.nbr_cnt[p0 + i] = nw;
      if (cnt > cap) atomicOr(&a.scene_err[sid], (uint32_t)PBDR_EBIT_NBR_OVERFLOW);
    }
    __syncthreads();

    // ---- K solver iterations over chunks ------------------------------------
    // biter per body: [0] rotation, [1] c_bsm - a, [2] P_bsm, [3] L_bsm,
    // [4] c_asm - a, [5] dv, [6]/[7] the anchor a of even/odd iterations,
    // [8] w.  Anchors alternate so that a body's next anchor can be written
    // while its chunks still use the current one.
    const Chunk *ch = a.chunks + sp.c0;
    const int NC = sp.nc;
    const bool multi = sp.multi_chunk_bodies > 0;
    for (int bl = tid; bl < B; bl += nt) {
      float4 *bt = a.biter + (size_t)kBodyScratch * (b0 + bl);
      bt[0] = a.quat[b0 + bl];
      bt[6] = a.bcom[b0 + bl];
    }
    __syncthreads();
    const float r = sp.radius, dc = 2.f * r, mu = sp.friction;
    const float3 nrm = make_float3(sp.nx, sp.ny, sp.nz);
    for (int it = 0; it < sp.iterations; ++it) {
      const int aslot = 6 + (it & 1), nslot = 6 + ((it + 1) & 1);
      // (A) contacts from X_i (Jacobi) and the first body sums, per chunk
      for (int c = warp; c < NC; c += nwarps) {
        const Chunk C = ch[c];
        const BodyRec br = a.bodies[C.body];
        float4 *bt = a.biter + (size_t)kBodyScratch * C.body;
        const float3 anc = f3(bt[aslot]);
        float red[18];
#pragma unroll
        for (int k = 0; k < 18; ++k) red[k] = 0.f;
        const int32_t l0 = C.first - p0, l1 = l0 + C.count;
        for (int32_t i = l0 + lane; i < l1; i += 32) {
          const int32_t p = p0 + i;
          const float4 xp = Xs[i];
          const float4 vp = a.V[p];
          float3 dX = make_float3(0.f, 0.f, 0.f);
          const float pen_g = r - (dot3(nrm, f3(xp)) - sp.nd);
          if (pen_g > 0.f) dX = sub(mul(pen_g, nrm), friction(mul(dt, f3(vp)), nrm, mu * pen_g));
          const int32_t cnt = a.nbr_cnt[p];
          float3 acc = make_float3(0.f, 0.f, 0.f);
          int active = 0;
          for (int32_t j = 0; j < cnt; ++j) {
            const int32_t q = a.nbr[(int64_t)j * a.nbr_stride + p];
            const float4 xq = Xs[q - p0];
            const float3 diff = sub(f3(xp), f3(xq));
            const float dd = dot3(diff, diff);
            if (dd > 0.f && dd < dc * dc) {
              const float d = sqrtf(dd);
              const float pen = dc - d;
              const float3 nh = mul(1.f / d, diff);
              const float4 vq = a.V[q];
              const float sw = xp.w / (xp.w + xq.w);
              const float3 del = mul(dt, sub(f3(vp), f3(vq)));
              acc = add(acc, mul(sw, sub(mul(pen, nh), friction(del, nh, mu * pen))));
              ++active;
            }
          }
          if ((sp.flags & kContactAvg) && active > 0) acc = mul(1.f / (float)active, acc);
          dX = add(dX, acc);
          DX[i] = make_float4(dX.x, dX.y, dX.z, 0.f);
          const float3 xb = add(f3(xp), dX);
          const float3 vb = std_vel ? mul(idt, sub(xb, f3(a.X[p]))) : add(f3(vp), mul(idt, dX));
          const float4 q = a.Q[p];
          const float m = q.w;
          const float3 e = sub(xb, anc);
          const float3 me = mul(m, e);
          red[0] += me.x; red[1] += me.y; red[2] += me.z;
          red[3] += me.x * q.x; red[4] += me.x * q.y; red[5] += me.x * q.z;
          red[6] += me.y * q.x; red[7] += me.y * q.y; red[8] += me.y * q.z;
          red[9] += me.z * q.x; red[10] += me.z * q.y; red[11] += me.z * q.z;
          red[12] += m * vb.x; red[13] += m * vb.y; red[14] += m * vb.z;
          const float3 l = cross3(me, vb);
          red[15] += l.x; red[16] += l.y; red[17] += l.z;
        }
#pragma unroll
        for (int k = 0; k < 18; ++k) red[k] = wsum(red[k]);
        if (br.nk == 1) {
          body_rotation(red, br, bt, lane);
        } else if (lane == 0) {
          float *pt = a.partials + (size_t)kPartialFloats * (br.slot0 + C.k);
#pragma unroll
          for (int k = 0; k < 18; ++k) pt[k] = red[k];
        }
      }
      __syncthreads();
      if (multi) {   // bodies split over several chunks: sum the chunk partials in chunk order
        for (int bl = warp; bl < B; bl += nwarps) {
          const BodyRec br = a.bodies[b0 + bl];
          if (br.nk <= 1) continue;
          float red[18];
          sum_partials<18>(a.partials, br, lane, red);
          body_rotation(red, br, a.biter + (size_t)kBodyScratch * (b0 + bl), lane);
        }
        __syncthreads();
      }
      // (B) shape-matching goals g = R q + c -> X_asm, V_asm and the second sums
      for (int c = warp; c < NC; c += nwarps) {
        const Chunk C = ch[c];
        const BodyRec br = a.bodies[C.body];
        float4 *bt = a.biter + (size_t)kBodyScratch * C.body;
        const float3 anc = f3(bt[aslot]);
        float R[9];
        quat_mat(bt[0], R);
        const float3 cA = f3(bt[1]);
        float red[15];
#pragma unroll
        for (int k = 0; k < 15; ++k) red[k] = 0.f;
        const int32_t l0 = C.first - p0, l1 = l0 + C.count;
        for (int32_t i = l0 + lane; i < l1; i += 32) {
          const int32_t p = p0 + i;
          const float4 xi = Xs[i];
          const float3 dX = f3(DX[i]);
          const float4 vi = a.V[p];
          const float4 q = a.Q[p];
          const float m = q.w;
          const float3 xb = add(f3(xi), dX);
          const float3 vb = std_vel ? mul(idt, sub(xb, f3(a.X[p]))) : add(f3(vi), mul(idt, dX));
          const float3 grel = add(make_float3(R[0] * q.x + R[1] * q.y + R[2] * q.z,
                                              R[3] * q.x + R[4] * q.y + R[5] * q.z,
                                              R[6] * q.x + R[7] * q.y + R[8] * q.z), cA);
          const float3 dsm = sub(grel, sub(xb, anc));
          const float3 xa = add(xb, dsm);
          const float3 va = std_vel ? mul(idt, sub(xa, f3(a.X[p]))) : add(vb, mul(idt, dsm));
          DX[i] = make_float4(xa.x, xa.y, xa.z, 0.f);
          a.V[p] = make_float4(va.x, va.y, va.z, 0.f);
          const float3 e = sub(xa, anc);
          const float3 me = mul(m, e);
          red[0] += me.x; red[1] += me.y; red[2] += me.z;
          red[3] += m * va.x; red[4] += m * va.y; red[5] += m * va.z;
          const float3 l = cross3(me, va);
          red[6] += l.x; red[7] += l.y; red[8] += l.z;
          red[9] += me.x * e.x; red[10] += me.x * e.y; red[11] += me.x * e.z;
          red[12] += me.y * e.y; red[13] += me.y * e.z; red[14] += me.z * e.z;
        }
#pragma unroll
        for (int k = 0; k < 15; ++k) red[k] = wsum(red[k]);
        if (br.nk == 1) {
          body_momentum(red, br, bt, aslot, nslot, sp, lane);
        } else if (lane == 0) {
          float *pt = a.partials + (size_t)kPartialFloats * (br.slot0 + C.k);
#pragma unroll
          for (int k = 0; k < 15; ++k) pt[k] = red[k];
        }
      }
      __syncthreads();
      if (multi) {
        for (int bl = warp; bl < B; bl += nwarps) {
          const BodyRec br = a.bodies[b0 + bl];
          if (br.nk <= 1) continue;
          float red[15];
          sum_partials<15>(a.partials, br, lane, red);
          body_momentum(red, br, a.biter + (size_t)kBodyScratch * (b0 + bl), aslot, nslot, sp, lane);
        }
        __syncthreads();
      }
      // (C) uniform corrections: v = v_asm + dv - w x r, x = x_asm + (dv - w x r) dt
      for (int c = warp; c < NC; c += nwarps) {
        const Chunk C = ch[c];
        const float4 *bt = a.biter + (size_t)kBodyScratch * C.body;
        const float3 anc = f3(bt[aslot]);
        const float3 cA2 = f3(bt[4]), dv = f3(bt[5]), om = f3(bt[8]);
        bool bad = false;
        const int32_t l0 = C.first - p0, l1 = l0 + C.count;
        for (int32_t i = l0 + lane; i < l1; i += 32) {
          const int32_t p = p0 + i;
          const float3 xa = f3(DX[i]);
          const float3 va = f3(a.V[p]);
          const float3 rr = sub(sub(xa, anc), cA2);
          const float3 corr = sub(dv, cross3(om, rr));
          const float3 v = add(va, corr);
          const float3 x = add(xa, mul(dt, corr));
          Xs[i] = make_float4(x.x, x.y, x.z, Xs[i].w);
          a.V[p] = make_float4(v.x, v.y, v.z, 0.f);
          bad |= !(isfinite(x.x) && isfinite(x.y) && isfinite(x.z));
        }
        if (__any_sync(kFull, bad) && lane == 0) atomicOr(&a.scene_err[sid], (uint32_t)PBDR_EBIT_NONFINITE);
      }
      __syncthreads();
    }
    for (int bl = tid; bl < B; bl += nt) {
      const float4 *bt = a.biter + (size_t)kBodyScratch * (b0 + bl);
      a.quat[b0 + bl] = bt[0];
      a.bcom[b0 + bl] = bt[6 + (sp.iterations & 1)];
    }
    // ---- write the substep's positions back ------------------------------
    for (int32_t i = tid; i < N; i += nt) a.X[p0 + i] = Xs[i];
    __syncthreads();
  }
}

}  // namespace

size_t fused_smem_bytes(int ncap, bool dx_shared) {
  // X (16 B) + max(DX 16 B, build area) per particle
  size_t build = 4 * ((size_t)2 * ncap + 1) + 4 * (size_t)ncap;   // start[T'+1] + sidx + lbody
  size_t dxa = dx_shared ? 16 * (size_t)ncap : 0;
  return 16 * (size_t)ncap + (dxa > build ? dxa : build);
}

// kernel variant for a launch: <= 256 threads with registers capped for
// three CTAs per SM, else <= 512 threads for one CTA per SM
template <bool kDx>
static void *variant(int threads) {
  return threads <= 256 ? (void *)k_scene_substep<kDx, 256, 3> : (void *)k_scene_substep<kDx, 512, 1>;
}

int launch_scene_substep(const FusedArgs &a, int threads, cudaStream_t s) {
  if (a.nscenes <= 0) return 0;
  const bool dxs = a.dx_scratch == nullptr;
  const size_t smem = fused_smem_bytes(a.ncap, dxs);
  void *fn = dxs ? variant<true>(threads) : variant<false>(threads);
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  FusedArgs arg = a;
  void *params[] = {&arg};
  cudaLaunchKernel(fn, dim3(a.grid), dim3(threads), params, smem, s);
  return 1;
}

int fused_max_blocks_per_sm(int ncap, bool dx_shared, int threads) {
  const size_t smem = fused_smem_bytes(ncap, dx_shared);
  void *fn = dx_shared ? variant<true>(threads) : variant<false>(threads);
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem);
  return nb;
}

}  // namespace pbdr
