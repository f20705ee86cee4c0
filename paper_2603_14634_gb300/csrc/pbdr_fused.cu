// Scene-resident PBD-R substep: one CTA runs a whole substep of one scene
// (Algorithm 1: integration, neighbour build, K solver iterations) with the
// scene's positions held in shared memory, and loops over the scenes of a
// size class (persistent kernel, scenes handed out largest first).
//
// Shared memory per CTA (NCAP = particle capacity of the class):
//   Xs    float4[NCAP]  x~, then X_i; w = 1/m, negative for particles that
//                       have contact candidates
//   DXs   float4[NCAP]  contact correction dX, later x_asm (or global scratch)
//   build area, aliased with DXs while the neighbour lists are built:
//     lbody u16[N] body of every particle, slist u16 interface particles,
//     sidx u16 interface particles by bucket, start u32[T+1] buckets,
//     cand u8 per interface particle
//   V     float4[NCAP]  velocities (or in global memory)
//   partials            chunk sums (or in global memory)
// Rest offsets, neighbour lists and the per-body scratch stay in global
// memory, L2-resident while a CTA works on a scene.
//
// The neighbour lists are the same sets as the streaming form's (every pair
// within R_n by the same FP32 predicate, ascending), so the contact sums run
// in the same order.  Chunks of a body are summed in chunk order by its owner
// warp and every warp reduction is a fixed shuffle tree, so a scene's result
// depends neither on the other scenes of the launch nor on the launch shape.
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


// u16 array lengths are padded to a multiple of 8 so the next array stays 16-byte aligned
__device__ __forceinline__ int ncap_even(int n) { return (n + 7) & ~7; }
// bucket-table capacity of a class: the smallest power of two >= ncap
__host__ __device__ __forceinline__ int fused_tcap(int ncap) {
  int t = 1;
  while (t < ncap) t <<= 1;
  return t;
}

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// One step of a recursive-halving warp reduction of N values per lane over
// lane distance D: lanes with bit D clear keep values [0, H), lanes with it
// set keep [H, 2H) (indices >= N are zero), each adding its partner's copy.
// With N = 1 both partners keep the single value.
template <int N, int H, int D>
__device__ __forceinline__ void halve(float *v, int lane) {
  if (N == 1) {
    v[0] += __shfl_xor_sync(kFull, v[0], D);
    return;
  }
  const bool up = (lane & D) != 0;
#pragma unroll
  for (int k = 0; k < H; ++k) {
    const float lo = v[k];
    const float hi = (k + H < N) ? v[k + H] : 0.f;
    v[k] = (up ? hi : lo) + __shfl_xor_sync(kFull, up ? lo : hi, D);
  }
}

// index of the value whose total lane `lane` holds after warp_sums<V>, or -1
__host__ __device__ constexpr int ws_index(int V, int lane) {
  const int N0 = V, N1 = (N0 + 1) / 2, N2 = (N1 + 1) / 2, N3 = (N2 + 1) / 2, N4 = (N3 + 1) / 2,
            N5 = (N4 + 1) / 2;
  const int o4 = (N4 > 1 && (lane & 1)) ? N5 : 0, o3 = (N3 > 1 && (lane & 2)) ? N4 : 0,
            o2 = (N2 > 1 && (lane & 4)) ? N3 : 0, o1 = (N1 > 1 && (lane & 8)) ? N2 : 0,
            o0 = (N0 > 1 && (lane & 16)) ? N1 : 0;
  const int s4 = o4, s3 = s4 + o3, s2 = s3 + o2, s1 = s2 + o1, s0 = s1 + o0;
  return (s4 < N4 && s3 < N3 && s2 < N2 && s1 < N1 && s0 < N0) ? s0 : -1;
}

// a lane holding the total of value j after warp_sums<V>
__host__ __device__ constexpr int ws_lane(int V, int j) {
  int found = 0;
  for (int l = 31; l >= 0; --l)
    if (ws_index(V, l) == j) found = l;
  return found;
}

// Sums of V <= 32 values over the 32 lanes of a warp by recursive halving
// (about V shuffles instead of 5 V for one butterfly per value): afterwards
// lane l holds the total of value ws_index(V, l) in v[0].  The order of the
// additions is fixed, so the sums are deterministic.
template <int V>
__device__ __forceinline__ void warp_sums(float *v, int lane) {
  static_assert(V >= 1 && V <= 32, "one value per lane at most");
  constexpr int N0 = V, N1 = (N0 + 1) / 2, N2 = (N1 + 1) / 2, N3 = (N2 + 1) / 2, N4 = (N3 + 1) / 2,
                N5 = (N4 + 1) / 2;
  halve<N0, N1, 16>(v, lane);
  halve<N1, N2, 8>(v, lane);
  halve<N2, N3, 4>(v, lane);
  halve<N3, N4, 2>(v, lane);
  halve<N4, N5, 1>(v, lane);
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

template <bool kDxShared, bool kVShared, int kMaxThreads, int kMinBlocks>
__global__ void __launch_bounds__(kMaxThreads, kMinBlocks) k_scene_substep(FusedArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int32_t s_scene;
  __shared__ uint32_t s_wsums[32];
  float4 *Xs = reinterpret_cast<float4 *>(smem);
  float4 *DXs = kDxShared ? Xs + a.ncap : nullptr;
  unsigned char *build = reinterpret_cast<unsigned char *>(Xs + a.ncap);
  // velocities of the scene: in shared memory after the DX/build area, or global
  float4 *Vsm = kVShared ? reinterpret_cast<float4 *>(smem + a.v_off) : nullptr;
  // partial sums of the chunks: in shared memory when the scene has at most
  // ccap chunks, else in global memory
  float *part_sm = reinterpret_cast<float *>(smem + a.part_off);
  // per-body rotation and anchor table (bcap bodies)
  float4 *btab = reinterpret_cast<float4 *>(smem + a.bt_off);
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
    float4 *Vl = kVShared ? Vsm : a.V + p0;   // velocities, scene-local index
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
      Vl[i] = make_float4(vt.x, vt.y, vt.z, 0.f);
    }
    __syncthreads();   // the body passes below read x~ of particles other threads wrote

    // ---- neighbour lists ---------------------------------------------------
    // Only "interface" particles can be in a pair: p within R_n of q puts p
    // within R_n of the bounding box of q's body.  So (1) every body gets an
    // oriented bounding box of its x~ in the frame of its warm-start rotation
    // and a bounding sphere, (2) bodies whose spheres come within R_n of each
    // other are listed as near, (3) a particle is an interface particle if it
    // lies within R_n of the box of a body near its own, and (4) only interface
    // particles are hashed into the grid and searched.  All tests carry
    // margins that cover FP32 rounding, so the lists are exactly those of the
    // O(N^2) definition.
    uint16_t *lbody = reinterpret_cast<uint16_t *>(build);          // [N]
    uint16_t *slist = lbody + ncap_even(a.ncap);                     // [N] interface particles
    uint16_t *sidx = slist + ncap_even(a.ncap);                      // [|S|] sorted by bucket
    uint32_t *start = reinterpret_cast<uint32_t *>(sidx + ncap_even(a.ncap));   // [T+1]
    uint8_t *cand = reinterpret_cast<uint8_t *>(start + (a.tcap + 1));   // [|S|]
    __shared__ uint32_t s_nS;
    if (tid == 0) s_nS = 0;
    for (int bl = warp; bl < B; bl += nwarps) {
      const int32_t b = b0 + bl;
      const BodyRec br = a.bodies[b];
      const int32_t l0 = br.start - p0, l1 = l0 + br.count;
      for (int32_t i = l0 + lane; i < l1; i += 32) lbody[i] = (uint16_t)bl;
      const float3 o = f3(Xs[l0]);
      float sx = 0.f, sy = 0.f, sz = 0.f;
      for (int32_t i = l0 + lane; i < l1; i += 32) {
        const float3 e = sub(f3(Xs[i]), o);
        sx += e.x; sy += e.y; sz += e.z;
      }
      sx = wsum(sx); sy = wsum(sy); sz = wsum(sz);
      const float inv = 1.f / (float)br.count;
      const float3 cen = add(o, make_float3(sx * inv, sy * inv, sz * inv));
      float R[9];
      quat_mat(a.quat[b], R);
      float ex = 0.f, ey = 0.f, ez = 0.f;
      for (int32_t i = l0 + lane; i < l1; i += 32) {
        const float3 d = sub(f3(Xs[i]), cen);
        ex = fmaxf(ex, fabsf(R[0] * d.x + R[3] * d.y + R[6] * d.z));
        ey = fmaxf(ey, fabsf(R[1] * d.x + R[4] * d.y + R[7] * d.z));
        ez = fmaxf(ez, fabsf(R[2] * d.x + R[5] * d.y + R[8] * d.z));
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        ex = fmaxf(ex, __shfl_xor_sync(kFull, ex, off));
        ey = fmaxf(ey, __shfl_xor_sync(kFull, ey, off));
        ez = fmaxf(ez, __shfl_xor_sync(kFull, ez, off));
      }
      if (lane == 0) {
        // grow the box for the rounding of the frame change and of |R| != 1
        const float g = 1e-5f * (ex + ey + ez + fabsf(cen.x) + fabsf(cen.y) + fabsf(cen.z)) + 1e-6f;
        ex += g; ey += g; ez += g;
        const float rad = sqrtf(ex * ex + ey * ey + ez * ez) * (1.f + 1e-5f) + 1e-6f;
        float4 *bt = a.biter + (size_t)kBodyScratch * b;
        bt[9] = make_float4(cen.x, cen.y, cen.z, rad);
        bt[10] = make_float4(ex, ey, ez, 0.f);
      }
    }
    __syncthreads();
    const float reach = sqrtf(sp.Rn2) * (1.f + 1e-5f) + 1e-6f;
    // near bodies (up to kNearMax per body; more marks the body "all")
    for (int bl = tid; bl < B; bl += nt) {
      float4 *bt = a.biter + (size_t)kBodyScratch * (b0 + bl);
      const float4 sa = bt[9];
      const float ma = fabsf(sa.x) + fabsf(sa.y) + fabsf(sa.z);
      int nn = 0;
      uint16_t near[kNearMax];
      for (int bo = 0; bo < B; ++bo) {
        if (bo == bl) continue;
        const float4 sb = a.biter[(size_t)kBodyScratch * (b0 + bo) + 9];
        const float3 d = make_float3(sa.x - sb.x, sa.y - sb.y, sa.z - sb.z);
        const float lim = sa.w + sb.w + reach +
                          1e-5f * (ma + fabsf(sb.x) + fabsf(sb.y) + fabsf(sb.z) + sa.w + sb.w) + 1e-6f;
        if (dot3(d, d) <= lim * lim) {
          if (nn < kNearMax) near[nn] = (uint16_t)bo;
          ++nn;
        }
      }
      uint32_t packed[kNearMax / 2];
#pragma unroll
      for (int k = 0; k < kNearMax / 2; ++k)
        packed[k] = (2 * k < nn ? near[2 * k] : 0u) | ((2 * k + 1 < nn ? (uint32_t)near[2 * k + 1] : 0u) << 16);
      bt[11] = make_float4(__uint_as_float(packed[0]), __uint_as_float(packed[1]),
                           __uint_as_float(packed[2]), __uint_as_float(packed[3]));
      float4 e = bt[10];
      e.w = __int_as_float(nn);
      bt[10] = e;
    }
    __syncthreads();
    // interface particles -> compact list
    for (int32_t i = tid; i < N; i += nt) {
      const int32_t bl = lbody[i];
      const float4 *bt = a.biter + (size_t)kBodyScratch * (b0 + bl);
      const int nn = __float_as_int(bt[10].w);
      bool iface = nn > kNearMax;
      if (nn > 0 && !iface) {
        const float3 xp = f3(Xs[i]);
        const float4 pk = bt[11];
        const uint32_t packed[4] = {__float_as_uint(pk.x), __float_as_uint(pk.y), __float_as_uint(pk.z),
                                    __float_as_uint(pk.w)};
        for (int k = 0; k < nn && !iface; ++k) {
          const int32_t bo = (packed[k >> 1] >> (16 * (k & 1))) & 0xFFFFu;
          const int32_t gb = b0 + bo;
          const float4 *bo_t = a.biter + (size_t)kBodyScratch * gb;
          const float4 sc = bo_t[9], ext = bo_t[10];
          float R[9];
          quat_mat(a.quat[gb], R);
          const float3 d = sub(xp, f3(sc));
          const float ux = fmaxf(fabsf(R[0] * d.x + R[3] * d.y + R[6] * d.z) - ext.x, 0.f);
          const float uy = fmaxf(fabsf(R[1] * d.x + R[4] * d.y + R[7] * d.z) - ext.y, 0.f);
          const float uz = fmaxf(fabsf(R[2] * d.x + R[5] * d.y + R[8] * d.z) - ext.z, 0.f);
          const float lim = reach + 1e-5f * (fabsf(d.x) + fabsf(d.y) + fabsf(d.z)) + 1e-6f;
          iface = ux * ux + uy * uy + uz * uz <= lim * lim;
        }
      }
      if (iface) {
        const uint32_t at = atomicAdd(&s_nS, 1u);
        slist[at] = (uint16_t)i;
      } else {
        a.nbr_cnt[p0 + i] = 0;
      }
    }
    __syncthreads();
    const int32_t nS = (int32_t)s_nS;
    // bucket table of the interface grid: load factor <= 1/4 where the
    // class's shared memory allows (fewer hash collisions per search)
    uint32_t T = 1;
    while (T < (uint32_t)nS * 4u && T < (uint32_t)a.tcap) T <<= 1;
    for (uint32_t k = tid; k <= T; k += nt) start[k] = 0u;
    __syncthreads();
    for (int32_t s = tid; s < nS; s += nt) {
      const float4 x = Xs[slist[s]];
      const uint32_t key = chash(cellc(x.x, sp.inv_h), cellc(x.y, sp.inv_h), cellc(x.z, sp.inv_h)) & (T - 1u);
      atomicAdd(&start[key], 1u);
    }
    __syncthreads();
    block_scan_excl(start, (int)T + 1, s_wsums);
    for (int32_t s = tid; s < nS; s += nt) {
      const int32_t i = slist[s];
      const float4 x = Xs[i];
      const uint32_t key = chash(cellc(x.x, sp.inv_h), cellc(x.y, sp.inv_h), cellc(x.z, sp.inv_h)) & (T - 1u);
      const uint32_t at = atomicAdd(&start[key], 1u);
      sidx[at] = (uint16_t)i;
    }
    __syncthreads();
    // start[k] now holds the end of bucket k; bucket k = [start[k-1], start[k])
    const int cap = a.nbr_cap;
    for (int32_t s = tid; s < nS; s += nt) {
      const int32_t i = slist[s];
      const float3 xp = f3(Xs[i]);
      const uint16_t bp = lbody[i];
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
      cand[s] = nw > 0;
    }
    __syncthreads();
    // a negative w in shared memory marks a particle with contact candidates
    // (the list is only read for those)
    for (int32_t s = tid; s < nS; s += nt)
      if (cand[s]) Xs[slist[s]].w = -Xs[slist[s]].w;
    __syncthreads();

    // ---- K solver iterations ---------------------------------------------
    // (A) contacts per chunk, spread over all warps, each chunk writing its
    //     partial first body sums;
    // (B) one owner warp per body (bodies handed out largest first): chunk
    //     totals in chunk order -> rotation -> goals -> second sums ->
    //     momentum corrections -> X_{i+1}, V_{i+1}.
    // Every contact reads X_i before the barrier that ends (A), so the
    // owners may then overwrite positions (Jacobi order of Alg. 1).
    // Per body: the rotation (warm start) and the anchor of the FP32 sums, in
    // a shared-memory table when the scene has at most bcap bodies, else in
    // biter [0] and [6].
    const Chunk *ch = a.chunks + sp.c0;
    const bool bt_local = B <= a.bcap;
    auto rotp = [&](int32_t bl) -> float4 * {
      return bt_local ? btab + 2 * bl : a.biter + (size_t)kBodyScratch * (b0 + bl);
    };
    auto ancp = [&](int32_t bl) -> float4 * {
      return bt_local ? btab + 2 * bl + 1 : a.biter + (size_t)kBodyScratch * (b0 + bl) + 6;
    };
    const int NC = sp.nc;
    const int32_t *order = a.border + b0;
    // partial-sum slots: local chunk numbering in shared memory, or the
    // global slots of the bodies
    const bool part_local = NC <= a.ccap;
    const int32_t slot_base = a.bodies[b0].slot0;   // slots of a scene are contiguous
    for (int bl = tid; bl < B; bl += nt) {
      *rotp(bl) = a.quat[b0 + bl];
      *ancp(bl) = a.bcom[b0 + bl];
    }
    __syncthreads();
    const float r = sp.radius, dc = 2.f * r, mu = sp.friction;
    const float3 nrm = make_float3(sp.nx, sp.ny, sp.nz);
    for (int it = 0; it < sp.iterations; ++it) {
      // chunks (largest first) dealt to warps in snake order: round r goes
      // forward when r is even, backward when odd, which evens out the load
      for (int rd = 0, c = warp; c < NC; ++rd, c = rd * nwarps + ((rd & 1) ? nwarps - 1 - warp : warp)) {
        const Chunk C = ch[c];
        const BodyRec br = a.bodies[C.body];
        const float3 anc = f3(*ancp(C.body - b0));
        const int32_t l0 = C.first - p0, l1 = l0 + C.count;
        float4 q4[kChunk / 32];
#pragma unroll
        for (int j = 0; j < kChunk / 32; ++j) {
          const int32_t i = l0 + lane + 32 * j;
          if (i < l1) q4[j] = __ldg(a.Q + p0 + i);
        }
        // first sums: centroid (3) and A (9)
        float red[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) red[k] = 0.f;
#pragma unroll
        for (int j = 0; j < kChunk / 32; ++j) {
          const int32_t i = l0 + lane + 32 * j;
          if (i >= l1) continue;
          const int32_t p = p0 + i;
          const float4 xp = Xs[i];
          const float4 vp = Vl[i];
          float3 dX = make_float3(0.f, 0.f, 0.f);
          const float pen_g = r - (dot3(nrm, f3(xp)) - sp.nd);
          if (pen_g > 0.f) dX = sub(mul(pen_g, nrm), friction(mul(dt, f3(vp)), nrm, mu * pen_g));
          if (xp.w < 0.f) {   // particle with contact candidates
            const int32_t cnt = a.nbr_cnt[p];
            float3 acc = make_float3(0.f, 0.f, 0.f);
            int active = 0;
            for (int32_t jj = 0; jj < cnt; ++jj) {
              const int32_t q = a.nbr[(int64_t)jj * a.nbr_stride + p];
              const float4 xq = Xs[q - p0];
              const float3 diff = sub(f3(xp), f3(xq));
              const float dd = dot3(diff, diff);
              if (dd > 0.f && dd < dc * dc) {
                const float d = sqrtf(dd);
                const float pen = dc - d;
                const float3 nh = mul(1.f / d, diff);
                const float4 vq = Vl[q - p0];
                const float wp = fabsf(xp.w), wq = fabsf(xq.w);
                const float sw = wp / (wp + wq);
                const float3 del = mul(dt, sub(f3(vp), f3(vq)));
                acc = add(acc, mul(sw, sub(mul(pen, nh), friction(del, nh, mu * pen))));
                ++active;
              }
            }
            if ((sp.flags & kContactAvg) && active > 0) acc = mul(1.f / (float)active, acc);
            dX = add(dX, acc);
          }
          DX[i] = make_float4(dX.x, dX.y, dX.z, 0.f);
          const float3 xb = add(f3(xp), dX);   // X_bsm (V_bsm is formed by the owner)
          shape_terms(red, q4[j].w, sub(xb, anc), q4[j]);
        }
        warp_sums<12>(red, lane);
        {
          const int k = ws_index(12, lane);
          float *pt = part_local ? part_sm + kPartialFloats * (br.slot0 - slot_base + C.k)
                                 : a.partials + (size_t)kPartialFloats * (br.slot0 + C.k);
          if (k >= 0) pt[k] = red[0];
        }
      }
      __syncthreads();   // every contact of this iteration has read X_i
      for (int rd = 0, o = warp; o < B; ++rd, o = rd * nwarps + ((rd & 1) ? nwarps - 1 - warp : warp)) {
        const int32_t b = order[o];
        const BodyRec br = a.bodies[b];
        float4 *rp = rotp(b - b0), *ap = ancp(b - b0);
        const float3 anc = f3(*ap);
        // first sums: the chunks' partials in chunk order (lane j adds value j)
        float red1[12];
        {
          float mine = 0.f;
          if (lane < 12) {
            const float *pt = (part_local ? part_sm + kPartialFloats * (br.slot0 - slot_base)
                                          : a.partials + (size_t)kPartialFloats * br.slot0) + lane;
            mine = pt[0];
            for (int k = 1; k < br.nk; ++k) mine += pt[(size_t)kPartialFloats * k];
          }
#pragma unroll
          for (int j = 0; j < 12; ++j) red1[j] = __shfl_sync(kFull, mine, j);
        }
        const float M = br.mass, iM = br.inv_mass;
        float Am[9];
        const float3 cA = shape_matrix(red1, iM, br.qsx, br.qsy, br.qsz, Am);
        const float4 qrot = shape_rotation(Am, *rp);
        float R[9];
        quat_mat(qrot, R);
        // goals g = R q + c -> X_asm, V_asm; second sums
        const int32_t l0 = br.start - p0, l1 = l0 + br.count;
        // the sums of the momentum step (momentum_terms)
        float red[kMomentumSums];
#pragma unroll
        for (int k = 0; k < kMomentumSums; ++k) red[k] = 0.f;
        for (int32_t i = l0 + lane; i < l1; i += 32) {
          const int32_t p = p0 + i;
          const float4 xi = Xs[i];
          const float3 dX = f3(DX[i]);
          const float4 vi = Vl[i];
          const float4 q = __ldg(a.Q + p);
          const float m = q.w;
          const float3 xb = add(f3(xi), dX);
          float3 vb, xinit = make_float3(0.f, 0.f, 0.f);
          if (std_vel) {
            xinit = f3(a.X[p]);
            vb = mul(idt, sub(xb, xinit));
          } else {
            vb = add(f3(vi), mul(idt, dX));
          }
          const float3 grel = add(make_float3(R[0] * q.x + R[1] * q.y + R[2] * q.z,
                                              R[3] * q.x + R[4] * q.y + R[5] * q.z,
                                              R[6] * q.x + R[7] * q.y + R[8] * q.z), cA);
          const float3 dsm = sub(grel, sub(xb, anc));
          const float3 xa = add(xb, dsm);
          const float3 va = std_vel ? mul(idt, sub(xa, xinit)) : add(vb, mul(idt, dsm));
          DX[i] = make_float4(xa.x, xa.y, xa.z, 0.f);
          Vl[i] = make_float4(va.x, va.y, va.z, 0.f);
          momentum_terms(red, m, sub(sub(xb, anc), cA), xb, vb, xa, va, sub(xa, anc));
        }
        warp_sums<kMomentumSums>(red, lane);
        {
          const float t0 = red[0];
#pragma unroll
          for (int k = 0; k < kMomentumSums; ++k) red[k] = __shfl_sync(kFull, t0, ws_lane(kMomentumSums, k));
        }
        // momentum enforcement (Sec. III-C)
        float3 cA2, dv, om;
        momentum_step(red, cA, M, iM, !(sp.flags & kNoLinMom), !(sp.flags & kNoAngMom), cA2, dv, om);
        bool bad = false;
        for (int32_t i = l0 + lane; i < l1; i += 32) {
          const float3 xa = f3(DX[i]);
          const float3 va = f3(Vl[i]);
          const float3 rr = sub(sub(xa, anc), cA2);
          const float3 corr = sub(dv, cross3(om, rr));
          const float3 v = add(va, corr);
          const float3 x = add(xa, mul(dt, corr));
          Xs[i] = make_float4(x.x, x.y, x.z, Xs[i].w);
          Vl[i] = make_float4(v.x, v.y, v.z, 0.f);
          bad |= !(isfinite(x.x) && isfinite(x.y) && isfinite(x.z));
        }
        __syncwarp();
        if (lane == 0) {
          *rp = qrot;
          const float3 cn = add(add(anc, cA2), mul(dt, dv));   // CoM after the correction
          *ap = make_float4(cn.x, cn.y, cn.z, 0.f);
        }
        if (__any_sync(kFull, bad) && lane == 0) atomicOr(&a.scene_err[sid], (uint32_t)PBDR_EBIT_NONFINITE);
      }
      __syncthreads();
    }
    for (int bl = tid; bl < B; bl += nt) {
      a.quat[b0 + bl] = *rotp(bl);
      a.bcom[b0 + bl] = *ancp(bl);
    }
    // ---- write the substep's positions back ------------------------------
    for (int32_t i = tid; i < N; i += nt) {
      const float4 x = Xs[i];
      a.X[p0 + i] = make_float4(x.x, x.y, x.z, fabsf(x.w));
      if (kVShared) a.V[p0 + i] = Vl[i];
    }
    __syncthreads();
  }
}

}  // namespace

// shared-memory layout of a class: Xs | DX or build area | V | partials
FusedLayout fused_layout(int ncap, bool dx_shared, bool v_shared, bool part_shared) {
  FusedLayout L{};
  const size_t pad = ((size_t)ncap + 7) & ~(size_t)7;
  L.tcap = dx_shared ? 2 * fused_tcap(ncap) : fused_tcap(ncap);
  const size_t build = 7 * pad + 4 * ((size_t)L.tcap + 1);   // lbody, slist, sidx, cand + starts
  const size_t dxa = dx_shared ? 16 * (size_t)ncap : 0;
  size_t off = 16 * (size_t)ncap + (dxa > build ? dxa : build);
  off = (off + 15) & ~(size_t)15;
  L.v_off = v_shared ? off : 0;
  if (v_shared) off += 16 * (size_t)ncap;
  L.ccap = part_shared ? ncap / 16 : 0;
  L.part_off = off;
  off += (size_t)L.ccap * kPartialFloats * sizeof(float);
  off = (off + 15) & ~(size_t)15;
  L.bcap = kFusedBodyCap;
  L.bt_off = off;
  off += (size_t)L.bcap * 2 * sizeof(float4);
  L.bytes = off;
  return L;
}

// kernel variant for a launch: <= 256 threads with registers capped for
// three CTAs per SM, else <= 512 threads for one CTA per SM (768- and
// 1024-thread variants, registers capped at 80 / 64, measured no faster)
template <bool kDx, bool kV>
static void *variant(int threads) {
  return threads <= 256 ? (void *)k_scene_substep<kDx, kV, 256, 3> : (void *)k_scene_substep<kDx, kV, 512, 1>;
}

static void *pick(bool dx, bool v, int threads) {
  if (dx) return v ? variant<true, true>(threads) : variant<true, false>(threads);
  return v ? variant<false, true>(threads) : variant<false, false>(threads);
}

int launch_scene_substep(const FusedArgs &a, int threads, cudaStream_t s) {
  if (a.nscenes <= 0) return 0;
  const bool dxs = a.dx_scratch == nullptr;
  const size_t smem = a.smem_bytes;
  void *fn = pick(dxs, a.v_shared != 0, threads);
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  FusedArgs arg = a;
  void *params[] = {&arg};
  cudaLaunchKernel(fn, dim3(a.grid), dim3(threads), params, smem, s);
  return 1;
}

int fused_max_blocks_per_sm(int ncap, bool dx_shared, bool v_shared, int threads) {
  const size_t smem = fused_layout(ncap, dx_shared, v_shared, dx_shared).bytes;
  void *fn = pick(dx_shared, v_shared, threads);
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem);
  return nb;
}

}  // namespace pbdr
