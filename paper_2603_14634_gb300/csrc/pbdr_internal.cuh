// Internal declarations of the PBD-R sm_103a library: device-side records,
// kernel argument blocks and the host launchers each .cu file exports.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pbdr.h"

namespace pbdr {

// scene flags used by the kernels (same bits as PBDR_* in pbdr.h)
constexpr uint32_t kStdVelocity = PBDR_STD_VELOCITY;
constexpr uint32_t kNoLinMom = PBDR_NO_LINMOM;
constexpr uint32_t kNoAngMom = PBDR_NO_ANGMOM;
constexpr uint32_t kContactAvg = PBDR_CONTACT_AVG;
constexpr uint32_t kSmFromXi = PBDR_SM_FROM_XI;

// internal scene flag (not part of the ABI): the scene has a body with a wrench
constexpr uint32_t kSceneHasWrench = 1u << 16;

constexpr uint32_t kEmptyCell = 0xFFFFFFFFu;
constexpr int kFusedNbrCap = 32;    // neighbour slots per particle in the fused kernel
constexpr int kNearMax = 8;         // near bodies kept per body; more: every particle is searched
constexpr int kFusedBodyCap = 64;   // bodies per scene whose rotation / anchor sit in shared memory
constexpr int kMaxBodyParticles = 1 << 20;

// Per-scene constants, read by every kernel (one 80-byte record per scene).
struct alignas(16) ScenePar {
  float radius, friction, dt, inv_dt;
  float gx, gy, gz, Rn2;        // gravity; squared neighbour radius (FP32)
  float nx, ny, nz, nd;         // ground plane n.x = d
  float inv_h;                  // inverse cell size of the neighbour grid
  int32_t iterations;
  uint32_t flags;
  uint32_t T;                   // hash-table size (power of two)
  int32_t p0, np, b0, nb;       // global particle and body ranges
  int32_t c0, nc;               // the scene's work chunks (scene-resident kernel)
  int32_t multi_chunk_bodies;   // bodies split over more than one chunk
  int32_t pad;
};

// Per-body constants.
struct alignas(16) BodyRec {
  int32_t start, count, scene, has_wrench;
  float mass, inv_mass;
  int32_t slot0, nk;            // first partial-sum slot and number of chunks
  float qsx, qsy, qsz, pad2;    // sum_p m_p q_p (FP32 rest offsets; ~0)
};

// A chunk: up to kChunk particles of one body, processed by one warp of the
// scene-resident kernel (lane l owns particles l, l+32, ...).  The chunks of
// a scene are stored largest first; chunk k of a body covers
// [start + k*kChunk, ...) and writes partial sums to slot slot0 + k.
constexpr int kChunk = 128;
struct alignas(16) Chunk {
  int32_t body;                 // global body index
  int32_t first;                // global index of the chunk's first particle
  int32_t count;
  int32_t k;                    // index of the chunk within its body
};
constexpr int kBodyScratch = 12;    // float4 per body in FusedArgs::biter
constexpr int kPartialFloats = 12;  // floats per partial-sum slot: centroid (3), A (9)

// Per-body external wrench, set by the host (force, torque) and the
// per-substep derived accelerations (aF = F/M, alpha = I^-1 tau about c).
struct alignas(16) BodyWrench {
  float4 force;    // xyz
  float4 torque;   // xyz
  float4 aF;       // xyz: F/M
  float4 alpha;    // xyz: I^-1 tau
  float4 com;      // xyz: c at the start of the substep
};

// ---- kernel argument blocks ---------------------------------------------

struct PredictArgs {
  const float4 *X0, *V0;   // state at the start of the substep
  float4 *Xp, *Vp;         // predicted state (may alias X0/V0)
  float4 *Xinit;           // X_init copy, or nullptr
  const int32_t *pbody;
  const BodyRec *bodies;
  const ScenePar *scenes;
  const BodyWrench *wrench;
  const int32_t *pmap;     // plan particle -> global particle (nullptr: pbase + i)
  int32_t pbase, np;
  const uint32_t *hbase;   // scene -> first key of its hash range in this plan
  uint32_t *keys, *vals;   // cell key and global particle id per plan particle
  int predict;             // 0: keys of the current positions only
};

struct CellArgs {
  const uint32_t *skeys, *svals;
  const float4 *Xp;
  const int32_t *pbody;
  uint4 *cells;            // per bucket: first, end, lowest body, ~highest body
  float4 *spos;            // sorted (x, y, z, body id bits)
  int32_t np;
};

struct NbrArgs {
  const uint32_t *skeys, *svals;
  const float4 *spos;
  const float4 *Xp;        // predicted positions (caller order)
  const int32_t *pbody;
  const int32_t *pmap;     // plan particle -> global particle (nullptr: pbase + i)
  int32_t pbase;
  const uint4 *cells;
  const BodyRec *bodies;
  const ScenePar *scenes;
  const uint32_t *hbase;
  int32_t *nbr_cnt;        // [global particle]
  int32_t *nbr;            // [slot * nbr_stride + global particle]
  int64_t nbr_stride;
  int32_t cap;
  uint32_t *scene_err;
  int32_t np;
  // culling (nullptr: search every particle): per body its bounding box
  // (2 float4: centre and sphere radius, half-extents and near-body count),
  // its near bodies (kNearMax ids) and its warm-start rotation
  const float4 *bounds;
  const int32_t *near;
  const float4 *quat;
  // with culling: the particles within reach of another body (the search
  // list, global ids) and their number (zero before k_interface)
  int32_t *ilist;
  uint32_t *icount;
};

// per-body bounding boxes and near-body lists of the streaming neighbour stage
struct BoundArgs {
  const float4 *Xp;        // predicted positions
  const float4 *quat;      // warm-start rotations (box frames)
  const BodyRec *bodies;
  const ScenePar *scenes;
  const int32_t *bmap;     // plan body -> global body (nullptr: bbase + i)
  int32_t bbase, nbodies;
  float4 *bounds;          // [2 per body]
  int32_t *near;           // [kNearMax per body]
};

struct IterArgs {
  const float4 *Xin, *Vin;
  float4 *Xout, *Vout;
  const float4 *Q;         // rest offset xyz, particle mass w
  const float4 *Xinit;     // for PBDR_STD_VELOCITY, else nullptr
  const int32_t *nbr_cnt, *nbr;
  int64_t nbr_stride;
  const BodyRec *bodies;
  const ScenePar *scenes;
  float4 *quat;            // per-body rotation (warm start), updated
  float4 *bcom;            // per-body centre of mass after the last iteration, updated
  const int32_t *bmap;     // plan body -> global body (nullptr: bbase + i)
  int32_t bbase, nbodies;
  uint32_t *scene_err;
  int32_t k;               // iteration index
};

// scene-resident substep (one CTA per scene, persistent over a scene list)
struct FusedArgs {
  float4 *X, *V;           // state; X keeps x_init until the end of the substep
  const float4 *Q;
  const int32_t *pbody;
  const BodyRec *bodies;
  const ScenePar *scenes;
  BodyWrench *wrench;
  float4 *quat, *bcom;     // per-body warm start and sum anchor, updated
  float4 *biter;           // per-body scratch: kBodyScratch float4 per body
  const Chunk *chunks;     // all chunks (scenes index them through c0, nc)
  const int32_t *border;   // per scene (at b0): its bodies, largest first
  float *partials;         // kPartialFloats per slot
  float4 *dx_scratch;      // global dX / x_asm scratch, or nullptr (shared memory)
  int32_t *nbr_cnt, *nbr;
  int64_t nbr_stride;
  int32_t nbr_cap;
  uint32_t *scene_err;
  const int32_t *scene_list;   // scenes of this size class, largest first
  int32_t nscenes;
  uint32_t *ticket;        // work counter, zeroed before the launch
  int32_t ncap;            // particle capacity of the class
  int32_t grid;
  int32_t v_shared;        // velocities held in shared memory during the substep
  int32_t tcap;            // largest bucket table of the interface grid
  int32_t ccap;            // chunks whose partial sums fit in shared memory
  size_t v_off, part_off;  // shared-memory offsets of V and of the partial sums
  int32_t bcap;            // bodies whose rotation and anchor live in shared memory
  size_t bt_off;           // shared-memory offset of that table
  size_t smem_bytes;
};

// shared-memory layout of a size class of the scene-resident kernel
struct FusedLayout {
  int32_t tcap, ccap, bcap;
  size_t v_off, part_off, bt_off, bytes;
};

// Tangent (forward-mode derivative) of the streaming form: dX, dV per
// particle, double-buffered like X, V.  The neighbour lists and the branch
// of every contact and friction test are those of the primal state.
struct TangentArgs {
  const float4 *Xdin, *Vdin;
  float4 *Xdout, *Vdout;
  const float *dmu;        // per scene: tangent of the friction coefficient (nullptr: 0)
};

struct TangentPredictArgs {
  const float4 *Xd0, *Vd0; // tangents at the start of the substep
  float4 *Xdp, *Vdp;       // tangents of x~, v~ (may alias)
  const int32_t *pbody;
  const BodyRec *bodies;
  const ScenePar *scenes;
  const int32_t *pmap;
  int32_t pbase, np;
};

// Adjoint (reverse-mode derivative) of one solver iteration of the streaming
// form.  The primal inputs are the saved state at the start of the iteration
// (IterArgs::Xin/Vin, quat and bcom as they were before it); Xout/Vout serve
// as scratch for X_bsm, V_bsm.
struct AdjointArgs {
  const float4 *Xbin, *Vbin;   // adjoint of X_{i+1}, V_{i+1}; Xb.w accumulates, per
                               // particle, the adjoint of the friction coefficient
                               // over the friction terms of its own correction
  float4 *Xbout, *Vbout;       // adjoint of X_i, V_i
  float4 *U;                   // per particle: adjoint of the contact correction dX (xyz),
                               // the particle's contact weight (w)
};

struct WrenchArgs {
  const float4 *X, *Q;
  const BodyRec *bodies;
  BodyWrench *wrench;
  const int32_t *blist;
  int32_t nb;
};

struct PackArgs {
  float4 *X, *V;           // device state
  float *hpos, *hvel;      // packed xyz staging (device)
  const int32_t *seg_p0;   // per segment: first global particle
  const int64_t *seg_off;  // per segment: first packed particle (n+1 entries)
  int32_t nseg;
  int64_t total;
};

// ---- launchers (return the number of kernel launches issued) -------------

int launch_predict(const PredictArgs &a, cudaStream_t s);
int launch_cells(const CellArgs &a, cudaStream_t s);
int launch_neighbors(const NbrArgs &a, int num_sms, cudaStream_t s);
int launch_body_bounds(const BoundArgs &a, cudaStream_t s);
int launch_iterate(const IterArgs &a, int warps_per_block, cudaStream_t s);
int launch_iterate_tangent(const IterArgs &a, const TangentArgs &t, cudaStream_t s);
int launch_predict_tangent(const TangentPredictArgs &a, cudaStream_t s);
int launch_iterate_adjoint(const IterArgs &a, const AdjointArgs &t, const int32_t *pbody, const int32_t *pmap,
                           int32_t pbase, int32_t np, cudaStream_t s);
int launch_predict_adjoint(const TangentPredictArgs &a, cudaStream_t s);
int launch_wrench(const WrenchArgs &a, cudaStream_t s);
int launch_pack(const PackArgs &a, int unpack, cudaStream_t s);
int launch_expand_map(const int32_t *seg_start, const int32_t *seg_base, int32_t nseg, int32_t *map,
                      cudaStream_t s);
int launch_scene_substep(const FusedArgs &a, int threads, cudaStream_t s);
FusedLayout fused_layout(int ncap, bool dx_shared, bool v_shared, bool part_shared);
int fused_max_blocks_per_sm(int ncap, bool dx_shared, bool v_shared, int threads);

// Stable LSD radix sort of (key, value) pairs, keys < 2^bits.  Buffers:
// ka/va hold the input; kb/vb are scratch of the same size; hist holds
// radix_hist_words(n) words.  The sorted result ends in (ka, va) when the
// number of 8-bit passes is even, else in (kb, vb); *out_in_b tells which.
size_t radix_hist_words(int64_t n);
int radix_sort_pairs(uint32_t *ka, uint32_t *va, uint32_t *kb, uint32_t *vb,
                     uint32_t *hist, int64_t n, int bits, int *out_in_b,
                     cudaStream_t s);

// records the calling thread's message for pbdr_last_error(); returns code
int set_last_error(int code, const char *msg);

}  // namespace pbdr
