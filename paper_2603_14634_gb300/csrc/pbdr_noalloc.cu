// Allocation-free variant of the neighbour stage for one scene.
//
// Some callers may not allocate device memory themselves: a host framework
// that owns all device memory through its own pool or a pre-reserved arena,
// or a control loop with a hard latency budget in which a cudaMalloc could
// stall.  pbdr_neighbors_noalloc serves them: it takes the caller's device
// buffers for inputs and outputs and keeps every intermediate (sort keys and
// values, radix histograms, bucket ranges, sorted positions) in one
// file-scope __device__ array of fixed size, sized for scenes of up to
// kNoAllocMaxParticles particles.  Every GPU that loads the library holds
// that array until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "pbdr_internal.cuh"

namespace pbdr {
namespace {

constexpr int32_t kNoAllocMaxParticles = 65536;
constexpr int64_t kNoAllocMaxTable = 2 * (int64_t)kNoAllocMaxParticles;   // smallest pow2 >= 2N
constexpr int kNoAllocMaxCap = 64;

// scratch layout (byte offsets, every part 256-byte aligned)
constexpr size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }
constexpr size_t kOffKeysA = 0;
constexpr size_t kOffValsA = align256(kOffKeysA + 4 * (size_t)kNoAllocMaxParticles);
constexpr size_t kOffKeysB = align256(kOffValsA + 4 * (size_t)kNoAllocMaxParticles);
constexpr size_t kOffValsB = align256(kOffKeysB + 4 * (size_t)kNoAllocMaxParticles);
constexpr size_t kOffSpos = align256(kOffValsB + 4 * (size_t)kNoAllocMaxParticles);
constexpr size_t kOffCstart = align256(kOffSpos + 16 * (size_t)kNoAllocMaxParticles);
constexpr size_t kOffCend = align256(kOffCstart + 4 * (size_t)kNoAllocMaxTable);
constexpr size_t kOffHist = align256(kOffCend + 4 * (size_t)kNoAllocMaxTable);
// radix histogram: 256 digits x 16 tiles of 4096 keys, plus scan partials
constexpr size_t kHistWords = 256 * ((kNoAllocMaxParticles + 4095) / 4096) + 1024;
constexpr size_t kScratchBytes = align256(kOffHist + 4 * kHistWords);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// per-device address of g_noalloc_scratch (host code may not use the symbol
// itself as a device address)
std::mutex g_mu;
void *g_scratch_addr[128] = {nullptr};

__device__ __forceinline__ int32_t na_cell(float x, float inv_h) {
  float u = floorf(__fmul_rn(x, inv_h));
  u = fminf(fmaxf(u, -1.0e9f), 1.0e9f);
  return (int32_t)u;
}

__device__ __forceinline__ uint32_t na_hash(int32_t ix, int32_t iy, int32_t iz) {
  return ((uint32_t)ix * 73856093u) ^ ((uint32_t)iy * 19349663u) ^ ((uint32_t)iz * 83492791u);
}

__global__ void k_na_keys(const float *__restrict__ pos, int32_t n, float inv_h, uint32_t T,
                          uint32_t *__restrict__ keys, uint32_t *__restrict__ vals) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t h = na_hash(na_cell(pos[3 * i], inv_h), na_cell(pos[3 * i + 1], inv_h),
                             na_cell(pos[3 * i + 2], inv_h));
  keys[i] = h & (T - 1u);
  vals[i] = (uint32_t)i;
}

__global__ void k_na_cells(const uint32_t *__restrict__ skeys, const uint32_t *__restrict__ svals,
                           const float *__restrict__ pos, const int32_t *__restrict__ body,
                           int32_t n, uint32_t *__restrict__ cstart, uint32_t *__restrict__ cend,
                           float4 *__restrict__ spos) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t key = skeys[i];
  if (i == 0 || skeys[i - 1] != key) cstart[key] = (uint32_t)i;
  if (i == n - 1 || skeys[i + 1] != key) cend[key] = (uint32_t)(i + 1);
  const uint32_t p = svals[i];
  spos[i] = make_float4(pos[3 * p], pos[3 * p + 1], pos[3 * p + 2], __int_as_float(body[p]));
}

__global__ void k_na_neighbors(const float *__restrict__ pos, const int32_t *__restrict__ body,
                               int32_t n, float inv_h, float Rn2, uint32_t T,
                               const uint32_t *__restrict__ svals,
                               const uint32_t *__restrict__ cstart,
                               const uint32_t *__restrict__ cend,
                               const float4 *__restrict__ spos, int32_t *__restrict__ nbr_cnt,
                               int32_t *__restrict__ nbr, int32_t cap) {
  const int32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const float px = pos[3 * p], py = pos[3 * p + 1], pz = pos[3 * p + 2];
  const int32_t bp = body[p];
  const int32_t ix = na_cell(px, inv_h), iy = na_cell(py, inv_h), iz = na_cell(pz, inv_h);
  int32_t list[kNoAllocMaxCap];
  int cnt = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int32_t cx = ix + dx, cy = iy + dy, cz = iz + dz;
        const uint32_t bkt = na_hash(cx, cy, cz) & (T - 1u);
        const uint32_t st = cstart[bkt];
        if (st == kEmptyCell) continue;
        const uint32_t en = cend[bkt];
        for (uint32_t j = st; j < en; ++j) {
          const float4 xq = spos[j];
          if (__float_as_int(xq.w) == bp) continue;
          if (na_cell(xq.x, inv_h) != cx || na_cell(xq.y, inv_h) != cy || na_cell(xq.z, inv_h) != cz)
            continue;
          const float ddx = __fsub_rn(xq.x, px), ddy = __fsub_rn(xq.y, py), ddz = __fsub_rn(xq.z, pz);
          const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(ddx, ddx), __fmul_rn(ddy, ddy)), __fmul_rn(ddz, ddz));
          if (!(d2 < Rn2)) continue;
          const int32_t q = (int32_t)svals[j];
          // keep the cap lowest indices, ascending: a full list drops its largest
          if (cnt < cap || q < list[cap - 1]) {
            int at = cnt < cap ? cnt : cap - 1;
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
  for (int k = 0; k < nw; ++k) nbr[(int64_t)k * n + p] = list[k];
  nbr_cnt[p] = cnt;
}

int na_fail(int code, const std::string &m) { return set_last_error(code, m.c_str()); }

}  // namespace
}  // namespace pbdr

using namespace pbdr;

extern "C" int pbdr_neighbors_noalloc(const float *pos, const int32_t *body, int32_t n,
                                      float radius, uint32_t *sorted_key, uint32_t *sorted_id,
                                      int32_t *nbr_cnt, int32_t *nbr, int32_t cap, void *stream) {
  if (n < 0 || n > kNoAllocMaxParticles)
    return na_fail(PBDR_ERR_INVALID, "pbdr_neighbors_noalloc: n = " + std::to_string(n) +
                                         " is outside 0.." + std::to_string(kNoAllocMaxParticles));
  if (cap < 1 || cap > kNoAllocMaxCap)
    return na_fail(PBDR_ERR_INVALID, "pbdr_neighbors_noalloc: cap must be in 1..64");
  if (!(radius > 0.f)) return na_fail(PBDR_ERR_INVALID, "pbdr_neighbors_noalloc: radius must be > 0");
  if (n > 0 && (!pos || !body || !sorted_key || !sorted_id || !nbr_cnt || !nbr))
    return na_fail(PBDR_ERR_INVALID, "pbdr_neighbors_noalloc: NULL buffer");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(PBDR_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 128) return na_fail(PBDR_ERR_INVALID, "pbdr_neighbors_noalloc: device index out of range");
  unsigned char *base = nullptr;
  {
    // set-up, once per device, with that device current
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
      void *ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr)
        return na_fail(PBDR_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_addr[dev] = ptr;
    }
    base = static_cast<unsigned char *>(g_scratch_addr[dev]);
  }
  set_last_error(PBDR_OK, "");
  if (n == 0) return PBDR_OK;
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t *ka = reinterpret_cast<uint32_t *>(base + kOffKeysA);
  uint32_t *va = reinterpret_cast<uint32_t *>(base + kOffValsA);
  uint32_t *kb = reinterpret_cast<uint32_t *>(base + kOffKeysB);
  uint32_t *vb = reinterpret_cast<uint32_t *>(base + kOffValsB);
  float4 *spos = reinterpret_cast<float4 *>(base + kOffSpos);
  uint32_t *cstart = reinterpret_cast<uint32_t *>(base + kOffCstart);
  uint32_t *cend = reinterpret_cast<uint32_t *>(base + kOffCend);
  uint32_t *hist = reinterpret_cast<uint32_t *>(base + kOffHist);
  // FP32 grid constants of the neighbour search (same definitions as pbdr_create_scene)
  const float Rn = (float)(2.2 * (double)radius);
  const float h = (float)((double)Rn * (1.0 + 1.0 / 1024.0));
  volatile float rr = Rn * Rn;
  const float Rn2 = rr;
  const float inv_h = (float)(1.0 / (double)h);
  uint32_t T = 1;
  while (T < 2u * (uint32_t)n) T <<= 1;
  int bits = 1;
  while ((1u << bits) < T) ++bits;
  if (radix_hist_words(n) > kHistWords) return na_fail(PBDR_ERR_INVALID, "pbdr_neighbors_noalloc: histogram too small");
  // the bucket starts of the previous call must not leak into this one
  e = cudaMemsetAsync(cstart, 0xFF, (size_t)T * 4, s);
  if (e != cudaSuccess) return na_fail(PBDR_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  const int tb = 256, nb = (n + tb - 1) / tb;
  k_na_keys<<<nb, tb, 0, s>>>(pos, n, inv_h, T, ka, va);
  int in_b = 0;
  radix_sort_pairs(ka, va, kb, vb, hist, n, bits, &in_b, s);
  const uint32_t *sk = in_b ? kb : ka;
  const uint32_t *sv = in_b ? vb : va;
  k_na_cells<<<nb, tb, 0, s>>>(sk, sv, pos, body, n, cstart, cend, spos);
  k_na_neighbors<<<(n + 127) / 128, 128, 0, s>>>(pos, body, n, inv_h, Rn2, T, sv, cstart, cend, spos,
                                                 nbr_cnt, nbr, cap);
  e = cudaMemcpyAsync(sorted_key, sk, (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sorted_id, sv, (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(PBDR_ERR_CUDA, std::string("pbdr_neighbors_noalloc: ") + cudaGetErrorString(e));
  return PBDR_OK;
}
