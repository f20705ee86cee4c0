// Stable LSD radix sort of (uint32 key, uint32 value) pairs, 8-bit digits.
//
// Per pass: (1) every 4096-key tile counts its digits in shared memory and
// writes a digit-major histogram hist[digit][tile] (a thread loads its 16
// keys of the tile at once, as the scatter below does); (2) an exclusive scan of
// that histogram (reduce / top / down-sweep) gives each (digit, tile) its
// first output slot; (3) every tile re-reads its keys in 16 rounds of 256 and
// scatters them: within a round, lanes with equal digits are ranked with
// __match_any_sync, warps are ordered through a small shared-memory prefix,
// and rounds are processed in order, so equal keys keep their input order.
// Integer atomics only touch counters, so the output is deterministic.
#include "pbdr_internal.cuh"

namespace pbdr {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void __launch_bounds__(kThreads) k_hist(const uint32_t *__restrict__ keys, int64_t n,
                                                   int shift, uint32_t *__restrict__ hist,
                                                   int ntiles) {
  __shared__ uint32_t cnt[256];
  cnt[threadIdx.x] = 0;
  const int64_t base = (int64_t)blockIdx.x * kTile;
  // the tile's keys are requested together: one memory round trip
  uint32_t k[kItems];
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const int64_t i = base + r * kThreads + threadIdx.x;
    k[r] = i < n ? keys[i] : 0u;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kItems; ++r)
    if (base + r * kThreads + threadIdx.x < n) atomicAdd(&cnt[(k[r] >> shift) & 255u], 1u);
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// block-wide exclusive scan of one value per thread; returns the block total
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *warp_sums,
                                                         uint32_t &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    uint32_t s = lane < nw ? warp_sums[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) warp_sums[lane] = s;   // inclusive
  }
  __syncthreads();
  total = warp_sums[(blockDim.x >> 5) - 1];
  uint32_t before = warp > 0 ? warp_sums[warp - 1] : 0u;
  __syncthreads();
  return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *__restrict__ a,
                                                              int64_t m,
                                                              uint32_t *__restrict__ part) {
  __shared__ uint32_t ws[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < m) s += a[base + k];
  uint32_t total;
  block_exclusive_scan(s, ws, total);
  if (threadIdx.x == 0) part[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(uint32_t *__restrict__ part, int np) {
  __shared__ uint32_t ws[32];
  uint32_t carry = 0;
  for (int base = 0; base < np; base += kScanThreads) {
    int i = base + threadIdx.x;
    uint32_t v = i < np ? part[i] : 0u;
    uint32_t total;
    uint32_t ex = block_exclusive_scan(v, ws, total);
    if (i < np) part[i] = carry + ex;
    carry += total;
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(uint32_t *__restrict__ a, int64_t m,
                                                            const uint32_t *__restrict__ part) {
  __shared__ uint32_t ws[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = base + k < m ? a[base + k] : 0u;
    s += v[k];
  }
  uint32_t total;
  uint32_t ex = block_exclusive_scan(s, ws, total) + part[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < m) a[base + k] = ex;
    ex += v[k];
  }
}

__global__ void __launch_bounds__(kThreads) k_scatter(const uint32_t *__restrict__ kin,
                                                      const uint32_t *__restrict__ vin,
                                                      uint32_t *__restrict__ kout,
                                                      uint32_t *__restrict__ vout, int64_t n,
                                                      int shift,
                                                      const uint32_t *__restrict__ offs,
                                                      int ntiles) {
  __shared__ uint32_t base[256];
  __shared__ uint32_t wcnt[kThreads / 32][256];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const uint32_t lt_mask = (1u << lane) - 1u;
  base[t] = offs[(int64_t)t * ntiles + blockIdx.x];
  const int64_t tile0 = (int64_t)blockIdx.x * kTile;
  // the thread's keys and values of all rounds are requested together (one
  // memory round trip per tile instead of one per round)
  uint32_t kr[kItems], vr[kItems];
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const int64_t i = tile0 + r * kThreads + t;
    if (i < n) {
      kr[r] = kin[i];
      vr[r] = vin[i];
    }
  }
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) wcnt[w][t] = 0u;
    __syncthreads();
    const int64_t i = tile0 + r * kThreads + t;
    const bool valid = i < n;
    uint32_t key = 0, val = 0, d = 256u;
    if (valid) {
      key = kr[r];
      val = vr[r];
      d = (key >> shift) & 255u;
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t rank = __popc(peers & lt_mask);
    const bool leader = (__ffs(peers) - 1) == lane;
    if (valid && leader) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) {
      uint32_t c = wcnt[w][t];
      wcnt[w][t] = run;
      run += c;
    }
    __syncthreads();
    if (valid) {
      const uint32_t pos = base[d] + wcnt[warp][d] + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
    base[t] += run;
  }
}

}  // namespace

size_t radix_hist_words(int64_t n) {
  int64_t ntiles = (n + kTile - 1) / kTile;
  if (ntiles < 1) ntiles = 1;
  int64_t m = 256 * ntiles;
  int64_t nparts = (m + kScanTile - 1) / kScanTile;
  return (size_t)(m + nparts + 32);
}

int radix_sort_pairs(uint32_t *ka, uint32_t *va, uint32_t *kb, uint32_t *vb, uint32_t *hist,
                     int64_t n, int bits, int *out_in_b, cudaStream_t s) {
  *out_in_b = 0;
  if (n <= 1 || bits <= 0) return 0;
  const int ntiles = (int)((n + kTile - 1) / kTile);
  const int64_t m = 256 * (int64_t)ntiles;
  const int nparts = (int)((m + kScanTile - 1) / kScanTile);
  uint32_t *part = hist + m;
  int launches = 0;
  uint32_t *kin = ka, *vin = va, *kout = kb, *vout = vb;
  int passes = (bits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    k_hist<<<ntiles, kThreads, 0, s>>>(kin, n, shift, hist, ntiles);
    k_scan_reduce<<<nparts, kScanThreads, 0, s>>>(hist, m, part);
    k_scan_top<<<1, kScanThreads, 0, s>>>(part, nparts);
    k_scan_down<<<nparts, kScanThreads, 0, s>>>(hist, m, part);
    k_scatter<<<ntiles, kThreads, 0, s>>>(kin, vin, kout, vout, n, shift, hist, ntiles);
    launches += 5;
    uint32_t *tk = kin, *tv = vin;
    kin = kout;
    vin = vout;
    kout = tk;
    vout = tv;
  }
  *out_in_b = (passes & 1);
  return launches;
}

}  // namespace pbdr
