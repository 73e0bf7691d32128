// sph_sort.cu -- stable LSD radix sort of (cell key, index) pairs and the
// cell offsets of the cell-linked list (Sec. 2.4.1: the list is rebuilt
// after deletion every advection step, Sec. 2.4.3).
//
// One pass per 8-bit digit, three kernels per pass:
//   upsweep   : per-tile digit histogram (shared-memory atomics)
//   scan      : exclusive scan of the [digit][tile] histogram (one block)
//   downsweep : stable rank of every element inside its tile -- warps walk
//               their 256 consecutive elements in 8 rounds of 32, peers of
//               a digit are found with __match_any_sync, per-warp digit
//               counters make the rank stable -- then scatter.
// The element count lives in device memory, so the whole step can be
// enqueued without a host round trip; tiles past the count exit.
#include "sph_internal.cuh"

namespace sphk {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;  // 2048
constexpr int RADIX = 256;

__global__ void __launch_bounds__(RS_THREADS) rs_upsweep(const uint32_t *__restrict__ keys,
                                                         const int32_t *__restrict__ d_count, int shift,
                                                         uint32_t *__restrict__ hist, int nblocks) {
  __shared__ uint32_t cnt[RADIX];
  const int n = *d_count;
  const int base = blockIdx.x * RS_TILE;
  cnt[threadIdx.x] = 0;
  __syncthreads();
  if (base < n) {
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
      int i = base + r * RS_THREADS + threadIdx.x;
      if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & (RADIX - 1)], 1u);
    }
  }
  __syncthreads();
  hist[threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// exclusive scan of hist[0 .. total) in place, one block of 1024 threads
__global__ void __launch_bounds__(1024) rs_scan(uint32_t *__restrict__ hist, int total) {
  __shared__ uint32_t warp_sums[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int base = 0; base < total; base += 1024) {
    int i = base + threadIdx.x;
    uint32_t v = i < total ? hist[i] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t s = warp_sums[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      warp_sums[lane] = s;  // inclusive
    }
    __syncthreads();
    uint32_t excl = carry + (warp > 0 ? warp_sums[warp - 1] : 0u) + x - v;
    if (i < total) hist[i] = excl;
    __syncthreads();
    if (threadIdx.x == 1023) carry = excl + v;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(RS_THREADS) rs_downsweep(
    const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
    uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out, const int32_t *__restrict__ d_count,
    int shift, const uint32_t *__restrict__ hist, int nblocks) {
  __shared__ uint32_t wh[RS_WARPS][RADIX];
  const int n = *d_count;
  const int base = blockIdx.x * RS_TILE;
  if (base >= n) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < RS_WARPS * RADIX; d += RS_THREADS) (&wh[0][0])[d] = 0;
  __syncthreads();
  uint32_t key[RS_ROUNDS], val[RS_ROUNDS], rank[RS_ROUNDS];
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {
    int i = base + warp * (RS_ROUNDS * 32) + r * 32 + lane;
    bool ok = i < n;
    key[r] = ok ? keys_in[i] : 0u;
    val[r] = ok ? vals_in[i] : 0u;
    uint32_t d = ok ? ((key[r] >> shift) & (RADIX - 1)) : (uint32_t)RADIX;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    uint32_t before = __popc(peers & lt);
    uint32_t prev = ok ? wh[warp][d] : 0u;
    rank[r] = prev + before;
    __syncwarp();
    if (ok && before == 0) wh[warp][d] = prev + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit, exclusive prefix over warps
  for (int d = threadIdx.x; d < RADIX; d += RS_THREADS) {
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) {
      uint32_t t = wh[w][d];
      wh[w][d] = run;
      run += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {
    int i = base + warp * (RS_ROUNDS * 32) + r * 32 + lane;
    if (i < n) {
      uint32_t d = (key[r] >> shift) & (RADIX - 1);
      uint32_t pos = hist[d * nblocks + blockIdx.x] + wh[warp][d] + rank[r];
      keys_out[pos] = key[r];
      vals_out[pos] = val[r];
    }
  }
}

void radix_sort(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                const int32_t *d_count, int max_count, int bits, const SortTemp &tmp, cudaStream_t st,
                uint32_t **keys_result, uint32_t **vals_result) {
  int nblocks = (max_count + RS_TILE - 1) / RS_TILE;
  if (nblocks < 1) nblocks = 1;
  uint32_t *ki = keys, *vi = vals, *ko = keys_alt, *vo = vals_alt;
  for (int shift = 0; shift < bits; shift += 8) {
    rs_upsweep<<<nblocks, RS_THREADS, 0, st>>>(ki, d_count, shift, tmp.hist, nblocks);
    rs_scan<<<1, 1024, 0, st>>>(tmp.hist, RADIX * nblocks);
    rs_downsweep<<<nblocks, RS_THREADS, 0, st>>>(ki, vi, ko, vo, d_count, shift, tmp.hist, nblocks);
    uint32_t *t;
    t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
  }
  *keys_result = ki;
  *vals_result = vi;
}

// off[c] = first index t with keys[t] >= c (lower bound), c in [0, ncell];
// the sentinel key ncell marks deleted entries, so off[ncell] = live count
__global__ void k_cell_offsets(const uint32_t *__restrict__ keys, const int32_t *__restrict__ d_count,
                               uint32_t ncell, uint32_t *__restrict__ off, int32_t *__restrict__ d_nlive) {
  uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c > ncell) return;
  int lo = 0, hi = *d_count;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (keys[mid] < c)
      lo = mid + 1;
    else
      hi = mid;
  }
  off[c] = (uint32_t)lo;
  if (c == ncell) *d_nlive = lo;
}

void cell_offsets(const uint32_t *keys, const int32_t *d_count, uint32_t ncell, uint32_t *off,
                  int32_t *d_nlive, cudaStream_t st) {
  uint32_t n = ncell + 1;
  k_cell_offsets<<<(n + 255) / 256, 256, 0, st>>>(keys, d_count, ncell, off, d_nlive);
}

}  // namespace sphk
