// sph_sort.cu -- stable LSD radix sort of (cell key, index) pairs and the
// cell offsets of the cell-linked list (Sec. 2.4.1), in launches that never
// wait on one another: the cell sort of a caller's point set
// (sph_cell_sort_noalloc).  The stepping path sorts with the single
// cooperative launch of sph_cellsort.cu instead.
//
// Digit width RB (8..10 bits) is chosen from the key length so that keys of
// up to 20 bits sort in two passes.  Per pass:
//   upsweep   : per-tile digit histogram (shared-memory atomics), laid out
//               [digit][tile] so that one exclusive scan yields every
//               (digit, tile) output offset;
//   scan      : the [digit][tile] array is scanned in chunks of 2048 by many
//               blocks (local exclusive scans + chunk totals), the chunk
//               totals by one block; the chunk offset is added in the
//               downsweep;
//   downsweep : stable rank of every element inside its tile -- each warp
//               walks 256 consecutive elements in 8 rounds of 32, peers of a
//               digit are found with __match_any_sync, per-warp digit
//               counters keep the rank stable -- then scatter.
// Element counts live in device memory so the whole step is enqueued without
// a host round trip; tiles past the count exit.
#include "sph_internal.cuh"

namespace sphk {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;  // 2048
constexpr int SC_THREADS = 1024;
constexpr int SC_CHUNK = 2 * SC_THREADS;  // scan chunk

template <int RB>
__global__ void __launch_bounds__(RS_THREADS) rs_upsweep(const uint32_t *__restrict__ keys,
                                                         const int32_t *__restrict__ d_count, int shift,
                                                         uint32_t *__restrict__ hist, int nblocks) {
  constexpr int RADIX = 1 << RB;
  __shared__ uint32_t cnt[RADIX];
  const int n = *d_count;
  const int base = blockIdx.x * RS_TILE;
  for (int d = threadIdx.x; d < RADIX; d += RS_THREADS) cnt[d] = 0;
  __syncthreads();
  if (base < n) {
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
      int i = base + r * RS_THREADS + threadIdx.x;
      if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & (RADIX - 1)], 1u);
    }
  }
  __syncthreads();
  for (int d = threadIdx.x; d < RADIX; d += RS_THREADS) hist[d * nblocks + blockIdx.x] = cnt[d];
}

// block-wide exclusive scan of one value per thread (1024 threads)
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *warp_sums, uint32_t *total) {
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
    uint32_t s = warp_sums[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    warp_sums[lane] = s;  // inclusive
  }
  __syncthreads();
  uint32_t excl = (warp > 0 ? warp_sums[warp - 1] : 0u) + x - v;
  if (total) *total = warp_sums[31];
  return excl;
}

// local exclusive scan of each chunk of SC_CHUNK entries; chunk totals out
__global__ void __launch_bounds__(SC_THREADS) rs_scan_local(uint32_t *__restrict__ hist, int total,
                                                            uint32_t *__restrict__ chunk_sum) {
  __shared__ uint32_t ws[32];
  const int base = blockIdx.x * SC_CHUNK;
  const int i0 = base + 2 * threadIdx.x;
  uint32_t a = i0 < total ? hist[i0] : 0u;
  uint32_t b = i0 + 1 < total ? hist[i0 + 1] : 0u;
  uint32_t tot = 0;
  uint32_t ex = block_exclusive_scan(a + b, ws, &tot);
  if (i0 < total) hist[i0] = ex;
  if (i0 + 1 < total) hist[i0 + 1] = ex + a;
  if (threadIdx.x == 0) chunk_sum[blockIdx.x] = tot;
}

// exclusive scan of the chunk totals (any count), one block
__global__ void __launch_bounds__(SC_THREADS) rs_scan_chunks(uint32_t *__restrict__ chunk_sum, int nchunks) {
  __shared__ uint32_t ws[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nchunks; base += SC_THREADS) {
    int i = base + threadIdx.x;
    uint32_t v = i < nchunks ? chunk_sum[i] : 0u;
    uint32_t tot = 0;
    uint32_t ex = block_exclusive_scan(v, ws, &tot);
    uint32_t c = carry;
    if (i < nchunks) chunk_sum[i] = c + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry = c + tot;
    __syncthreads();
  }
}

template <int RB>
__global__ void __launch_bounds__(RS_THREADS) rs_downsweep(
    const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
    uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out, const int32_t *__restrict__ d_count,
    int shift, const uint32_t *__restrict__ hist, const uint32_t *__restrict__ chunk_off, int nblocks) {
  constexpr int RADIX = 1 << RB;
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
      uint32_t h = d * nblocks + blockIdx.x;
      uint32_t pos = hist[h] + chunk_off[h / SC_CHUNK] + wh[warp][d] + rank[r];
      keys_out[pos] = key[r];
      vals_out[pos] = val[r];
    }
  }
}

static int digit_bits(int bits, int *passes) {
  int p = (bits + 9) / 10;  // passes of at most 10 bits
  if (p < 1) p = 1;
  int rb = (bits + p - 1) / p;
  if (rb < 8) rb = 8;
  *passes = p;
  return rb;
}

template <int RB>
static void sort_passes(uint32_t *&ki, uint32_t *&vi, uint32_t *&ko, uint32_t *&vo, const int32_t *d_count,
                        int nblocks, int passes, const SortTemp &tmp, cudaStream_t st) {
  const int total = (1 << RB) * nblocks;
  const int nchunks = (total + SC_CHUNK - 1) / SC_CHUNK;
  uint32_t *hist = tmp.hist, *chunks = tmp.hist + total;
  for (int p = 0; p < passes; ++p) {
    const int shift = p * RB;
    rs_upsweep<RB><<<nblocks, RS_THREADS, 0, st>>>(ki, d_count, shift, hist, nblocks);
    rs_scan_local<<<nchunks, SC_THREADS, 0, st>>>(hist, total, chunks);
    rs_scan_chunks<<<1, SC_THREADS, 0, st>>>(chunks, nchunks);
    rs_downsweep<RB><<<nblocks, RS_THREADS, 0, st>>>(ki, vi, ko, vo, d_count, shift, hist, chunks, nblocks);
    uint32_t *t;
    t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
  }
}

void radix_sort(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt, const int32_t *d_count,
                int max_count, int bits, const SortTemp &tmp, cudaStream_t st, uint32_t **keys_result,
                uint32_t **vals_result) {
  int nblocks = (max_count + RS_TILE - 1) / RS_TILE;
  if (nblocks < 1) nblocks = 1;
  int passes;
  const int rb = digit_bits(bits, &passes);
  uint32_t *ki = keys, *vi = vals, *ko = keys_alt, *vo = vals_alt;
  if (rb <= 8)
    sort_passes<8>(ki, vi, ko, vo, d_count, nblocks, passes, tmp, st);
  else if (rb == 9)
    sort_passes<9>(ki, vi, ko, vo, d_count, nblocks, passes, tmp, st);
  else
    sort_passes<10>(ki, vi, ko, vo, d_count, nblocks, passes, tmp, st);
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

void cell_offsets(const uint32_t *keys, const int32_t *d_count, uint32_t ncell, uint32_t *off, int32_t *d_nlive,
                  cudaStream_t st) {
  uint32_t n = ncell + 1;
  k_cell_offsets<<<(n + 255) / 256, 256, 0, st>>>(keys, d_count, ncell, off, d_nlive);
}

}  // namespace sphk
