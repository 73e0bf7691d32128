// sph_cellsort.cu -- the cell sort of the stepping path in one cooperative
// launch: a stable LSD radix sort of (cell key, index) pairs (the cell-linked
// list is rebuilt after deletion every advection step, Sec. 2.4.1 and
// 2.4.3), the live count (keys below the deletion sentinel) and the clearing
// of a few words the step accumulates into later (time-step maxima).
//
// Every block owns one contiguous slice of the input.  Per digit pass:
//   1. the block counts its slice's digits -> hist[digit][block];
//   2. grid barrier; one warp per digit scans that digit's row across the
//      blocks (exclusive) and writes the digit total;
//   3. grid barrier; every block scans the digit totals, adds its own row
//      prefix and so knows its first output slot per digit; it then ranks
//      its slice chunk by chunk -- warps in order, rounds in order, lanes in
//      order, so equal keys keep their input order -- and scatters;
//   4. grid barrier before the next pass reads what this one wrote.
// A slice of at most one chunk is loaded and ranked once per pass (step 1)
// and kept in registers until its scatter.  The grid never exceeds what the
// device holds at once (cooperative launch) and every wait is bounded
// (sph_grid.cuh); after a wait ran out every block skips its remaining
// writes.
//
// This replaces, on the stepping path, the four launches per pass of the
// multi-kernel sort in sph_sort.cu (kept for sph_cell_sort_noalloc, whose
// launches must not wait on one another).
#include "sph_internal.cuh"

namespace sphk {

constexpr int CS_THREADS = 256;
constexpr int CS_WARPS = CS_THREADS / 32;
constexpr int CS_ROUNDS = 16;
constexpr int CS_CHUNK = CS_THREADS * CS_ROUNDS;  // 4096 keys ranked at once
constexpr int CS_MAX_RADIX = 1 << 10;

struct CellSortArgs {
  uint32_t *keys[2], *vals[2];  // ping-pong buffers; pass p reads [p & 1]
  const int32_t *d_count;       // keys to sort (device)
  int max_count;                // buffer length
  int passes;                   // digit passes of RB bits
  uint32_t sentinel;            // keys >= sentinel are not counted as live
  int32_t *d_below;             // out: keys below the sentinel
  int32_t *status;              // SPH_ERR_TIMEOUT on a wait that ran out
  uint32_t *hist;               // [radix][grid]
  uint32_t *total;              // [radix]
  GridBarrier *sync;            // word: keys at or above the sentinel
  ClearSpans clear;             // words zeroed by the launch
};

template <int RB>
__global__ void __launch_bounds__(CS_THREADS) k_cell_sort(CellSortArgs a) {
  constexpr int RADIX = 1 << RB;
  constexpr int DPT = RADIX / CS_THREADS;  // digits per thread (RB >= 8)
  constexpr int ROW = 16;                  // row entries per lane in one scan batch
  __shared__ uint32_t wh[CS_WARPS][RADIX];  // per-warp digit counts / offsets of a chunk
  __shared__ uint32_t s_base[RADIX];        // next output slot per digit
  __shared__ uint32_t s_ws[CS_WARPS];
  __shared__ int s_ok;
  const int G = gridDim.x, b = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  int n = *a.d_count;
  if (n < 0) n = 0;
  if (n > a.max_count) n = a.max_count;
  const int per = (n + G - 1) / G;
  const int s0 = min(n, b * per), s1 = min(n, s0 + per);
  // a slice of at most one chunk (the usual case: up to grid x 4096 keys)
  // is loaded and ranked once per pass and kept in registers
  const bool one = s1 - s0 <= CS_CHUNK;

#pragma unroll
  for (int q = 0; q < 3; ++q)
    if (a.clear.p[q])
      for (int i = b * CS_THREADS + threadIdx.x; i < a.clear.n[q]; i += G * CS_THREADS) a.clear.p[q][i] = 0u;

  uint32_t key[CS_ROUNDS], val[CS_ROUNDS], rank[CS_ROUNDS], tot[DPT];
  // load chunk c0 of the slice, rank every key among the equal digits of
  // its warp (rounds in order, lanes in order), then turn the per-warp
  // counts into per-warp offsets (warps in order) and the chunk's totals
  auto rank_chunk = [&](const uint32_t *ki, const uint32_t *vi, int shift, int c0) {
    for (int d = threadIdx.x; d < CS_WARPS * RADIX; d += CS_THREADS) (&wh[0][0])[d] = 0u;
#pragma unroll
    for (int r = 0; r < CS_ROUNDS; ++r) {
      const int i = c0 + warp * (CS_ROUNDS * 32) + r * 32 + lane;
      const bool v = i < s1;
      key[r] = v ? __ldcg(ki + i) : 0u;
      val[r] = v ? __ldcg(vi + i) : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < CS_ROUNDS; ++r) {
      const int i = c0 + warp * (CS_ROUNDS * 32) + r * 32 + lane;
      const bool v = i < s1;
      const uint32_t d = v ? ((key[r] >> shift) & (RADIX - 1)) : (uint32_t)RADIX;
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      const uint32_t before = __popc(peers & lt);
      const uint32_t prev = v ? wh[warp][d] : 0u;
      rank[r] = prev + before;
      __syncwarp();
      if (v && before == 0) wh[warp][d] = prev + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
      const int d = threadIdx.x + j * CS_THREADS;
      uint32_t run = 0;
#pragma unroll
      for (int w = 0; w < CS_WARPS; ++w) {
        const uint32_t t = wh[w][d];
        wh[w][d] = run;
        run += t;
      }
      tot[j] = run;
    }
    __syncthreads();
  };
  auto scatter_chunk = [&](uint32_t *ko, uint32_t *vo, int shift, int c0) {
#pragma unroll
    for (int r = 0; r < CS_ROUNDS; ++r) {
      const int i = c0 + warp * (CS_ROUNDS * 32) + r * 32 + lane;
      if (i < s1) {
        const uint32_t d = (key[r] >> shift) & (RADIX - 1);
        const uint32_t pos = s_base[d] + wh[warp][d] + rank[r];
        if (pos < (uint32_t)a.max_count) {
          ko[pos] = key[r];
          vo[pos] = val[r];
        }
      }
    }
  };

  uint32_t nsync = 0;
  bool ok = true;
  for (int p = 0; p < a.passes && ok; ++p) {
    const bool odd = p & 1;  // selects, not indexing: keeps the arguments in registers
    const uint32_t *ki = odd ? a.keys[1] : a.keys[0], *vi = odd ? a.vals[1] : a.vals[0];
    uint32_t *ko = odd ? a.keys[0] : a.keys[1], *vo = odd ? a.vals[0] : a.vals[1];
    const int shift = p * RB;

    // 1. digit counts of the slice -> hist[digit][block]
    uint32_t above = 0;
    if (one) {
      rank_chunk(ki, vi, shift, s0);
#pragma unroll
      for (int j = 0; j < DPT; ++j) a.hist[(size_t)(threadIdx.x + j * CS_THREADS) * G + b] = tot[j];
      if (p == 0)
#pragma unroll
        for (int r = 0; r < CS_ROUNDS; ++r) {
          const int i = s0 + warp * (CS_ROUNDS * 32) + r * 32 + lane;
          above += (i < s1 && key[r] >= a.sentinel) ? 1u : 0u;
        }
    } else {
      // several chunks: count with one shared atomic per run of equal
      // digits in a warp (keys arrive nearly sorted)
      for (int d = threadIdx.x; d < RADIX; d += CS_THREADS) s_base[d] = 0u;
      __syncthreads();
      for (int c0 = s0; c0 < s1; c0 += CS_CHUNK) {
        uint32_t kk[CS_ROUNDS];
#pragma unroll
        for (int r = 0; r < CS_ROUNDS; ++r) {
          const int i = c0 + warp * (CS_ROUNDS * 32) + r * 32 + lane;
          kk[r] = i < s1 ? __ldcg(ki + i) : 0u;
        }
#pragma unroll
        for (int r = 0; r < CS_ROUNDS; ++r) {
          const int i = c0 + warp * (CS_ROUNDS * 32) + r * 32 + lane;
          const bool v = i < s1;
          const uint32_t d = v ? ((kk[r] >> shift) & (RADIX - 1)) : (uint32_t)RADIX;
          const unsigned peers = __match_any_sync(0xffffffffu, d);
          if (v && (peers & lt) == 0) atomicAdd(&s_base[d], (uint32_t)__popc(peers));
          above += (v && kk[r] >= a.sentinel) ? 1u : 0u;
        }
      }
      __syncthreads();
      for (int d = threadIdx.x; d < RADIX; d += CS_THREADS) a.hist[(size_t)d * G + b] = s_base[d];
    }
    if (p == 0) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) above += __shfl_xor_sync(0xffffffffu, above, o);
      if (lane == 0 && above) atomicAdd(&a.sync->word, above);
    }
    if (!(ok = grid_sync(a.sync, ++nsync, a.status, &s_ok))) break;

    // 2. one warp per digit: exclusive scan of its row across the blocks,
    //    each lane holding up to ROW consecutive entries of a batch
    if (p == 0 && b == 0 && threadIdx.x == 0) *a.d_below = n - (int)__ldcg(&a.sync->word);
    for (int d = b * CS_WARPS + warp; d < RADIX; d += G * CS_WARPS) {
      uint32_t *row = a.hist + (size_t)d * G;
      uint32_t carry = 0;
      for (int j0 = 0; j0 < G; j0 += 32 * ROW) {
        const int jl = j0 + lane * ROW;
        uint32_t e[ROW], sum = 0;
#pragma unroll
        for (int q = 0; q < ROW; ++q) e[q] = jl + q < G ? __ldcg(row + jl + q) : 0u;
#pragma unroll
        for (int q = 0; q < ROW; ++q) sum += e[q];
        uint32_t x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x += y;
        }
        uint32_t run = carry + x - sum;
#pragma unroll
        for (int q = 0; q < ROW; ++q) {
          if (jl + q < G) row[jl + q] = run;
          run += e[q];
        }
        carry += __shfl_sync(0xffffffffu, x, 31);
      }
      if (lane == 0) a.total[d] = carry;
    }
    if (!(ok = grid_sync(a.sync, ++nsync, a.status, &s_ok))) break;

    // 3a. first output slot of every digit for this block
    {
      uint32_t tv[DPT], sum = 0;
#pragma unroll
      for (int j = 0; j < DPT; ++j) {
        tv[j] = __ldcg(a.total + threadIdx.x * DPT + j);
        sum += tv[j];
      }
      uint32_t x = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) s_ws[warp] = x;
      __syncthreads();
      uint32_t run = x - sum;
      for (int w = 0; w < warp; ++w) run += s_ws[w];
#pragma unroll
      for (int j = 0; j < DPT; ++j) {
        const int d = threadIdx.x * DPT + j;
        s_base[d] = run + __ldcg(a.hist + (size_t)d * G + b);
        run += tv[j];
      }
    }
    __syncthreads();

    // 3b. scatter: the ranked chunk in registers, or chunk by chunk
    if (one) {
      scatter_chunk(ko, vo, shift, s0);
    } else {
      for (int c0 = s0; c0 < s1; c0 += CS_CHUNK) {
        rank_chunk(ki, vi, shift, c0);
        scatter_chunk(ko, vo, shift, c0);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < DPT; ++j) s_base[threadIdx.x + j * CS_THREADS] += tot[j];
        __syncthreads();
      }
    }
    if (p + 1 < a.passes && !(ok = grid_sync(a.sync, ++nsync, a.status, &s_ok))) break;
  }

  grid_leave(a.sync);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int cs_digit_bits(int bits, int *passes) {
  int p = (bits + 9) / 10;  // passes of at most 10 bits
  if (p < 1) p = 1;
  int rb = (bits + p - 1) / p;
  if (rb < 8) rb = 8;
  *passes = p;
  return rb;
}

template <int RB>
static int cs_blocks_per_sm() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cell_sort<RB>, CS_THREADS, 0) != cudaSuccess) return 0;
  return nb;
}

int cell_sort_plan(int bits, CellSortPlan *plan) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) return -1;
  int coop = 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return -1;
  int passes = 1;
  const int rb = cs_digit_bits(bits, &passes);
  const int nb = rb <= 8 ? cs_blocks_per_sm<8>() : rb == 9 ? cs_blocks_per_sm<9>() : cs_blocks_per_sm<10>();
  if (nb < 1) return -1;
  plan->rb = rb;
  plan->passes = passes;
  plan->grid = nsm * (nb < kCellSortBlocksPerSm ? nb : kCellSortBlocksPerSm);
  return 0;
}

size_t cell_sort_words(const CellSortPlan &plan) {
  // histogram [radix][grid], digit totals, barrier words
  return (size_t)CS_MAX_RADIX * plan.grid + CS_MAX_RADIX + sizeof(GridBarrier) / 4;
}

void cell_sort(const CellSortPlan &plan, uint32_t *scratch, uint32_t *keys[2], uint32_t *vals[2],
               const int32_t *d_count, int max_count, uint32_t sentinel, int32_t *d_below, int32_t *status,
               const ClearSpans &clear, cudaStream_t st, uint32_t **keys_result, uint32_t **vals_result) {
  CellSortArgs a{};
  for (int q = 0; q < 2; ++q) {
    a.keys[q] = keys[q];
    a.vals[q] = vals[q];
  }
  a.d_count = d_count;
  a.max_count = max_count;
  a.passes = plan.passes;
  a.sentinel = sentinel;
  a.d_below = d_below;
  a.status = status;
  a.hist = scratch;
  a.total = scratch + (size_t)CS_MAX_RADIX * plan.grid;
  a.sync = reinterpret_cast<GridBarrier *>(a.total + CS_MAX_RADIX);
  a.clear = clear;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)plan.grid);
  cfg.blockDim = dim3(CS_THREADS);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (plan.rb <= 8)
    cudaLaunchKernelEx(&cfg, k_cell_sort<8>, a);
  else if (plan.rb == 9)
    cudaLaunchKernelEx(&cfg, k_cell_sort<9>, a);
  else
    cudaLaunchKernelEx(&cfg, k_cell_sort<10>, a);
  *keys_result = keys[plan.passes & 1];
  *vals_result = vals[plan.passes & 1];
}

}  // namespace sphk
