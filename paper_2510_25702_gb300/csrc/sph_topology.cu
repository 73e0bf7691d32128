// sph_topology.cu -- particle bookkeeping of one advection step:
//   * permute  : gather every master field into cell order (a2), label each
//                particle by the buffer boxes of its instance (a3,
//                Sec. 3.2) and fold the time-step maxima (a4);
//   * time step: dual-criteria advection / acoustic steps (a4, Sec. 2.3);
//   * buffer update: injection across the generation line and ID-checked
//                deletion (a12, a13; Sec. 2.4.2, 2.4.3, 3.1, 3.2) with stable
//                compaction (a14): survivors keep index order, copies are
//                appended in index order, deleted entries get the sentinel
//                key so the next sort drops them.
#include "sph_internal.cuh"

namespace sphk {

// ------------------------------------------------------------------------
// permute + label + time-step maxima
// ------------------------------------------------------------------------

// gather of particle t (source slot sorted_vals[t]) into cell order, its
// label, its advection record; returns |v|^2 and nu_t (as the bit patterns
// of non-negative doubles, which order like the values) and its instance
template <typename R>
__device__ __forceinline__ int permute_one(const TopoArgs &a, const Packs<R> &pk, int t, unsigned long long *v2_out,
                                           unsigned long long *nu_out) {
  const int s = (int)a.sorted_vals[t];
  const Masters S = a.src, D = a.dst;
  const int ii = S.inst[s];
  const InstDev &I = a.inst[ii];
  const bool d3 = I.dim == 3;
  // in 2D the z components of both master copies stay 0 (set at creation,
  // written as 0 by sph_write_fields) and are not moved
  double x = S.x[0][s], y = S.x[1][s], z = d3 ? S.x[2][s] : 0.0;
  double vx = S.v[0][s], vy = S.v[1][s], vz = d3 ? S.v[2][s] : 0.0;
  double rho = S.rho[s], mass = S.mass[s];
  D.x[0][t] = x;
  D.x[1][t] = y;
  D.v[0][t] = vx;
  D.v[1][t] = vy;
  if (d3) {
    D.x[2][t] = z;
    D.v[2][t] = vz;
  }
  D.rho[t] = rho;
  D.mass[t] = mass;
  D.drho[t] = S.drho[s];
  // the pressure master is rewritten by the advection or continuity sweep
  // of every step before anything reads it; only kinematic stepping keeps it
  if (a.carry_p) D.p[t] = S.p[s];
  double k = S.k[s], eps = S.eps[s], nut = S.nut[s];
  D.k[t] = k;
  D.eps[t] = eps;
  D.nut[t] = nut;
  D.uid[t] = S.uid[s];
  D.inst[t] = (uint16_t)ii;
  int32_t lab = S.label[s];
  const float xf = f64_to_f32(x), yf = f64_to_f32(y), zf = f64_to_f32(z);
  for (int b = 0; b < I.nbuf; ++b) {
    const BufDev &B = a.buf[I.buf0 + b];
    const float ex = xf - B.cen[0], ey = yf - B.cen[1], ez = zf - B.cen[2];
    if (ex * ex + ey * ey + ez * ez > B.rad2) continue;  // far from the box
    if (box_contains(B, I.dim, x, y, z)) lab = B.local_id + 1;
  }
  D.label[t] = lab;
  // advection-sweep record of this particle
  const R V = to_R<R>(mass) / to_R<R>(rho);
  const R vxr = to_R<R>(vx), vyr = to_R<R>(vy);
  // positions: FP64 as they are; FP32 in the fixed point of the instance,
  // with the absolute FP32 coordinates for the list builder beside them
  R px = to_R<R>(x), py = to_R<R>(y), pz = to_R<R>(z);
  if constexpr (sizeof(R) == 4) {
    pk.lpos[t] = V4<R>{px, py, pz, (R)0};
    px = fx_encode(I, x, 0);
    py = fx_encode(I, y, 1);
    pz = d3 ? fx_encode(I, z, 2) : (R)0;
  }
  if (!d3) {
    pk.adv[2 * (size_t)t] = V4<R>{px, py, V, vxr};
    pk.adv[2 * (size_t)t + 1] = V4<R>{vyr, to_R<R>(k), to_R<R>(eps), to_R<R>(nut)};
  } else {
    pk.adv[2 * (size_t)t] = V4<R>{px, py, pz, V};
    pk.adv[2 * (size_t)t + 1] = V4<R>{vxr, vyr, to_R<R>(vz), to_R<R>(k)};
    if (I.rans) pk.adv_b[t] = V4<R>{to_R<R>(eps), to_R<R>(nut), (R)0, (R)0};
  }
  // |v|^2 with the plain left-to-right sum (in the sweep precision: the
  // FP64 form keeps the exact FP64 maximum), nu_t
  double v2;
  if (sizeof(R) == 8) {
    v2 = dmul(vx, vx);
    v2 = dadd(v2, dmul(vy, vy));
    if (d3) v2 = dadd(v2, dmul(vz, vz));
  } else {
    const float fx = f64_to_f32(vx), fy = f64_to_f32(vy), fz = f64_to_f32(vz);
    v2 = f32_to_f64(fx * fx + fy * fy + (d3 ? fz * fz : 0.0f));
  }
  *v2_out = (unsigned long long)__double_as_longlong(v2);
  *nu_out = I.rans ? (unsigned long long)__double_as_longlong(nut) : 0ull;
  return ii;
}

// cell offsets of the sorted keys: off[c] = first slot t whose key is >= c,
// for c in [0, sentinel]; slot t writes the cells after its predecessor's key
// up to its own, the last live slot also the cells up to the sentinel, so
// off[sentinel] = n (the live count)
__device__ __forceinline__ void cell_offsets_at(const TopoArgs &a, int t, int n) {
  if (n == 0) {
    for (uint32_t c = (uint32_t)t; c <= a.sentinel; c += gridDim.x * blockDim.x) a.off[c] = 0u;
    return;
  }
  if (t >= n) return;
  const uint32_t key = a.sorted_keys[t];
  const uint32_t c0 = t > 0 ? a.sorted_keys[t - 1] + 1u : 0u;
  for (uint32_t c = c0; c <= key; ++c) a.off[c] = (uint32_t)t;
  if (t == n - 1)
    for (uint32_t c = key + 1u; c <= a.sentinel; ++c) a.off[c] = (uint32_t)n;
}

template <typename R>
__global__ void __launch_bounds__(kBlock) k_permute(TopoArgs a, Packs<R> pk) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  // an earlier error (the sort's bounded waits among them) leaves the sorted
  // order undefined: nothing after it runs
  if (a.cnt->status) return;
  const int n = a.cnt->n_live;
  if (a.off) cell_offsets_at(a, t, n);
  // time-step maxima: reduced over the warp, then the block, for the
  // instance of the block's first particle (particles are instance-sorted,
  // so almost every block has one); other instances go straight to global
  // memory
  __shared__ int s_ii;
  __shared__ unsigned long long s_v2, s_nu;
  const int base = blockIdx.x * blockDim.x;
  if (threadIdx.x == 0) {
    s_ii = base < n ? (int)a.src.inst[a.sorted_vals[base]] : -1;
    s_v2 = 0ull;
    s_nu = 0ull;
  }
  __syncthreads();
  unsigned long long v2 = 0ull, nu = 0ull;
  int ii = -1;
  if (t < n) ii = permute_one<R>(a, pk, t, &v2, &nu);
  const bool mine = ii == s_ii;
  unsigned long long w2 = mine ? v2 : 0ull, wn = mine ? nu : 0ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y2 = __shfl_xor_sync(0xffffffffu, w2, o);
    const unsigned long long yn = __shfl_xor_sync(0xffffffffu, wn, o);
    w2 = y2 > w2 ? y2 : w2;
    wn = yn > wn ? yn : wn;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&s_v2, w2);
    atomicMax(&s_nu, wn);
  }
  if (ii >= 0 && !mine) {
    atomicMax(&a.v2max[ii], v2);
    atomicMax(&a.nutmax[ii], nu);
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_ii >= 0) {
    atomicMax(&a.v2max[s_ii], s_v2);
    atomicMax(&a.nutmax[s_ii], s_nu);
  }
}

void launch_permute(const TopoArgs &a, int max_n, int prec, cudaStream_t st, void *packs) {
  int g = (max_n + kBlock - 1) / kBlock;
  if (g < 1) g = 1;
  if (prec == SPH_PREC_FP32)
    k_permute<float><<<g, kBlock, 0, st>>>(a, *(Packs<float> *)packs);
  else
    k_permute<double><<<g, kBlock, 0, st>>>(a, *(Packs<double> *)packs);
}

// ------------------------------------------------------------------------
// a4 dual-criteria time step, one thread per instance
// ------------------------------------------------------------------------
__global__ void k_time_step(StepArgs a) {
  const int ii = blockIdx.x * blockDim.x + threadIdx.x;
  if (ii < a.ninst) time_step_instance(a, ii);
}

StepArgs step_args(const TopoArgs &a) {
  StepArgs s{};
  s.inst = const_cast<InstDev *>(a.inst);
  s.v2max = a.v2max;
  s.nutmax = a.nutmax;
  s.cnt = a.cnt;
  s.ninst = a.ninst;
  s.n_ac_max = a.n_ac_max;
  return s;
}

void launch_time_step(const TopoArgs &a, cudaStream_t st) {
  k_time_step<<<(a.ninst + 63) / 64, 64, 0, st>>>(step_args(a));
}

// ------------------------------------------------------------------------
// buffer update
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_flags(TopoArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = a.cnt->n_live;
  uint8_t f = kKeep;
  if (i < n) {
    int32_t lab = a.src.label[i];
    const int ii = a.src.inst[i];
    const InstDev &I = a.inst[ii];
    if (lab > 0 && lab <= I.nbuf) {
      f = buffer_flag(a.buf[I.buf0 + lab - 1], I.dim, a.src.x[0][i], a.src.x[1][i], a.src.x[2][i]);
      if (f == kInject) atomicAdd(&a.inst_spawn[ii], 1);
    }
    a.flag[i] = f;
  }
  unsigned bal = __ballot_sync(0xffffffffu, f == kInject);
  __shared__ int32_t wc[kBlock / 32];
  if ((threadIdx.x & 31) == 0) wc[threadIdx.x >> 5] = __popc(bal);
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t s = 0;
    for (int w = 0; w < kBlock / 32; ++w) s += wc[w];
    a.block_cnt[blockIdx.x] = s;
  }
}

// single block: exclusive scan of the per-block inject counts, per-instance
// uid bases, capacity check (nothing is committed on overflow)
__global__ void __launch_bounds__(1024) k_spawn_scan(TopoArgs a, int nblocks, uint32_t *uid_base) {
  __shared__ int32_t carry;
  __shared__ int32_t ws[32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // four consecutive counts per thread: up to 4096 blocks in one pass, their
  // loads in flight together
  constexpr int V = 4;
  for (int base = 0; base < nblocks; base += 1024 * V) {
    const int i0 = base + threadIdx.x * V;
    int32_t v[V], sum = 0;
#pragma unroll
    for (int q = 0; q < V; ++q) {
      v[q] = i0 + q < nblocks ? a.block_cnt[i0 + q] : 0;
      sum += v[q];
    }
    int32_t x = sum;
    for (int o = 1; o < 32; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int32_t s = ws[lane];
      for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      ws[lane] = s;
    }
    __syncthreads();
    int32_t excl = carry + (warp > 0 ? ws[warp - 1] : 0) + x - sum;
#pragma unroll
    for (int q = 0; q < V; ++q) {
      if (i0 + q < nblocks) a.block_cnt[i0 + q] = excl;
      excl += v[q];
    }
    __syncthreads();
    if (threadIdx.x == 1023) carry = excl;
    __syncthreads();
  }
  const int32_t total = carry;
  const int32_t n = a.cnt->n_live;
  const int over = (int64_t)n + total > a.capacity;
  // per-instance uid bases: copy number r (global rank) of instance ii gets
  // uid next_uid[ii] + (r - first global rank of ii); an exclusive scan of
  // the per-instance copy counts, by the whole block
  __syncthreads();
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < a.ninst; base += 1024) {
    const int ii = base + threadIdx.x;
    const int32_t c = ii < a.ninst ? a.inst_spawn[ii] : 0;
    int32_t x = c;
    for (int o = 1; o < 32; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int32_t t = ws[lane];
      for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      ws[lane] = t;
    }
    __syncthreads();
    const int32_t run = carry + (warp > 0 ? ws[warp - 1] : 0) + x - c;
    if (ii < a.ninst) {
      uid_base[ii] = a.next_uid[ii] - (uint32_t)run;
      if (!over) a.next_uid[ii] += (uint32_t)c;
      a.inst_spawn[ii] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 1023) carry = run + c;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    a.cnt->overflow = over;
    if (over) set_status(&a.cnt->status, SPH_ERR_CAPACITY);
    const int32_t S = over ? 0 : total;
    a.cnt->n_spawn = S;
    a.cnt->m_pending = n + S;
    a.cnt->n_del_step = 0;
    a.cnt->spawned += (unsigned long long)S;
    a.cnt->spawn_step = a.cnt->step;
    a.cnt->step += 1;
  }
}

// periodic wrap of the position (same test and order as the plain
// definition), then the cell key of the wrapped position
__device__ __forceinline__ void wrap_and_key(const InstDev &I, const Masters &m, int i, uint32_t *keys) {
  double p[3] = {m.x[0][i], m.x[1][i], m.x[2][i]};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (d >= I.dim || !I.periodic[d]) continue;
    if (p[d] >= I.hi[d])
      p[d] = dsub(p[d], I.L[d]);
    else if (p[d] < I.lo[d])
      p[d] = dadd(p[d], I.L[d]);
    m.x[d][i] = p[d];
  }
  keys[i] = cell_key(I, p[0], p[1], p[2]);
}

__global__ void __launch_bounds__(kBlock) k_spawn(TopoArgs a, const uint32_t *uid_base) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = a.cnt->n_live;
  const Masters m = a.src;
  uint8_t f = (i < n) ? a.flag[i] : kKeep;
  const int over = a.cnt->overflow;
  const unsigned bal = __ballot_sync(0xffffffffu, f == kInject);
  __shared__ int32_t wc[kBlock / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) wc[warp] = __popc(bal);
  __syncthreads();
  int32_t off = a.block_cnt[blockIdx.x];
  for (int w = 0; w < warp; ++w) off += wc[w];
  const int32_t rank = off + __popc(bal & ((1u << lane) - 1u));
  if (i >= n) return;
  a.idx[i] = (uint32_t)i;
  const int ii = m.inst[i];
  const InstDev &I = a.inst[ii];
  if (over || f == kKeep) {
    wrap_and_key(I, m, i, a.keys);
    return;
  }
  if (f == kDelete) {
    a.keys[i] = a.sentinel;
    atomicAdd(&a.cnt->deleted, 1ull);
    atomicAdd(&a.cnt->n_del_step, 1);
    return;
  }
  // injection: copy at the parent's position, parent recycled by -L_b n_b
  const int dst = n + rank;
  if (a.spawn_dst) a.spawn_dst[i] = dst;
  for (int d = 0; d < 3; ++d) {
    m.x[d][dst] = m.x[d][i];
    m.v[d][dst] = m.v[d][i];
    a.der.an[d][dst] = a.der.an[d][i];
  }
  for (int c = 0; c < 6; ++c) a.der.B[c][dst] = a.der.B[c][i];
  m.rho[dst] = m.rho[i];
  m.mass[dst] = m.mass[i];
  m.drho[dst] = m.drho[i];
  m.p[dst] = m.p[i];
  m.k[dst] = m.k[i];
  m.eps[dst] = m.eps[i];
  m.nut[dst] = m.nut[i];
  m.inst[dst] = (uint16_t)ii;
  m.label[dst] = 0;
  m.uid[dst] = uid_base[ii] + (uint32_t)rank;
  a.idx[dst] = (uint32_t)dst;
  wrap_and_key(I, m, dst, a.keys);
  const BufDev &B = a.buf[I.buf0 + m.label[i] - 1];
#pragma unroll
  for (int d = 0; d < 3; ++d)
    if (d < I.dim) m.x[d][i] = dsub(m.x[d][i], dmul(B.length, B.frame[d]));
  apply_bc(I, B, m, i, a.cnt->spawn_step, kSubRecycle);
  wrap_and_key(I, m, i, a.keys);
}

void launch_buffer_update(const TopoArgs &a, int max_n, int flags_done, cudaStream_t st) {
  int g = (max_n + kBlock - 1) / kBlock;
  if (g < 1) g = 1;
  if (!flags_done) k_flags<<<g, kBlock, 0, st>>>(a);
  // uid bases live after the per-instance spawn counters
  uint32_t *uid_base = reinterpret_cast<uint32_t *>(a.inst_spawn + a.ninst);
  k_spawn_scan<<<1, 1024, 0, st>>>(a, g, uid_base);
  k_spawn<<<g, kBlock, 0, st>>>(a, uid_base);
}

// keys of every live entry from its current position (after creation or a
// write of positions); entries keyed out as deleted stay deleted
__global__ void k_keys(TopoArgs a, int all_live) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.cnt->m_pending) return;
  a.idx[i] = (uint32_t)i;
  if (!all_live && a.keys[i] == a.sentinel) return;
  const InstDev &I = a.inst[a.src.inst[i]];
  wrap_and_key(I, a.src, i, a.keys);
}

void launch_keys(const TopoArgs &a, int max_n, int all_live, cudaStream_t st) {
  int g = (max_n + kBlock - 1) / kBlock;
  if (g < 1) g = 1;
  k_keys<<<g, kBlock, 0, st>>>(a, all_live);
}

__global__ void k_iota(uint32_t *idx, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) idx[i] = (uint32_t)i;
}

void launch_iota(uint32_t *idx, int max_n, cudaStream_t st) {
  int g = (max_n + 255) / 256;
  if (g < 1) g = 1;
  k_iota<<<g, 256, 0, st>>>(idx, max_n);
}

}  // namespace sphk
