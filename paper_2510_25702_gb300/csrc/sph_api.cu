// sph_api.cu -- host side of the C ABI declared in include/sph.h: context
// creation and validation, device memory layout, the per-step launch
// sequence, field transfer and statistics.
//
// Per advection step, all on the context's stream and without a host round
// trip (counts stay in device memory and kernels read them):
//   cell sort of pending (key, index) pairs, one cooperative launch ->
//   permute (+ cell offsets, + labels, + time-step maxima) -> neighbour
//   list (+ time step) -> advection sweep ->
//   n_ac_max x (momentum sweep, continuity sweep) -> buffer update (flags,
//   scan, spawn + recycle + keys of the next step).
// Instances whose own sub-step count is smaller skip the surplus sub-steps
// inside the kernels, so the launch sequence is the same every step.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <fstream>
#include <sstream>
#include <numeric>
#include <string>
#include <vector>

#include "sph_internal.cuh"

using namespace sphk;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}

#define CUDA_TRY(x)                                                                   \
  do {                                                                                \
    cudaError_t e_ = (x);                                                             \
    if (e_ != cudaSuccess) return fail(SPH_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

const double kPi = 3.14159265358979323846;

}  // namespace

namespace sphk {
// the message sph_last_error returns, for the entry points of other files
int set_error(int code, const char *msg) { return fail(code, msg); }
}  // namespace sphk

struct sph_ctx {
  int dim = 2, prec = SPH_PREC_FP64, ninst = 0;
  bool kinematic = false;
  std::vector<sph_config> cfg;
  std::vector<InstDev> inst;
  std::vector<std::vector<BufDev>> bufs;  // per instance
  sph_alloc alloc{};
  cudaStream_t stream = nullptr;
  // pinned host staging: the readback of counters, instance tail and
  // status word, and one slot per buffer for profile uploads (each with an
  // event, so that a slot is rewritten only after its last copy ran)
  struct Pinned {
    Counters cnt;
    char inst_tail[sizeof(InstDev)];
    int32_t status;
  };
  Pinned *pin = nullptr;
  int red_slices = 0;  // reduction blocks per instance, fixed at the first reduction
  char *prof_stage = nullptr;  // ninst x SPH_MAX_BUFFERS slots of kProfSlot bytes
  std::vector<cudaEvent_t> prof_ev;
  int64_t cap = 0, nw = 0;
  uint32_t ncell = 0;  // all instances; also the sentinel key of deleted entries
  int key_bits = 8;
  int n_ac_max = 1;
  bool started = false;
  int64_t step = 0;
  int64_t launches = 0;  // kernels enqueued by this context
  std::vector<void *> blocks;
  size_t bytes = 0;
  // device
  InstDev *d_inst = nullptr;
  BufDev *d_buf = nullptr;
  Masters M[2];
  int cur = 0;
  Derived der;
  Packs<float> pkf{};
  Packs<double> pkd{};
  uint32_t *K[2] = {nullptr, nullptr}, *Vv[2] = {nullptr, nullptr};
  uint32_t *off = nullptr, *woff = nullptr, *wall_index = nullptr;
  double *wx[3] = {nullptr, nullptr, nullptr};
  Counters *cnt = nullptr;
  unsigned long long *v2max = nullptr, *nutmax = nullptr, *pair_counter = nullptr;
  uint32_t *next_uid = nullptr;
  int32_t *inst_spawn = nullptr;
  uint8_t *flag = nullptr;
  int32_t *block_cnt = nullptr;
  CellSortPlan cs_plan{};
  uint32_t *cs_scratch = nullptr;  // cell_sort_words(cs_plan) words
  GridBarrier *gbar = nullptr;     // barrier words of the sub-step launch
  double *red = nullptr;           // mass / momentum reduction buffers (first use)
  uint32_t *sorted_keys = nullptr, *sorted_vals = nullptr;
  NbrList nl{};
  // stage timing (CUDA event pairs on the context's stream)
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_stage;
  size_t ev_used = 0;
  double stage_ms[SPH_N_STAGES] = {0};
  int64_t stage_n[SPH_N_STAGES] = {0};
  // threads per block of the sweeps: list, advection, momentum, continuity
  int32_t blk[4] = {128, 128, 128, 128};
  // CUDA-graph stepping: one executable graph per master-copy parity
  bool use_graph = false;
  bool graph_warm = false;  // an uncaptured step ran since the last change
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  int64_t graph_kernels[2] = {0, 0};
  // state snapshots: one device allocation each
  struct Snap {
    void *mem = nullptr;
    size_t bytes = 0;
    int64_t step = 0;
  };
  std::vector<Snap> snaps;
  // differentiated window (adjoint)
  struct Adj {
    bool fwd = false;
    sph_adjoint_desc d{};
    std::vector<int32_t> ckpt;
    int32_t end_slot = -1;
    void *mem = nullptr;
    size_t bytes = 0;
    AdjTape T{};
    double *lam[8] = {}, *out[8] = {};  // x3, v3, rho, drho
    double *lxg[3] = {}, *lxs[3] = {}, *lrhos = nullptr, *lB[6] = {}, *lan[3] = {}, *sd[12] = {};
    double *grad = nullptr, *J = nullptr;
    V4<double> *rc = nullptr, *rm = nullptr, *rs = nullptr, *ra = nullptr;
    // what the reverse pass of one step reads, recorded while the segment
    // is recomputed: the tape, the neighbour list, B and a_nu, the masters
    // after the step that the reverse kernels index, the pending keys, the
    // buffer-update flags, the cell offsets and the counters
    struct Slot {
      void *mem = nullptr;
      AdjTape T{};
      NbrList nl{};
      Derived der{};
      Masters m{};
      uint32_t *keys = nullptr, *off = nullptr;
      uint8_t *flag = nullptr;
      Counters *cnt = nullptr;
    };
    std::vector<Slot> slots;
    uint8_t *region = nullptr;
    int32_t *mask = nullptr;
    int64_t n_region = 0;
    double dt = 0.0;
  } adj;

  void drop_graphs() {
    for (int q = 0; q < 2; ++q) {
      if (gexec[q]) cudaGraphExecDestroy(gexec[q]);
      gexec[q] = nullptr;
    }
    graph_warm = false;
  }

  int prof_begin(int stage) {
    if (!prof) return -1;
    if (ev_used + 2 > ev_pool.size()) {
      for (int t = 0; t < 64; ++t) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        ev_pool.push_back(e);
      }
      ev_stage.resize(ev_pool.size());
    }
    int idx = (int)ev_used;
    ev_used += 2;
    ev_stage[idx] = stage;
    cudaEventRecord(ev_pool[idx], stream);
    return idx;
  }
  void prof_end(int idx) {
    if (idx >= 0) cudaEventRecord(ev_pool[idx + 1], stream);
  }
  // after a synchronisation: fold the recorded pairs into the totals
  void prof_collect() {
    for (size_t t = 0; t + 1 < ev_used; t += 2) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev_pool[t], ev_pool[t + 1]) == cudaSuccess) {
        stage_ms[ev_stage[t]] += ms;
        stage_n[ev_stage[t]] += 1;
      }
    }
    ev_used = 0;
  }

  void *packs() { return prec == SPH_PREC_FP32 ? (void *)&pkf : (void *)&pkd; }

  // one block from the caller's allocator (or cudaMalloc), NULL on failure;
  // a block off a 256-byte boundary is handed back and counts as a failure
  // (the sweeps' 256-bit record loads need 32-byte alignment, and 256 is
  // what cudaMalloc gives and what the ABI asks of an allocator)
  void *raw_alloc(size_t n) {
    void *p = nullptr;
    if (alloc.alloc) {
      p = alloc.alloc(alloc.user, n, alloc.stream);
    } else if (cudaMalloc(&p, n) != cudaSuccess) {
      p = nullptr;
    }
    if (p && ((uintptr_t)p & 255u) != 0) {
      if (alloc.free)
        alloc.free(alloc.user, p, alloc.stream);
      else
        cudaFree(p);
      p = nullptr;
    }
    return p;
  }

  void *dalloc(size_t n) {
    if (n == 0) n = 16;
    n = (n + 255) & ~(size_t)255;
    void *p = raw_alloc(n);
    if (p) {
      blocks.push_back(p);
      bytes += n;
    }
    return p;
  }

  void release() {
    for (void *p : blocks) {
      if (alloc.free)
        alloc.free(alloc.user, p, alloc.stream);
      else
        cudaFree(p);
    }
    blocks.clear();
  }

  TopoArgs topo() {
    TopoArgs a{};
    a.inst = d_inst;
    a.buf = d_buf;
    a.src = M[cur];
    a.dst = M[1 - cur];
    a.der = der;
    a.keys = K[0];
    a.idx = Vv[0];
    a.sorted_vals = nullptr;
    a.cnt = cnt;
    a.v2max = v2max;
    a.nutmax = nutmax;
    a.next_uid = next_uid;
    a.inst_spawn = inst_spawn;
    a.flag = flag;
    a.block_cnt = block_cnt;
    a.sentinel = ncell;
    a.ninst = ninst;
    a.n_ac_max = n_ac_max;
    a.capacity = cap;
    return a;
  }

  // later sub-steps as separate launches per sweep (3D: a sweep there takes
  // hundreds of microseconds, and each runs at its own register count and
  // block size with no grid barrier: 8 % faster per sub-step than the fused
  // launch on the 3D mixer) or as one cooperative launch (2D, where a
  // single sub-step is the usual case and the fused launch costs one empty
  // launch instead of 2 (n_ac_max - 1))
  bool split_substeps() const { return dim == 3; }

  SweepArgs with_flags(SweepArgs a) {
    a.flag = flag;
    a.inst_spawn = inst_spawn;
    a.block_cnt = block_cnt;
    return a;
  }

  SweepArgs sweep(int sub, int which) {
    SweepArgs a{};
    a.block = blk[which];
    a.inst = d_inst;
    a.buf = d_buf;
    a.m = M[cur];
    a.der = der;
    a.nl = nl;
    a.keys = sorted_keys;
    a.off = off;
    a.woff = woff;
    a.cnt = cnt;
    a.status = &cnt->status;
    a.sub = sub;
    a.gbar = gbar;
    for (int q = 0; q < 3; ++q) a.wx[q] = wx[q];
    a.any_periodic = 0;
    a.any_extra = 0;
    for (const InstDev &I : inst) {
      a.any_periodic |= I.periodic[0] | I.periodic[1] | I.periodic[2];
      a.any_extra |= I.tvf | I.density_sum | I.wall_fn;
    }
    return a;
  }
};

extern "C" {
static void adj_free(sph_ctx *c);
}

// ------------------------------------------------------------------------
// host-side derived constants (compiled without FP contraction so that the
// cell size, cut-off, lengths and boundary values match the plain
// definitions bit for bit)
// ------------------------------------------------------------------------
template <typename R>
static void fill_sweep_const(const InstDev &I, SweepConst<R> &k) {
  for (int a = 0; a < 3; ++a) {
    k.L[a] = (R)I.L[a];
    k.g[a] = (R)I.g[a];
  }
  k.cut2 = (R)I.cut2;
  k.inv_h = (R)I.inv_h;
  k.c5 = (R)(-5.0) * (R)I.alpha_h * (R)I.inv_h;
  k.reg = (R)I.reg;
  k.rho0 = (R)I.rho0;
  k.nu_l = (R)I.nu_l;
  k.c0 = (R)I.c0;
  k.eta = (R)I.eta;
  k.muR_k = (R)I.muR_k;
  k.inv_c0sq = (R)(1.0 / I.c0sq);
  k.inv_rc0 = (R)I.inv_rc0;
  k.c0sq = (R)I.c0sq;
}

static int build_inst(const sph_config &c, InstDev &I, std::string &why) {
  memset(&I, 0, sizeof(I));
  if (c.dim != 2 && c.dim != 3) return why = "dim must be 2 or 3", -1;
  if (!(c.dp > 0) || !(c.h > 0) || !(c.rho0 > 0) || !(c.c0 > 0) || !(c.nu_l >= 0))
    return why = "dp, h, rho0, c0 must be > 0 and nu_l >= 0", -1;
  if (c.rans && !(c.nu_l > 0)) return why = "RANS needs nu_l > 0", -1;
  if (c.dt_mode < 0 || c.dt_mode > 2) return why = "bad dt_mode", -1;
  if (c.dt_mode == SPH_DT_FIXED && (c.n_ac_fixed < 1 || !(c.dt_ad_fixed > 0)))
    return why = "fixed dt needs dt_ad_fixed > 0 and n_ac_fixed >= 1", -1;
  if (c.dt_mode != SPH_DT_FIXED && !(c.U_ref > 0)) return why = "U_ref must be > 0", -1;
  if (c.dt_mode != SPH_DT_FIXED && !c.rans && !(c.nu_l > 0)) return why = "nu_l must be > 0", -1;
  if (c.obc < SPH_OBC_IMPROVED || c.obc > SPH_OBC_MINIMAL_MIRROR) return why = "bad obc", -1;
  if (c.density_sum != 0 && c.density_sum != 1) return why = "density_sum must be 0 or 1", -1;
  if (!(c.tvf_alpha >= 0.0 && c.tvf_alpha < 1.0)) return why = "tvf_alpha must be in [0, 1)", -1;
  if (c.wall_function != 0 && c.wall_function != 1) return why = "wall_function must be 0 or 1", -1;
  if (c.tvf_pbuf != 0 && c.tvf_pbuf != 1) return why = "tvf_pbuf must be 0 or 1", -1;
  I.dim = c.dim;
  I.rans = c.rans ? 1 : 0;
  I.dt_mode = c.dt_mode;
  I.n_ac_fixed = c.n_ac_fixed;
  I.kinematic = c.kinematic ? 1 : 0;
  I.obc = c.obc;
  I.density_sum = c.density_sum;
  I.tvf = c.tvf_alpha > 0.0 ? 1 : 0;
  I.tvf_k = -2.0 * c.tvf_alpha * c.h * c.h;
  I.tvf_pbuf = c.tvf_pbuf;
  I.wall_fn = c.wall_function ? 1 : 0;
  I.wf_cmu34 = std::pow(kCmu, 0.75);
  I.seed = c.seed;
  I.dp = c.dp;
  I.h = c.h;
  I.rho0 = c.rho0;
  I.c0 = c.c0;
  I.nu_l = c.nu_l;
  I.eta = c.eta;
  I.U_ref = c.U_ref;
  I.dt_ad_fixed = c.dt_ad_fixed;
  I.cs = 2.0 * c.h;
  I.cut2 = I.cs * I.cs;
  uint64_t ncell = 1;
  for (int a = 0; a < 3; ++a) {
    I.g[a] = c.gravity[a];
    I.lo[a] = c.domain_lo[a];
    I.hi[a] = c.domain_hi[a];
    I.L[a] = c.domain_hi[a] - c.domain_lo[a];
    I.periodic[a] = (a < c.dim) ? (c.periodic[a] ? 1 : 0) : 0;
    I.nc[a] = 1;
    if (a < c.dim) {
      if (!(I.L[a] > 0)) return why = "domain_hi must exceed domain_lo", -1;
      double f = std::floor(I.L[a] / I.cs);
      if (f > 1.0e6) return why = "cell grid too large", -1;
      I.nc[a] = (f >= 1.0) ? (int32_t)f : 1;
      if (I.periodic[a] && I.nc[a] < 3) return why = "periodic axes need at least 3 cells of 2h", -1;
    }
    ncell *= (uint64_t)I.nc[a];
  }
  if (ncell > (1ull << 31)) return why = "cell grid too large", -1;
  I.ncell = (uint32_t)ncell;
  double alpha = (c.dim == 2) ? 7.0 / (4.0 * kPi * c.h * c.h) : 21.0 / (16.0 * kPi * c.h * c.h * c.h);
  I.alpha_h = alpha / c.h;
  {
    // sigma_0 / alpha_d: the lattice sum of W(r) / alpha_d = (1 - q/2)^4 (1 + 2q)
    // over the sites of spacing dp within the support, the centre included
    const int R = (int)std::ceil(2.0 * c.h / c.dp) + 1, Rz = c.dim == 3 ? R : 0;
    double s0 = 0.0;
    for (int a = -R; a <= R; ++a)
      for (int b = -R; b <= R; ++b)
        for (int k = -Rz; k <= Rz; ++k) {
          const double q = c.dp * std::sqrt((double)(a * a + b * b + k * k)) / c.h;
          if (q < 2.0) {
            const double w = 1.0 - 0.5 * q;
            s0 += w * w * w * w * (1.0 + 2.0 * q);
          }
        }
    I.dsum_k = c.rho0 / s0;
  }
  I.Vw = (c.dim == 2) ? c.dp * c.dp : c.dp * c.dp * c.dp;
  I.rc0 = c.rho0 * c.c0;
  I.eos_k = c.rho0 * c.c0 * c.c0;
  I.muR_k = 0.5 * c.rho0 * c.h;
  I.reg = 0.01 * c.h;
  I.inv_h = 1.0 / c.h;
  I.inv_cs = 1.0 / I.cs;
  I.inv_rc0 = 1.0 / (c.rho0 * c.c0);
  I.c0sq = c.c0 * c.c0;
  fill_sweep_const(I, I.kf);
  fill_sweep_const(I, I.kd);
  for (int a = 0; a < 3; ++a) I.lo_f[a] = (float)I.lo[a];
  I.inv_cs_f = (float)I.inv_cs;
  {
    // fixed point of the FP32 form: q the smallest power of two that keeps a
    // listed pair's coordinate difference (below the cut-off 2h, with 50 %
    // to spare) under 2^22 units and the domain, with a quarter of its
    // extent again on either side, inside int32 (coordinates beyond wrap
    // modulo 2^32): dp 2^-20 < q <= dp 2^-19 up to a domain of about 1360 dp
    double ext = 1.0;
    for (int a = 0; a < c.dim; ++a) ext = std::max(ext, I.L[a] / c.dp);
    int e = (int)std::floor(std::log2(c.dp)) - 24;
    while (3.0 * c.h >= std::ldexp(4194304.0, e) || 1.5 * ext * c.dp >= std::ldexp(2147483648.0, e)) ++e;
    const double q = std::ldexp(1.0, e);
    I.fx_inv_q = 1.0 / q;
    I.fx_q = (float)q;
    for (int a = 0; a < 3; ++a) {
      I.fx_c[a] = 6755399441055744.0 - I.lo[a] * I.fx_inv_q;  // 1.5 2^52 - lo / q, rounded
      I.fx_o[a] = (float)((6755399441055744.0 - I.fx_c[a]) * q);
    }
    for (int a = 0; a < 3; ++a) I.fx_Lu[a] = (a < c.dim && I.periodic[a]) ? (int32_t)std::nearbyint(I.L[a] / q) : 0;
  }
  I.n_ac = 1;
  return 0;
}

static int n_ac_bound(const sph_config &c) {
  if (c.dt_mode == SPH_DT_FIXED) return c.n_ac_fixed;
  if (c.dt_mode == SPH_DT_SINGLE) return 1;
  // n = ceil(dt_ad / dt_ac) <= ceil((c0 + U_ref) / (2.4 U_ref)) for every
  // |v|max (the ratio is largest at |v|max <= U_ref); one more for rounding
  double b = (c.c0 + c.U_ref) / (2.4 * c.U_ref);
  return (int)std::ceil(b) + 1;
}

static uint32_t host_cell_key(const InstDev &I, const double *x) {
  uint32_t c[3] = {0, 0, 0};
  for (int a = 0; a < I.dim; ++a) {
    double f = std::floor((x[a] - I.lo[a]) / I.cs);
    if (!(f >= 0.0))
      c[a] = 0;
    else if (f >= (double)I.nc[a])
      c[a] = (uint32_t)I.nc[a] - 1;
    else
      c[a] = (uint32_t)f;
  }
  return I.cell_base + (c[2] * (uint32_t)I.nc[1] + c[1]) * (uint32_t)I.nc[0] + c[0];
}

// copy n doubles (or other bytes) from host or device into a host vector
template <typename T>
static int fetch(std::vector<T> &out, const T *src, int64_t n, int on_device) {
  out.resize((size_t)n);
  if (n == 0) return 0;
  if (!src) return fail(SPH_ERR_ARG, "required input array is NULL");
  if (on_device) {
    CUDA_TRY(cudaMemcpy(out.data(), src, sizeof(T) * (size_t)n, cudaMemcpyDeviceToHost));
  } else {
    memcpy(out.data(), src, sizeof(T) * (size_t)n);
  }
  return 0;
}

template <typename T>
static T *alloc_arr(sph_ctx *c, int64_t n) {
  return (T *)c->dalloc(sizeof(T) * (size_t)(n > 0 ? n : 1));
}

template <typename R>
static int alloc_packs(sph_ctx *c, Packs<R> &pk, int64_t cap, int64_t nw) {
  const int d3 = c->dim == 3;
  pk.adv = alloc_arr<V4<R>>(c, cap * (d3 ? RecLayout<3>::adv : RecLayout<2>::adv));
  pk.mom = alloc_arr<V4<R>>(c, cap * (d3 ? RecLayout<3>::mom : RecLayout<2>::mom));
  pk.cont = alloc_arr<V4<R>>(c, cap * (d3 ? RecLayout<3>::cont : RecLayout<2>::cont));
  pk.mom_b = alloc_arr<V4<R>>(c, d3 ? cap : 1);
  pk.adv_b = alloc_arr<V4<R>>(c, d3 ? cap : 1);
  pk.Ap = alloc_arr<V4<R>>(c, cap);
  pk.WP = alloc_arr<V4<R>>(c, nw);
  pk.WV = alloc_arr<V4<R>>(c, nw);
  // the FP32 form's absolute FP32 positions for the list builder
  pk.lpos = alloc_arr<V4<R>>(c, sizeof(R) == 4 ? cap + 4 : 1);
  pk.WPf = alloc_arr<V4<R>>(c, sizeof(R) == 4 ? nw + 4 : 1);
  if (!pk.adv || !pk.adv_b || !pk.mom || !pk.mom_b || !pk.cont || !pk.Ap || !pk.WP || !pk.WV || !pk.lpos || !pk.WPf)
    return -1;
  return 0;
}

// the fixed-point coordinate of the FP32 form, as fx_encode on the device:
// the low word of fma(x, 1 / q, 1.5 2^52 - lo / q)
static float host_fx_encode(const InstDev &I, double x, int a) {
  const double u = std::fma(x, I.fx_inv_q, I.fx_c[a]);
  uint64_t b;
  std::memcpy(&b, &u, sizeof(b));
  const uint32_t v = (uint32_t)b;
  float f;
  std::memcpy(&f, &v, sizeof(f));
  return f;
}

template <typename R>
static int upload_walls(sph_ctx *c, Packs<R> &pk, const std::vector<double> &wpos, const std::vector<double> &wvel,
                        const std::vector<double> &wV, const std::vector<int32_t> &winst) {
  int64_t nw = (int64_t)wV.size();
  std::vector<V4<R>> P((size_t)std::max<int64_t>(nw, 1)), V((size_t)std::max<int64_t>(nw, 1));
  std::vector<V4<R>> Pf((size_t)std::max<int64_t>(nw, 1));
  for (int64_t w = 0; w < nw; ++w) {
    P[w] = V4<R>{(R)wpos[3 * w], (R)wpos[3 * w + 1], (R)wpos[3 * w + 2], (R)wV[w]};
    V[w] = V4<R>{(R)wvel[3 * w], (R)wvel[3 * w + 1], (R)wvel[3 * w + 2], (R)0};
    if constexpr (sizeof(R) == 4) {
      // FP32 form: the sweeps' records in fixed point, the list builder's in FP32
      const InstDev &I = c->inst[winst[w]];
      Pf[w] = V4<R>{(R)wpos[3 * w], (R)wpos[3 * w + 1], (R)wpos[3 * w + 2], (R)0};
      P[w] = V4<R>{host_fx_encode(I, wpos[3 * w], 0), host_fx_encode(I, wpos[3 * w + 1], 1),
                   I.dim == 3 ? host_fx_encode(I, wpos[3 * w + 2], 2) : (R)0, (R)wV[w]};
    }
  }
  if (nw) {
    CUDA_TRY(cudaMemcpy(pk.WP, P.data(), sizeof(V4<R>) * nw, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(pk.WV, V.data(), sizeof(V4<R>) * nw, cudaMemcpyHostToDevice));
    if (sizeof(R) == 4) CUDA_TRY(cudaMemcpy(pk.WPf, Pf.data(), sizeof(V4<R>) * nw, cudaMemcpyHostToDevice));
  }
  return 0;
}

extern "C" {

int sph_abi_version(void) { return SPH_ABI_VERSION; }

const char *sph_last_error(void) { return g_err.c_str(); }

const char *sph_error_string(int code) {
  switch (code) {
    case SPH_OK: return "ok";
    case SPH_ERR_ARG: return "invalid argument";
    case SPH_ERR_CUDA: return "CUDA error";
    case SPH_ERR_CAPACITY: return "particle capacity exceeded";
    case SPH_ERR_NONFINITE: return "non-finite density or velocity";
    case SPH_ERR_TIMEOUT: return "device wait timed out";
    case SPH_ERR_OVERLAP: return "buffer boxes overlap";
    case SPH_ERR_STATE: return "call not valid in this state";
    case SPH_ERR_ALLOC: return "device allocation failed";
    default: return "unknown error";
  }
}

int sph_create(const sph_config *cfg, int32_t n_instances, const sph_particles *init, const sph_alloc *alloc,
               sph_ctx **out) {
  if (!out) return fail(SPH_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!cfg || !init || n_instances < 1 || n_instances > 65535)
    return fail(SPH_ERR_ARG, "need 1..65535 instances with cfg and init arrays");
  sph_ctx *c = new sph_ctx();
  if (alloc) c->alloc = *alloc;
  c->stream = (cudaStream_t)c->alloc.stream;
  c->ninst = n_instances;
  c->dim = cfg[0].dim;
  c->prec = cfg[0].precision;
  c->kinematic = cfg[0].kinematic != 0;
  if (c->prec != SPH_PREC_FP64 && c->prec != SPH_PREC_FP32) {
    delete c;
    return fail(SPH_ERR_ARG, "precision must be SPH_PREC_FP64 or SPH_PREC_FP32");
  }
  c->cfg.assign(cfg, cfg + n_instances);
  c->inst.resize(n_instances);
  c->bufs.resize(n_instances);
  uint64_t cell_base = 0;
  int64_t n_total = 0, cap_total = 0, nw_total = 0;
  for (int i = 0; i < n_instances; ++i) {
    std::string why;
    if (cfg[i].dim != c->dim || cfg[i].precision != c->prec || (cfg[i].kinematic != 0) != c->kinematic) {
      delete c;
      return fail(SPH_ERR_ARG, "all instances must share dim, precision and kinematic mode");
    }
    if (build_inst(cfg[i], c->inst[i], why)) {
      delete c;
      return fail(SPH_ERR_ARG, "instance " + std::to_string(i) + ": " + why);
    }
    if (init[i].n < 0 || init[i].nw < 0 || init[i].capacity < init[i].n) {
      delete c;
      return fail(SPH_ERR_ARG, "instance " + std::to_string(i) + ": need 0 <= n <= capacity, nw >= 0");
    }
    c->inst[i].cell_base = (uint32_t)cell_base;
    cell_base += c->inst[i].ncell;
    n_total += init[i].n;
    cap_total += init[i].capacity;
    nw_total += init[i].nw;
    c->n_ac_max = std::max(c->n_ac_max, n_ac_bound(cfg[i]));
  }
  if (cell_base + 1 >= (1ull << 31) || cap_total >= (1ll << 31) - 1 || nw_total >= (1ll << 31) - 1) {
    delete c;
    return fail(SPH_ERR_ARG, "too many cells or particles for 32-bit indices");
  }
  if (c->n_ac_max > 4096) {
    delete c;
    return fail(SPH_ERR_ARG, "sub-step bound above 4096 (c0 / U_ref too large)");
  }
  c->ncell = (uint32_t)cell_base;
  c->key_bits = 1;
  while ((1ull << c->key_bits) <= (uint64_t)c->ncell) ++c->key_bits;
  c->cap = cap_total;
  c->nw = nw_total;

  // ---- gather initial state on the host (SoA), walls sorted by cell ----
  std::vector<double> X[3], Vv[3], rho, mass, k, eps, nut;
  std::vector<uint32_t> uid;
  std::vector<uint16_t> instid;
  std::vector<uint32_t> next_uid(n_instances, 0);
  std::vector<double> wpos, wvel, wV;
  std::vector<uint32_t> wkey, windex;
  std::vector<int32_t> winst;
  for (int a = 0; a < 3; ++a) {
    X[a].reserve(n_total);
    Vv[a].reserve(n_total);
  }
  for (int i = 0; i < n_instances; ++i) {
    const sph_particles &p = init[i];
    const InstDev &I = c->inst[i];
    std::vector<double> pos, vel, r, m, kk, ee, wp, wv;
    std::vector<uint32_t> u;
    int rc = 0;
    if ((rc = fetch(pos, p.pos, 3 * p.n, p.on_device)) || (rc = fetch(vel, p.vel, 3 * p.n, p.on_device)) ||
        (rc = fetch(r, p.rho, p.n, p.on_device)) || (rc = fetch(m, p.mass, p.n, p.on_device)) ||
        (rc = fetch(wp, p.wall_pos, 3 * p.nw, p.on_device))) {
      delete c;
      return rc;
    }
    if (p.k && (rc = fetch(kk, p.k, p.n, p.on_device))) return delete c, rc;
    if (p.eps && (rc = fetch(ee, p.eps, p.n, p.on_device))) return delete c, rc;
    if (p.uid && (rc = fetch(u, p.uid, p.n, p.on_device))) return delete c, rc;
    if (p.wall_vel && (rc = fetch(wv, p.wall_vel, 3 * p.nw, p.on_device))) return delete c, rc;
    uint32_t umax = 0;
    for (int64_t j = 0; j < p.n; ++j) {
      for (int a = 0; a < 3; ++a) {
        X[a].push_back(a < I.dim ? pos[3 * j + a] : 0.0);
        Vv[a].push_back(a < I.dim ? vel[3 * j + a] : 0.0);
      }
      if (!(r[j] > 0) || !(m[j] > 0)) {
        delete c;
        return fail(SPH_ERR_ARG, "densities and masses must be positive");
      }
      rho.push_back(r[j]);
      mass.push_back(m[j]);
      double kj = kk.empty() ? 0.0 : kk[j], ej = ee.empty() ? 0.0 : ee[j];
      if (I.rans && !(kj > 0 && ej > 0)) {
        delete c;
        return fail(SPH_ERR_ARG, "RANS needs k > 0 and eps > 0 for every particle");
      }
      k.push_back(kj);
      eps.push_back(ej);
      nut.push_back(I.rans ? kCmu * kj * kj / ej : 0.0);
      uint32_t uj = u.empty() ? (uint32_t)j : u[j];
      uid.push_back(uj);
      umax = std::max(umax, uj);
      instid.push_back((uint16_t)i);
    }
    next_uid[i] = p.n ? umax + 1 : 0;
    for (int64_t w = 0; w < p.nw; ++w) {
      double x[3] = {wp[3 * w], wp[3 * w + 1], I.dim == 3 ? wp[3 * w + 2] : 0.0};
      for (int a = 0; a < 3; ++a) {
        wpos.push_back(x[a]);
        wvel.push_back(wv.empty() || a >= I.dim ? 0.0 : wv[3 * w + a]);
      }
      wV.push_back(I.Vw);
      winst.push_back(i);
      wkey.push_back(host_cell_key(I, x));
      windex.push_back((uint32_t)w);
    }
  }
  // sort walls by cell (stable)
  std::vector<int64_t> word((size_t)nw_total);
  std::iota(word.begin(), word.end(), 0);
  std::stable_sort(word.begin(), word.end(), [&](int64_t a, int64_t b) { return wkey[a] < wkey[b]; });
  std::vector<double> swpos(3 * nw_total), swvel(3 * nw_total), swV(nw_total);
  std::vector<uint32_t> swkey(nw_total), swindex(nw_total);
  std::vector<int32_t> swinst(nw_total);
  for (int64_t t = 0; t < nw_total; ++t) {
    int64_t s = word[t];
    for (int a = 0; a < 3; ++a) {
      swpos[3 * t + a] = wpos[3 * s + a];
      swvel[3 * t + a] = wvel[3 * s + a];
    }
    swV[t] = wV[s];
    swinst[t] = winst[s];
    swkey[t] = wkey[s];
    swindex[t] = windex[s];
  }
  std::vector<uint32_t> hwoff(c->ncell + 1);
  {
    int64_t t = 0;
    for (uint32_t cc = 0; cc <= c->ncell; ++cc) {
      while (t < nw_total && swkey[t] < cc) ++t;
      hwoff[cc] = (uint32_t)t;
    }
  }

  // ---- device memory ----
  const int64_t cap = c->cap;
  bool ok = true;
  for (int s = 0; s < 2; ++s) {
    Masters &M = c->M[s];
    for (int a = 0; a < 3; ++a) {
      ok &= (M.x[a] = alloc_arr<double>(c, cap)) != nullptr;
      ok &= (M.v[a] = alloc_arr<double>(c, cap)) != nullptr;
    }
    ok &= (M.rho = alloc_arr<double>(c, cap)) != nullptr;
    ok &= (M.mass = alloc_arr<double>(c, cap)) != nullptr;
    ok &= (M.drho = alloc_arr<double>(c, cap)) != nullptr;
    ok &= (M.p = alloc_arr<double>(c, cap)) != nullptr;
    ok &= (M.k = alloc_arr<double>(c, cap)) != nullptr;
    ok &= (M.eps = alloc_arr<double>(c, cap)) != nullptr;
    ok &= (M.nut = alloc_arr<double>(c, cap)) != nullptr;
    ok &= (M.label = alloc_arr<int32_t>(c, cap)) != nullptr;
    ok &= (M.uid = alloc_arr<uint32_t>(c, cap)) != nullptr;
    ok &= (M.inst = alloc_arr<uint16_t>(c, cap)) != nullptr;
    ok &= (c->K[s] = alloc_arr<uint32_t>(c, cap)) != nullptr;
    ok &= (c->Vv[s] = alloc_arr<uint32_t>(c, cap)) != nullptr;
  }
  for (int q = 0; q < 6; ++q) ok &= (c->der.B[q] = alloc_arr<double>(c, cap)) != nullptr;
  for (int a = 0; a < 3; ++a) {
    ok &= (c->der.an[a] = alloc_arr<double>(c, cap)) != nullptr;
    ok &= (c->wx[a] = alloc_arr<double>(c, nw_total)) != nullptr;
  }
  ok &= (c->off = alloc_arr<uint32_t>(c, (int64_t)c->ncell + 1)) != nullptr;
  ok &= (c->woff = alloc_arr<uint32_t>(c, (int64_t)c->ncell + 1)) != nullptr;
  ok &= (c->wall_index = alloc_arr<uint32_t>(c, nw_total)) != nullptr;
  ok &= (c->cnt = alloc_arr<Counters>(c, 1)) != nullptr;
  ok &= (c->v2max = alloc_arr<unsigned long long>(c, 2 * (int64_t)n_instances)) != nullptr;
  c->nutmax = c->v2max ? c->v2max + n_instances : nullptr;
  ok &= (c->pair_counter = alloc_arr<unsigned long long>(c, 1)) != nullptr;
  ok &= (c->next_uid = alloc_arr<uint32_t>(c, n_instances)) != nullptr;
  ok &= (c->inst_spawn = alloc_arr<int32_t>(c, 2 * (int64_t)n_instances)) != nullptr;
  ok &= (c->flag = alloc_arr<uint8_t>(c, cap)) != nullptr;
  ok &= (c->block_cnt = alloc_arr<int32_t>(c, (cap + kBlock - 1) / kBlock + 1)) != nullptr;
  {
    // neighbour-list entries per particle: 2.5 x the full-support count
    // pi (2h/dp)^2 (2D) or 4/3 pi (2h/dp)^3 (3D), a multiple of 8
    double expect = 0.0;
    for (int i = 0; i < n_instances; ++i) {
      double s = 2.0 * cfg[i].h / cfg[i].dp;
      double e = (c->dim == 2) ? kPi * s * s : 4.0 / 3.0 * kPi * s * s * s;
      expect = std::max(expect, e);
    }
    int kmax = (int)std::ceil(2.5 * expect / 8.0) * 8;
    kmax = std::max(16, std::min(kmax, 4096));
    c->nl.kmax = kmax;
    c->nl.stride = (int32_t)cap;
    const int64_t tiles = (cap + kListTile - 1) / kListTile;
    ok &= (c->nl.nbr = alloc_arr<uint32_t>(c, tiles * kListTile * (int64_t)kmax)) != nullptr;
    ok &= (c->nl.rows = alloc_arr<uint16_t>(c, tiles)) != nullptr;
    ok &= (c->nl.n_real = alloc_arr<uint16_t>(c, cap)) != nullptr;
    ok &= (c->nl.n_wall = alloc_arr<uint16_t>(c, cap)) != nullptr;
  }
  if (cell_sort_plan(c->key_bits, &c->cs_plan) != 0) {
    c->release();
    delete c;
    return fail(SPH_ERR_CUDA, "device without cooperative launch (cell sort)");
  }
  ok &= (c->cs_scratch = alloc_arr<uint32_t>(c, (int64_t)cell_sort_words(c->cs_plan))) != nullptr;
  ok &= (c->gbar = alloc_arr<GridBarrier>(c, 1)) != nullptr;
  ok &= (c->d_inst = alloc_arr<InstDev>(c, n_instances)) != nullptr;
  ok &= (c->d_buf = alloc_arr<BufDev>(c, (int64_t)n_instances * SPH_MAX_BUFFERS)) != nullptr;
  if (ok) ok = (c->prec == SPH_PREC_FP32) ? alloc_packs(c, c->pkf, cap, nw_total) == 0
                                          : alloc_packs(c, c->pkd, cap, nw_total) == 0;
  if (!ok) {
    c->release();
    delete c;
    return fail(SPH_ERR_ALLOC, "device allocation failed");
  }

  {
    // pinned host staging for readback and profile uploads
    const size_t nslots = (size_t)n_instances * SPH_MAX_BUFFERS;
    void *pp = nullptr, *ps = nullptr;
    if (cudaHostAlloc(&pp, sizeof(sph_ctx::Pinned), cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc(&ps, nslots * sizeof(BufDev), cudaHostAllocDefault) != cudaSuccess) {
      if (pp) cudaFreeHost(pp);
      c->release();
      delete c;
      return fail(SPH_ERR_ALLOC, "pinned host allocation failed");
    }
    c->pin = (sph_ctx::Pinned *)pp;
    c->prof_stage = (char *)ps;
    c->prof_ev.assign(nslots, nullptr);
  }

  // ---- uploads ----
  auto up = [&](void *dst, const void *src, size_t n) -> int {
    if (n == 0) return 0;
    CUDA_TRY(cudaMemcpy(dst, src, n, cudaMemcpyHostToDevice));
    return 0;
  };
  int rc = 0;
  // z components of both master copies over the whole capacity: 0 in 2D,
  // where nothing moves them (the permute skips them)
  for (int q = 0; q < 2; ++q) {
    rc |= cudaMemset(c->M[q].x[2], 0, sizeof(double) * (size_t)cap) != cudaSuccess;
    rc |= cudaMemset(c->M[q].v[2], 0, sizeof(double) * (size_t)cap) != cudaSuccess;
  }
  Masters &M = c->M[0];
  for (int a = 0; a < 3 && !rc; ++a) {
    rc |= up(M.x[a], X[a].data(), sizeof(double) * n_total);
    rc |= up(M.v[a], Vv[a].data(), sizeof(double) * n_total);
  }
  std::vector<double> zeros((size_t)std::max<int64_t>(n_total, 1), 0.0);
  std::vector<double> p0((size_t)std::max<int64_t>(n_total, 1), 0.0);
  for (int64_t j = 0; j < n_total; ++j) {
    const InstDev &I = c->inst[instid[j]];
    p0[j] = I.eos_k * (rho[j] / I.rho0 - 1.0);
  }
  std::vector<int32_t> lab((size_t)std::max<int64_t>(n_total, 1), 0);
  rc |= up(M.rho, rho.data(), sizeof(double) * n_total);
  rc |= up(M.mass, mass.data(), sizeof(double) * n_total);
  rc |= up(M.drho, zeros.data(), sizeof(double) * n_total);
  rc |= up(M.p, p0.data(), sizeof(double) * n_total);
  rc |= up(M.k, k.data(), sizeof(double) * n_total);
  rc |= up(M.eps, eps.data(), sizeof(double) * n_total);
  rc |= up(M.nut, nut.data(), sizeof(double) * n_total);
  rc |= up(M.label, lab.data(), sizeof(int32_t) * n_total);
  rc |= up(M.uid, uid.data(), sizeof(uint32_t) * n_total);
  rc |= up(M.inst, instid.data(), sizeof(uint16_t) * n_total);
  {
    std::vector<double> wa(std::max<int64_t>(nw_total, 1));
    for (int a = 0; a < 3; ++a) {
      for (int64_t t = 0; t < nw_total; ++t) wa[t] = swpos[3 * t + a];
      rc |= up(c->wx[a], wa.data(), sizeof(double) * nw_total);
    }
  }
  rc |= up(c->woff, hwoff.data(), sizeof(uint32_t) * (c->ncell + 1));
  rc |= up(c->wall_index, swindex.data(), sizeof(uint32_t) * nw_total);
  rc |= up(c->next_uid, next_uid.data(), sizeof(uint32_t) * n_instances);
  rc |= (c->prec == SPH_PREC_FP32) ? upload_walls(c, c->pkf, swpos, swvel, swV, swinst)
                                   : upload_walls(c, c->pkd, swpos, swvel, swV, swinst);
  Counters h{};
  h.m_pending = (int32_t)n_total;
  rc |= up(c->cnt, &h, sizeof(h));
  {
    // grid-barrier words start at zero (each launch leaves them so)
    std::vector<uint32_t> zw(cell_sort_words(c->cs_plan), 0u);
    rc |= up(c->cs_scratch, zw.data(), sizeof(uint32_t) * zw.size());
    GridBarrier gz{};
    rc |= up(c->gbar, &gz, sizeof(gz));
  }
  std::vector<int32_t> zi(2 * n_instances, 0);
  rc |= up(c->inst_spawn, zi.data(), sizeof(int32_t) * 2 * n_instances);
  rc |= up(c->d_inst, c->inst.data(), sizeof(InstDev) * n_instances);
  if (rc) {
    c->release();
    delete c;
    return SPH_ERR_CUDA;
  }
  // keys of the initial (pending) entries
  launch_keys(c->topo(), (int)std::max<int64_t>(cap, 1), 1, c->stream);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    c->release();
    delete c;
    return fail(SPH_ERR_CUDA, std::string("initial keys: ") + cudaGetErrorString(e));
  }
  *out = c;
  return SPH_OK;
}

void sph_destroy(sph_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  if (c->pin) cudaFreeHost(c->pin);
  if (c->prof_stage) cudaFreeHost(c->prof_stage);
  for (cudaEvent_t e : c->prof_ev)
    if (e) cudaEventDestroy(e);
  adj_free(c);
  for (size_t q = 0; q < c->snaps.size(); ++q)
    if (c->snaps[q].mem) sph_drop_state(c, (int32_t)q);
  c->drop_graphs();
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  c->release();
  delete c;
}

const char *sph_stage_name(int32_t stage) {
  static const char *names[SPH_N_STAGES] = {"sort", "cells", "permute", "time_step",
                                            "advection_sweep", "momentum_sweep", "continuity_sweep",
                                            "buffer_update", "neighbour_list", "later_sub_steps"};
  return (stage >= 0 && stage < SPH_N_STAGES) ? names[stage] : "unknown";
}

int sph_set_profiling(sph_ctx *c, int32_t enable) {
  if (!c) return fail(SPH_ERR_ARG, "ctx is NULL");
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  c->prof_collect();
  if (enable == 2) {
    for (int s = 0; s < SPH_N_STAGES; ++s) {
      c->stage_ms[s] = 0.0;
      c->stage_n[s] = 0;
    }
  }
  c->prof = enable != 0;
  return SPH_OK;
}

int sph_get_stage_times(sph_ctx *c, double *ms_total, int64_t *launches, int32_t max_stages, int32_t *n_stages) {
  if (!c) return fail(SPH_ERR_ARG, "ctx is NULL");
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  c->prof_collect();
  int n = std::min<int>(max_stages, SPH_N_STAGES);
  for (int s = 0; s < n; ++s) {
    if (ms_total) ms_total[s] = c->stage_ms[s];
    if (launches) launches[s] = c->stage_n[s];
  }
  if (n_stages) *n_stages = SPH_N_STAGES;
  return SPH_OK;
}

// separating-axis test of two oriented boxes (2D rectangles / 3D cuboids);
// touching faces do not count as overlap
static bool boxes_overlap(int dim, const sph_buffer_desc &a, const sph_buffer_desc &b) {
  auto corners = [&](const sph_buffer_desc &q, std::vector<std::array<double, 3>> &out) {
    out.clear();
    int nz = dim == 3 ? 2 : 1;
    for (int i0 = 0; i0 < 2; ++i0)
      for (int i1 = 0; i1 < 2; ++i1)
        for (int i2 = 0; i2 < nz; ++i2) {
          double u0 = i0 ? q.length : 0.0, u1 = i1 ? q.half[0] : -q.half[0];
          double u2 = dim == 3 ? (i2 ? q.half[1] : -q.half[1]) : 0.0;
          std::array<double, 3> p;
          for (int d = 0; d < 3; ++d) p[d] = q.origin[d] + u0 * q.frame[d] + u1 * q.frame[3 + d] + u2 * q.frame[6 + d];
          out.push_back(p);
        }
  };
  std::vector<std::array<double, 3>> ca, cb;
  corners(a, ca);
  corners(b, cb);
  std::vector<std::array<double, 3>> axes;
  for (const sph_buffer_desc *q : {&a, &b})
    for (int r = 0; r < dim; ++r) axes.push_back({q->frame[3 * r], q->frame[3 * r + 1], q->frame[3 * r + 2]});
  if (dim == 3) {
    for (int r = 0; r < 3; ++r)
      for (int s = 0; s < 3; ++s) {
        const double *u = &a.frame[3 * r], *v = &b.frame[3 * s];
        std::array<double, 3> w = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
        double nn = std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        if (nn > 1e-9) axes.push_back({w[0] / nn, w[1] / nn, w[2] / nn});
      }
  }
  double scale = std::max({a.length, b.length, a.half[0], b.half[0], 1e-12});
  for (auto &ax : axes) {
    double amin = 1e300, amax = -1e300, bmin = 1e300, bmax = -1e300;
    for (auto &p : ca) {
      double s = p[0] * ax[0] + p[1] * ax[1] + p[2] * ax[2];
      amin = std::min(amin, s);
      amax = std::max(amax, s);
    }
    for (auto &p : cb) {
      double s = p[0] * ax[0] + p[1] * ax[1] + p[2] * ax[2];
      bmin = std::min(bmin, s);
      bmax = std::max(bmax, s);
    }
    if (amax <= bmin + 1e-12 * scale || bmax <= amin + 1e-12 * scale) return false;
  }
  return true;
}

int sph_add_buffer(sph_ctx *c, int32_t instance, const sph_buffer_desc *b, int32_t *out_id) {
  if (!c || !b) return fail(SPH_ERR_ARG, "ctx or buffer is NULL");
  if (instance < 0 || instance >= c->ninst) return fail(SPH_ERR_ARG, "instance out of range");
  if (c->started) return fail(SPH_ERR_STATE, "buffers must be added before the first step");
  const InstDev &I = c->inst[instance];
  const sph_config &cfg = c->cfg[instance];
  if (b->type != SPH_BUF_VELOCITY && b->type != SPH_BUF_PRESSURE) return fail(SPH_ERR_ARG, "bad buffer type");
  if (b->turb_bc != SPH_TURB_ZERO_GRADIENT && b->turb_bc != SPH_TURB_FREESTREAM)
    return fail(SPH_ERR_ARG, "bad turbulence BC");
  if (b->n_theta < 1 || b->n_theta > SPH_MAX_THETA) return fail(SPH_ERR_ARG, "n_theta must be 1..64");
  // the mirror search of a pressure buffer spans two cells each way
  for (int a = 0; a < I.dim; ++a)
    if (b->type == SPH_BUF_PRESSURE && I.periodic[a] && I.nc[a] < 5)
      return fail(SPH_ERR_ARG, "pressure buffers need at least 5 cells on periodic axes");
  if (!(b->length > 0) || !(b->half[0] > 0) || (I.dim == 3 && !(b->half[1] > 0)))
    return fail(SPH_ERR_ARG, "buffer length and half widths must be > 0");
  if (I.rans && b->turb_bc == SPH_TURB_FREESTREAM && !(b->k_in > 0 && b->eps_in > 0))
    return fail(SPH_ERR_ARG, "freestream turbulence needs k_in, eps_in > 0");
  for (int r = 0; r < I.dim; ++r)
    for (int s = 0; s < I.dim; ++s) {
      double d = 0;
      for (int a = 0; a < I.dim; ++a) d += b->frame[3 * r + a] * b->frame[3 * s + a];
      if (std::fabs(d - (r == s ? 1.0 : 0.0)) > 1e-9) return fail(SPH_ERR_ARG, "buffer frame not orthonormal");
    }
  if (c->bufs[instance].size() >= SPH_MAX_BUFFERS) return fail(SPH_ERR_ARG, "too many buffers in this instance");
  // overlap check against the boxes already added to this instance
  for (const BufDev &o : c->bufs[instance]) {
    sph_buffer_desc od{};
    memcpy(od.origin, o.origin, sizeof(od.origin));
    memcpy(od.frame, o.frame, sizeof(od.frame));
    od.length = o.length;
    od.half[0] = o.half[0];
    od.half[1] = o.half[1];
    if (boxes_overlap(I.dim, *b, od)) return fail(SPH_ERR_OVERLAP, "buffer boxes intersect");
  }
  BufDev d;
  memset(&d, 0, sizeof(d));
  d.type = b->type;
  d.turb = b->turb_bc;
  d.n_theta = b->n_theta;
  d.inst = instance;
  d.local_id = (int32_t)c->bufs[instance].size();
  for (int a = 0; a < 3; ++a) d.origin[a] = b->origin[a];
  for (int a = 0; a < 9; ++a) d.frame[a] = b->frame[a];
  d.length = b->length;
  d.half[0] = b->half[0];
  d.half[1] = b->half[1];
  d.p_ob = b->p_ob;
  d.rho_ob = cfg.rho0 * (1.0 + b->p_ob / (cfg.rho0 * cfg.c0 * cfg.c0));
  d.noise = b->noise;
  d.k_in = b->k_in;
  d.eps_in = b->eps_in;
  d.nut_in = (b->eps_in > 0) ? kCmu * b->k_in * b->k_in / b->eps_in : 0.0;
  d.gen_line = b->length + 0.5 * cfg.dp;
  {
    // FP32 bounding sphere: centre of the box and its half diagonal, widened
    // by far more than the FP32 rounding of coordinates and of the test
    double cen[3], hd2 = 0.25 * b->length * b->length + b->half[0] * b->half[0];
    if (I.dim == 3) hd2 += b->half[1] * b->half[1];
    double cabs = 0.0;
    for (int a = 0; a < 3; ++a) {
      cen[a] = b->origin[a] + 0.5 * b->length * b->frame[a];
      d.cen[a] = (float)cen[a];
      cabs = std::max(cabs, std::fabs(cen[a]));
    }
    const double rad = std::sqrt(hd2) + 1e-5 * (cabs + std::sqrt(hd2)) + 1e-3 * cfg.dp;
    d.rad2 = (float)(rad * rad * (1.0 + 1e-5));
  }
  for (int q = 0; q < b->n_theta; ++q) d.theta[q] = b->theta[q];
  c->bufs[instance].push_back(d);
  if (out_id) *out_id = d.local_id;
  return SPH_OK;
}

static int upload_buffers(sph_ctx *c) {
  std::vector<BufDev> all;
  for (int i = 0; i < c->ninst; ++i) {
    c->inst[i].buf0 = (int32_t)all.size();
    c->inst[i].nbuf = (int32_t)c->bufs[i].size();
    for (auto &b : c->bufs[i]) all.push_back(b);
  }
  if (!all.empty()) CUDA_TRY(cudaMemcpyAsync(c->d_buf, all.data(), sizeof(BufDev) * all.size(), cudaMemcpyHostToDevice, c->stream));
  // only the buffer fields of the instance table change here; the rest of
  // the device copy (time, dt) is authoritative
  for (int i = 0; i < c->ninst; ++i) {
    CUDA_TRY(cudaMemcpyAsync(&c->d_inst[i].nbuf, &c->inst[i].nbuf, 2 * sizeof(int32_t), cudaMemcpyHostToDevice,
                             c->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return 0;
}

}  // extern "C"

namespace {
// n 8-byte words from src to dst (one block)
__global__ void k_copy_words(unsigned long long *__restrict__ dst, const unsigned long long *__restrict__ src, int n) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
}
}  // namespace

extern "C" {

int sph_set_profile(sph_ctx *c, int32_t instance, int32_t buffer_id, const double *theta, int32_t n_theta) {
  if (!c || !theta) return fail(SPH_ERR_ARG, "NULL argument");
  if (instance < 0 || instance >= c->ninst) return fail(SPH_ERR_ARG, "instance out of range");
  if (buffer_id < 0 || buffer_id >= (int32_t)c->bufs[instance].size()) return fail(SPH_ERR_ARG, "no such buffer");
  if (n_theta < 1 || n_theta > SPH_MAX_THETA) return fail(SPH_ERR_ARG, "n_theta must be 1..64");
  BufDev &b = c->bufs[instance][buffer_id];
  b.n_theta = n_theta;
  for (int q = 0; q < n_theta; ++q) b.theta[q] = theta[q];
  if (c->started) {
    // only the profile moves: n_theta and theta[0..n_theta), from this
    // buffer's pinned slot, without waiting for the stream; the slot is
    // rewritten only after its previous copies have run
    const int g = c->inst[instance].buf0 + buffer_id;
    const int slot = instance * SPH_MAX_BUFFERS + buffer_id;
    BufDev *stage = reinterpret_cast<BufDev *>(c->prof_stage) + slot;
    cudaEvent_t &ev = c->prof_ev[slot];
    if (ev)
      CUDA_TRY(cudaEventSynchronize(ev));
    else
      CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    stage->n_theta = n_theta;
    for (int q = 0; q < n_theta; ++q) stage->theta[q] = theta[q];
    static_assert(offsetof(BufDev, theta) == offsetof(BufDev, n_theta) + 8, "n_theta directly before theta");
    // the slot is page-locked memory the device addresses: a one-block
    // kernel moves it (no switch to a copy engine between two steps); a
    // copy where the device cannot address it
    void *src = nullptr;
    if (cudaHostGetDevicePointer(&src, &stage->n_theta, 0) == cudaSuccess && src) {
      k_copy_words<<<1, 64, 0, c->stream>>>(reinterpret_cast<unsigned long long *>(&c->d_buf[g].n_theta),
                                            static_cast<const unsigned long long *>(src), 1 + n_theta);
      CUDA_TRY(cudaGetLastError());
    } else {
      cudaGetLastError();
      CUDA_TRY(cudaMemcpyAsync(&c->d_buf[g].n_theta, &stage->n_theta, 8 + sizeof(double) * n_theta,
                               cudaMemcpyHostToDevice, c->stream));
    }
    CUDA_TRY(cudaEventRecord(ev, c->stream));
  }
  return SPH_OK;
}

// sort + cell offsets + permute (+labels, +time-step maxima)
static void enqueue_topology(sph_ctx *c) {
  uint32_t *ks = nullptr, *vs = nullptr;
  // one cooperative launch: sort, live count, and the zeroing of the
  // per-instance time-step maxima (v2max and nutmax, 2 x ninst doubles), of
  // the sub-step count that the time step folds with atomicMax and of the
  // per-block inject counts that the continuity sweep adds to
  int ev = c->prof_begin(0);
  uint32_t *keys[2] = {c->K[0], c->K[1]}, *vals[2] = {c->Vv[0], c->Vv[1]};
  ClearSpans clear{};
  clear.p[0] = reinterpret_cast<uint32_t *>(c->v2max);
  clear.n[0] = 4 * c->ninst;
  clear.p[1] = reinterpret_cast<uint32_t *>(&c->cnt->n_ac_all);
  clear.n[1] = 1;
  clear.p[2] = reinterpret_cast<uint32_t *>(c->block_cnt);
  clear.n[2] = (int)((c->cap + kBlock - 1) / kBlock);
  cell_sort(c->cs_plan, c->cs_scratch, keys, vals, &c->cnt->m_pending, (int)c->cap, c->ncell, &c->cnt->n_live,
            &c->cnt->status, clear, c->stream, &ks, &vs);
  c->prof_end(ev);
  // the permute writes the cell offsets (stage 1 stays empty)
  TopoArgs t = c->topo();
  t.sorted_vals = vs;
  t.sorted_keys = ks;
  t.off = c->off;
  t.carry_p = c->kinematic;
  ev = c->prof_begin(2);
  launch_permute(t, (int)c->cap, c->prec, c->stream, c->packs());
  c->prof_end(ev);
  c->cur = 1 - c->cur;
  c->sorted_keys = ks;
  c->sorted_vals = vs;
  c->launches += 2;
}

static void enqueue_step(sph_ctx *c) {
  enqueue_topology(c);
  const int maxn = (int)c->cap;
  if (!c->kinematic) {
    // the list builder's block 0 also takes the time step (stage 3 stays
    // empty): one launch fewer on the step's critical path
    SweepArgs la = c->sweep(0, 0);
    la.ts = step_args(c->topo());
    la.with_time_step = 1;
    int ev = c->prof_begin(8);
    launch_neighbour_list(la, c->packs(), c->prec, c->dim, maxn, c->stream);
    c->prof_end(ev);
    ev = c->prof_begin(4);
    launch_advection_sweep(c->sweep(0, 1), c->packs(), c->prec, c->dim, maxn, c->stream);
    c->prof_end(ev);
    ev = c->prof_begin(5);
    launch_momentum_sweep(c->sweep(0, 2), c->packs(), c->prec, c->dim, maxn, 0, c->stream);
    c->prof_end(ev);
    // the continuity sweep of each instance's last sub-step also takes the
    // buffer-update flags
    ev = c->prof_begin(6);
    launch_continuity_sweep(c->with_flags(c->sweep(0, 3)), c->packs(), c->prec, c->dim, maxn, 0, c->stream);
    c->prof_end(ev);
    if (c->n_ac_max > 1) {
      ev = c->prof_begin(9);
      if (c->split_substeps()) {
        // sub-steps 1 .. n_ac_max - 1 as one momentum and one continuity
        // launch each; a launch past every instance's sub-step count
        // returns at once
        for (int s = 1; s < c->n_ac_max; ++s) {
          launch_momentum_sweep(c->sweep(s, 2), c->packs(), c->prec, c->dim, maxn, s, c->stream);
          launch_continuity_sweep(c->with_flags(c->sweep(s, 3)), c->packs(), c->prec, c->dim, maxn, s,
                                  c->stream);
        }
      } else {
        // sub-steps 1 .. n_ac - 1: one cooperative launch, empty when every
        // instance takes a single sub-step
        launch_substeps(c->with_flags(c->sweep(1, 2)), c->packs(), c->prec, c->dim, maxn, c->stream);
      }
      c->prof_end(ev);
    }
  }
  int ev = c->prof_begin(7);
  launch_buffer_update(c->topo(), maxn, c->kinematic ? 0 : 1, c->stream);
  c->prof_end(ev);
  const int later = c->n_ac_max <= 1 ? 0 : (c->split_substeps() ? 2 * (c->n_ac_max - 1) : 1);
  c->launches += c->kinematic ? 3 : 2 + 4 + later;
  c->step += 1;
}

static int read_status(sph_ctx *c, int32_t *status) {
  CUDA_TRY(cudaMemcpyAsync(&c->pin->status, &c->cnt->status, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  *status = c->pin->status;
  c->prof_collect();
  return 0;
}

// capture one advection step whose masters start in copy `parity` into an
// executable graph (nothing runs; host counters are left as they were)
static int capture_graph(sph_ctx *c, int parity) {
  if (!c->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  cudaStream_t user = c->stream;
  const bool prof = c->prof;
  const int64_t step = c->step, launches = c->launches;
  const int cur = c->cur;
  c->stream = c->cap_stream;
  c->prof = false;
  c->cur = parity;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    enqueue_step(c);
    e = cudaStreamEndCapture(c->cap_stream, &g);
  }
  c->graph_kernels[parity] = c->launches - launches;
  c->stream = user;
  c->prof = prof;
  c->step = step;
  c->launches = launches;
  c->cur = cur;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&c->gexec[parity], g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    c->gexec[parity] = nullptr;
    cudaGetLastError();
    return fail(SPH_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  }
  return 0;
}

static int enqueue_steps(sph_ctx *c, int32_t nsteps) {
  if (!c) return fail(SPH_ERR_ARG, "ctx is NULL");
  if (nsteps < 0) return fail(SPH_ERR_ARG, "nsteps < 0");
  if (!c->started) {
    int rc = upload_buffers(c);
    if (rc) return rc;
    c->started = true;
  }
  for (int s = 0; s < nsteps; ++s) {
    if (!c->use_graph || !c->graph_warm) {
      // uncaptured; also the first step after graphs were enabled or the
      // launch configuration changed, so that every lazily initialised
      // launch parameter is set before a capture
      enqueue_step(c);
      c->graph_warm = c->use_graph;
      continue;
    }
    if (!c->gexec[c->cur]) {
      int rc = capture_graph(c, c->cur);
      if (rc) return rc;
    }
    CUDA_TRY(cudaGraphLaunch(c->gexec[c->cur], c->stream));
    c->launches += c->graph_kernels[c->cur];
    c->cur = 1 - c->cur;
    c->step += 1;
  }
  CUDA_TRY(cudaGetLastError());
  return SPH_OK;
}

int sph_step_async(sph_ctx *c, int32_t nsteps) { return enqueue_steps(c, nsteps); }

int sph_step(sph_ctx *c, int32_t nsteps, double *t_out) {
  int rc0 = enqueue_steps(c, nsteps);
  if (rc0) return rc0;
  int32_t status = 0;
  int rc = read_status(c, &status);
  if (rc) return rc;
  if (t_out) CUDA_TRY(cudaMemcpy(t_out, &c->d_inst[0].t, sizeof(double), cudaMemcpyDeviceToHost));
  return status;
}

int sph_set_graph(sph_ctx *c, int32_t enable) {
  if (!c) return fail(SPH_ERR_ARG, "ctx is NULL");
  c->use_graph = enable != 0;
  return SPH_OK;
}

int sph_set_launch(sph_ctx *c, const int32_t block[4]) {
  if (!c || !block) return fail(SPH_ERR_ARG, "NULL argument");
  for (int q = 0; q < 4; ++q)
    if (block[q] != 64 && block[q] != 128 && block[q] != 256)
      return fail(SPH_ERR_ARG, "block sizes must be 64, 128 or 256");
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  for (int q = 0; q < 4; ++q) c->blk[q] = block[q];
  c->drop_graphs();
  return SPH_OK;
}

int sph_get_launch(sph_ctx *c, int32_t block[4]) {
  if (!c || !block) return fail(SPH_ERR_ARG, "NULL argument");
  for (int q = 0; q < 4; ++q) block[q] = c->blk[q];
  return SPH_OK;
}

// ------------------------------------------------------------------------
// snapshots
// ------------------------------------------------------------------------
// (device pointer, bytes) of every array a snapshot holds, in a fixed order
static void snap_parts(sph_ctx *c, std::vector<std::pair<void *, size_t>> &parts) {
  parts.clear();
  const size_t cap = (size_t)c->cap, d8 = 8 * cap;
  Masters &M = c->M[c->cur];
  for (int a = 0; a < 3; ++a) {
    parts.push_back({M.x[a], d8});
    parts.push_back({M.v[a], d8});
  }
  for (double *q : {M.rho, M.mass, M.drho, M.p, M.k, M.eps, M.nut}) parts.push_back({q, d8});
  parts.push_back({M.label, 4 * cap});
  parts.push_back({M.uid, 4 * cap});
  parts.push_back({M.inst, 2 * cap});
  parts.push_back({c->K[0], 4 * cap});
  parts.push_back({c->Vv[0], 4 * cap});
  for (int q = 0; q < 6; ++q) parts.push_back({c->der.B[q], d8});
  for (int a = 0; a < 3; ++a) parts.push_back({c->der.an[a], d8});
  parts.push_back({c->cnt, sizeof(Counters)});
  parts.push_back({c->d_inst, sizeof(InstDev) * (size_t)c->ninst});
  parts.push_back({c->next_uid, 4 * (size_t)c->ninst});
  parts.push_back({c->inst_spawn, 8 * (size_t)c->ninst});
}

static size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

int sph_save_state(sph_ctx *c, int32_t *slot_out) {
  if (!c || !slot_out) return fail(SPH_ERR_ARG, "NULL argument");
  std::vector<std::pair<void *, size_t>> parts;
  snap_parts(c, parts);
  size_t total = 0;
  for (auto &p : parts) total += align256(p.second);
  void *mem = c->raw_alloc(total);
  if (!mem) return fail(SPH_ERR_ALLOC, "snapshot allocation failed");
  size_t off = 0;
  for (auto &p : parts) {
    CUDA_TRY(cudaMemcpyAsync((char *)mem + off, p.first, p.second, cudaMemcpyDeviceToDevice, c->stream));
    off += align256(p.second);
  }
  sph_ctx::Snap sn;
  sn.mem = mem;
  sn.bytes = total;
  sn.step = c->step;
  int slot = -1;
  for (size_t q = 0; q < c->snaps.size(); ++q)
    if (!c->snaps[q].mem) {
      slot = (int)q;
      break;
    }
  if (slot < 0) {
    slot = (int)c->snaps.size();
    c->snaps.push_back(sn);
  } else {
    c->snaps[slot] = sn;
  }
  *slot_out = slot;
  return SPH_OK;
}

int sph_restore_state(sph_ctx *c, int32_t slot) {
  if (!c || slot < 0 || slot >= (int32_t)c->snaps.size() || !c->snaps[slot].mem)
    return fail(SPH_ERR_ARG, "unknown snapshot slot");
  std::vector<std::pair<void *, size_t>> parts;
  snap_parts(c, parts);
  const sph_ctx::Snap &sn = c->snaps[slot];
  size_t off = 0;
  for (auto &p : parts) {
    CUDA_TRY(cudaMemcpyAsync(p.first, (char *)sn.mem + off, p.second, cudaMemcpyDeviceToDevice, c->stream));
    off += align256(p.second);
  }
  c->step = sn.step;
  return SPH_OK;
}

int sph_drop_state(sph_ctx *c, int32_t slot) {
  if (!c || slot < 0 || slot >= (int32_t)c->snaps.size() || !c->snaps[slot].mem)
    return fail(SPH_ERR_ARG, "unknown snapshot slot");
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  sph_ctx::Snap &sn = c->snaps[slot];
  if (c->alloc.free)
    c->alloc.free(c->alloc.user, sn.mem, c->alloc.stream);
  else
    cudaFree(sn.mem);
  sn = sph_ctx::Snap();
  return SPH_OK;
}

// ------------------------------------------------------------------------
// differentiated windows
// ------------------------------------------------------------------------
static void adj_free(sph_ctx *c) {
  sph_ctx::Adj &A = c->adj;
  cudaStreamSynchronize(c->stream);
  for (int32_t s : A.ckpt) sph_drop_state(c, s);
  if (A.end_slot >= 0) sph_drop_state(c, A.end_slot);
  auto dfree = [&](void *p) {
    if (!p) return;
    if (c->alloc.free)
      c->alloc.free(c->alloc.user, p, c->alloc.stream);
    else
      cudaFree(p);
  };
  for (auto &sl : A.slots) dfree(sl.mem);
  dfree(A.mem);
  A = sph_ctx::Adj();
}

static void set_freeze(sph_ctx *c, int on) {
  for (int i = 0; i < c->ninst; ++i) {
    c->inst[i].freeze_turb = on;
    cudaMemcpyAsync(&c->d_inst[i].freeze_turb, &c->inst[i].freeze_turb, sizeof(int32_t), cudaMemcpyHostToDevice,
                    c->stream);
  }
}

// carve the work arrays of the reverse pass out of one allocation
static int adj_alloc(sph_ctx *c) {
  sph_ctx::Adj &A = c->adj;
  if (A.mem) return 0;
  const size_t cap = (size_t)c->cap, ns = (size_t)c->n_ac_max;
  const size_t nd = 8 + 8 + 3 + 3 + 1 + 6 + 3 + 12;
  (void)ns;
  const size_t bytes = nd * (cap * 8 + 256) + 2 * (cap * 4 + 256) + 2 * 256 + (size_t)A.d.n_theta * 8 + 8 +
                       (3 + 3 + 3 + 5) * (cap * 32 + 256) +
                       (size_t)A.n_region + 4096;
  void *mem = c->raw_alloc(bytes);
  if (!mem) return fail(SPH_ERR_ALLOC, "adjoint work arrays");
  A.mem = mem;
  A.bytes = bytes;
  char *p = (char *)mem;
  auto take = [&](size_t n) {
    void *q = p;
    p += (n + 255) & ~(size_t)255;
    return q;
  };
  auto d = [&]() { return (double *)take(cap * 8); };
  for (int k = 0; k < 8; ++k) A.lam[k] = d();
  for (int k = 0; k < 8; ++k) A.out[k] = d();
  for (int k = 0; k < 3; ++k) A.lxg[k] = d();
  for (int k = 0; k < 3; ++k) A.lxs[k] = d();
  A.lrhos = d();
  for (int k = 0; k < 6; ++k) A.lB[k] = d();
  for (int k = 0; k < 3; ++k) A.lan[k] = d();
  for (int k = 0; k < 12; ++k) A.sd[k] = d();
  A.rc = (V4<double> *)take(3 * cap * 32);
  A.rm = (V4<double> *)take(3 * cap * 32);
  A.rs = (V4<double> *)take(3 * cap * 32);
  A.ra = (V4<double> *)take(5 * cap * 32);
  A.grad = (double *)take((size_t)A.d.n_theta * 8);
  A.J = (double *)take(8);
  A.region = (uint8_t *)take((size_t)A.n_region + 1);
  A.mask = (int32_t *)take(SPH_MAX_BUFFERS * 4);
  return 0;
}

static int slot_alloc(sph_ctx *c, sph_ctx::Adj::Slot &sl) {
  if (sl.mem) return 0;
  const size_t cap = (size_t)c->cap, ns = (size_t)c->n_ac_max;
  const size_t tiles = (cap + kListTile - 1) / kListTile;
  const size_t nbr = tiles * kListTile * (size_t)c->nl.kmax;
  const size_t ncell1 = (size_t)c->ncell + 1;
  // doubles: tape 8 + ns (1 + 1 + 3 + 3 + 12); B 6, a_nu 3; masters mass, k, nut, x 3
  const size_t nd = 8 + ns * 20 + 9 + 6;
  const size_t bytes = nd * (cap * 8 + 256) + (nbr * 4 + 256) + 2 * (cap * 2 + 256) + 5 * (cap * 4 + 256) +
                       (cap * 2 + 256) + (cap + 256) + (ncell1 * 4 + 256) + 512 + 4096;
  void *mem = c->raw_alloc(bytes);
  if (!mem) return fail(SPH_ERR_ALLOC, "adjoint step records");
  sl.mem = mem;
  char *p = (char *)mem;
  auto take = [&](size_t n) {
    void *q = p;
    p += (n + 255) & ~(size_t)255;
    return q;
  };
  auto d = [&]() { return (double *)take(cap * 8); };
  AdjTape &T = sl.T;
  T.cap = (int64_t)cap;
  for (int k = 0; k < 3; ++k) T.x0[k] = d();
  for (int k = 0; k < 3; ++k) T.v0[k] = d();
  T.rho0 = d();
  T.drho0 = d();
  T.rho_s = (double *)take(ns * cap * 8);
  T.drho_s = (double *)take(ns * cap * 8);
  for (int k = 0; k < 3; ++k) T.v1[k] = (double *)take(ns * cap * 8);
  for (int k = 0; k < 3; ++k) T.xbc[k] = (double *)take(ns * cap * 8);
  T.S = (double *)take(ns * 12 * cap * 8);
  T.perm = (uint32_t *)take(cap * 4);
  T.spawn_dst = (int32_t *)take(cap * 4);
  sl.nl = c->nl;
  sl.nl.nbr = (uint32_t *)take(nbr * 4);
  sl.nl.n_real = (uint16_t *)take(cap * 2);
  sl.nl.n_wall = (uint16_t *)take(cap * 2);
  sl.nl.rows = nullptr;
  for (int q = 0; q < 6; ++q) sl.der.B[q] = d();
  for (int k = 0; k < 3; ++k) sl.der.an[k] = d();
  sl.m.mass = d();
  sl.m.k = d();
  sl.m.nut = d();
  for (int k = 0; k < 3; ++k) sl.m.x[k] = d();
  sl.m.label = (int32_t *)take(cap * 4);
  sl.m.uid = (uint32_t *)take(cap * 4);
  sl.m.inst = (uint16_t *)take(cap * 2);
  sl.keys = (uint32_t *)take(cap * 4);
  sl.flag = (uint8_t *)take(cap);
  sl.off = (uint32_t *)take(ncell1 * 4);
  sl.cnt = (Counters *)take(sizeof(Counters));
  return 0;
}

static AdjArgs adj_args(sph_ctx *c, const sph_ctx::Adj::Slot *sl = nullptr) {
  sph_ctx::Adj &A = c->adj;
  AdjArgs a{};
  a.inst = c->d_inst;
  a.buf = c->d_buf;
  a.m = c->M[c->cur];
  a.der = c->der;
  a.nl = c->nl;
  a.off = c->off;
  a.woff = c->woff;
  a.pending_keys = c->K[0];
  for (int k = 0; k < 3; ++k) a.wx[k] = c->wx[k];
  a.WV = c->pkd.WV;
  a.cnt = c->cnt;
  a.flag = c->flag;
  if (sl) {
    a.m = sl->m;
    a.der = sl->der;
    a.nl = sl->nl;
    a.off = sl->off;
    a.pending_keys = sl->keys;
    a.cnt = sl->cnt;
    a.flag = sl->flag;
    a.T = sl->T;
  }
  for (int k = 0; k < 3; ++k) {
    a.lx[k] = A.lam[k];
    a.lv[k] = A.lam[3 + k];
    a.lxg[k] = A.lxg[k];
    a.lxs[k] = A.lxs[k];
    a.lan[k] = A.lan[k];
  }
  a.lrho = A.lam[6];
  a.ldrho = A.lam[7];
  a.lrhos = A.lrhos;
  for (int k = 0; k < 6; ++k) a.lB[k] = A.lB[k];
  for (int k = 0; k < 12; ++k) a.sd[k] = A.sd[k];
  for (int k = 0; k < 8; ++k) a.out[k] = A.out[k];
  a.rc = A.rc;
  a.rm = A.rm;
  a.rs = A.rs;
  a.ra = A.ra;
  a.grad = A.grad;
  a.J = A.J;
  a.region = A.region;
  a.n_region = A.n_region;
  a.g_inst = A.d.instance;
  a.g_buf = A.d.profile_buffer;
  a.o_inst = A.d.instance;
  a.sentinel = c->ncell;
  a.w_s = A.d.slab;
  a.dt_obj = A.dt;
  return a;
}

// one advection step, recording into slot sl what its reverse pass reads
static void enqueue_step_taped(sph_ctx *c, sph_ctx::Adj::Slot &sl) {
  enqueue_topology(c);
  const int maxn = (int)c->cap;
  const size_t cap = (size_t)c->cap;
  cudaStream_t st = c->stream;
  AdjArgs a = adj_args(c);
  a.T = sl.T;  // tape kernels read the live masters and write the slot
  cudaMemcpyAsync(sl.T.perm, c->sorted_vals, 4 * cap, cudaMemcpyDeviceToDevice, st);
  launch_adj_tape_start(a, maxn, st);
  launch_time_step(c->topo(), st);
  launch_neighbour_list(c->sweep(0, 0), c->packs(), c->prec, c->dim, maxn, st);
  launch_advection_sweep(c->sweep(0, 1), c->packs(), c->prec, c->dim, maxn, st);
  for (int s = 0; s < c->n_ac_max; ++s) {
    SweepArgs sm = c->sweep(s, 2);
    sm.tape_S = sl.T.S;
    launch_momentum_sweep(sm, c->packs(), c->prec, c->dim, maxn, s, st);
    launch_adj_tape_sub(a, s, maxn, st);
    launch_continuity_sweep(c->sweep(s, 3), c->packs(), c->prec, c->dim, maxn, s, st);
    launch_adj_tape_drho(a, s, maxn, st);
  }
  TopoArgs t = c->topo();
  t.spawn_dst = sl.T.spawn_dst;
  launch_buffer_update(t, maxn, 0, st);
  // the state the reverse kernels index
  auto cp = [&](void *dst, const void *src, size_t n) { cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToDevice, st); };
  const size_t tiles = (cap + kListTile - 1) / kListTile;
  cp(sl.nl.nbr, c->nl.nbr, tiles * kListTile * (size_t)c->nl.kmax * 4);
  cp(sl.nl.n_real, c->nl.n_real, cap * 2);
  cp(sl.nl.n_wall, c->nl.n_wall, cap * 2);
  for (int q = 0; q < 6; ++q) cp(sl.der.B[q], c->der.B[q], cap * 8);
  for (int k = 0; k < 3; ++k) cp(sl.der.an[k], c->der.an[k], cap * 8);
  const Masters &M = c->M[c->cur];
  cp(sl.m.mass, M.mass, cap * 8);
  cp(sl.m.k, M.k, cap * 8);
  cp(sl.m.nut, M.nut, cap * 8);
  for (int k = 0; k < 3; ++k) cp(sl.m.x[k], M.x[k], cap * 8);
  cp(sl.m.label, M.label, cap * 4);
  cp(sl.m.uid, M.uid, cap * 4);
  cp(sl.m.inst, M.inst, cap * 2);
  cp(sl.keys, c->K[0], cap * 4);
  cp(sl.flag, c->flag, cap);
  cp(sl.off, c->off, ((size_t)c->ncell + 1) * 4);
  cp(sl.cnt, c->cnt, sizeof(Counters));
  c->launches += 3 + 3 + 4 * c->n_ac_max + 3;
  c->step += 1;
}

// reverse of the step recorded in slot sl; the adjoint arrays go from the
// state after the step to the state before it
static void enqueue_step_reverse(sph_ctx *c, const sph_ctx::Adj::Slot &sl) {
  sph_ctx::Adj &A = c->adj;
  const int maxn = (int)c->cap;
  const size_t b8 = 8 * (size_t)c->cap;
  for (int k = 0; k < 3; ++k) {
    cudaMemsetAsync(A.lxg[k], 0, b8, c->stream);
    cudaMemsetAsync(A.lxs[k], 0, b8, c->stream);
    cudaMemsetAsync(A.lan[k], 0, b8, c->stream);
  }
  cudaMemsetAsync(A.lrhos, 0, b8, c->stream);
  for (int k = 0; k < 6; ++k) cudaMemsetAsync(A.lB[k], 0, b8, c->stream);
  int any_per = 0;
  for (const InstDev &I : c->inst) any_per |= I.periodic[0] | I.periodic[1] | I.periodic[2];
  AdjArgs a = adj_args(c, &sl);
  launch_adj_objective(a, 1, maxn, c->stream);
  launch_adj_buffer_rev(a, maxn, c->stream);
  for (int s = c->n_ac_max - 1; s >= 0; --s) launch_adj_substep_rev(a, c->dim, any_per, s, maxn, c->stream);
  launch_adj_adv_rev(a, c->dim, any_per, maxn, c->stream);
  for (int k = 0; k < 8; ++k) cudaMemsetAsync(A.out[k], 0, b8, c->stream);
  launch_adj_perm_rev(a, maxn, c->stream);
  for (int k = 0; k < 8; ++k) std::swap(A.lam[k], A.out[k]);
  c->launches += 4 + 6 * c->n_ac_max + 3;
}

int sph_adjoint_forward(sph_ctx *c, const sph_adjoint_desc *d, double *J_out) {
  if (!c || !d) return fail(SPH_ERR_ARG, "NULL argument");
  if (c->prec != SPH_PREC_FP64) return fail(SPH_ERR_ARG, "differentiated windows need an FP64 context");
  if (c->kinematic) return fail(SPH_ERR_ARG, "kinematic contexts have no dynamics to differentiate");
  if (d->instance < 0 || d->instance >= c->ninst) return fail(SPH_ERR_ARG, "instance out of range");
  if (d->steps < 1 || d->checkpoint_every < 1) return fail(SPH_ERR_ARG, "steps and checkpoint_every must be >= 1");
  if (d->n_theta < 1 || d->n_theta > SPH_MAX_THETA) return fail(SPH_ERR_ARG, "n_theta must be 1..64");
  if (!(d->slab > 0)) return fail(SPH_ERR_ARG, "slab must be > 0");
  for (int i = 0; i < c->ninst; ++i) {
    if (c->cfg[i].dt_mode != SPH_DT_FIXED) return fail(SPH_ERR_ARG, "differentiated windows need SPH_DT_FIXED");
    if (c->cfg[i].obc != SPH_OBC_IMPROVED) return fail(SPH_ERR_ARG, "differentiated windows need SPH_OBC_IMPROVED");
    if (c->cfg[i].density_sum || c->cfg[i].tvf_alpha != 0.0 || c->cfg[i].wall_function)
      return fail(SPH_ERR_ARG, "differentiated windows need density_sum = 0, tvf_alpha = 0 and wall_function = 0");
  }
  const auto &bufs = c->bufs[d->instance];
  if (d->profile_buffer < 0 || d->profile_buffer >= (int32_t)bufs.size() ||
      bufs[d->profile_buffer].type != SPH_BUF_VELOCITY)
    return fail(SPH_ERR_ARG, "profile_buffer must be a velocity buffer of the instance");
  if (d->n_outlets < 1 || d->n_outlets > SPH_MAX_BUFFERS) return fail(SPH_ERR_ARG, "need 1..16 outlets");
  for (int q = 0; q < d->n_outlets; ++q)
    if (d->outlets[q] < 0 || d->outlets[q] >= (int32_t)bufs.size()) return fail(SPH_ERR_ARG, "outlet out of range");
  adj_free(c);
  int rc = sph_set_profile(c, d->instance, d->profile_buffer, d->theta, d->n_theta);
  if (rc) return rc;
  if (!c->started) {
    if ((rc = upload_buffers(c))) return rc;
    c->started = true;
  }
  sph_ctx::Adj &A = c->adj;
  A.d = *d;
  A.dt = c->cfg[d->instance].dt_ad_fixed;
  uint32_t nu = 0;
  CUDA_TRY(cudaMemcpy(&nu, c->next_uid + d->instance, 4, cudaMemcpyDeviceToHost));
  A.n_region = (int64_t)nu;
  if ((rc = adj_alloc(c))) return rc;
  int32_t mask[SPH_MAX_BUFFERS] = {0};
  for (int q = 0; q < d->n_outlets; ++q) mask[d->outlets[q]] = 1;
  CUDA_TRY(cudaMemcpyAsync(A.mask, mask, sizeof(mask), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(cudaMemsetAsync(A.region, 0, (size_t)A.n_region + 1, c->stream));
  CUDA_TRY(cudaMemsetAsync(A.J, 0, 8, c->stream));
  launch_adj_region(adj_args(c), A.region, A.mask, (int)c->cap, c->stream);
  set_freeze(c, 1);
  for (int n = 0; n < d->steps; ++n) {
    if (n % d->checkpoint_every == 0) {
      int32_t slot;
      if ((rc = sph_save_state(c, &slot))) break;
      A.ckpt.push_back(slot);
    }
    enqueue_step(c);
    launch_adj_objective(adj_args(c), 0, (int)c->cap, c->stream);
  }
  if (!rc) rc = sph_save_state(c, &A.end_slot);
  set_freeze(c, 0);
  if (rc) return rc;
  CUDA_TRY(cudaGetLastError());
  int32_t status = 0;
  if ((rc = read_status(c, &status))) return rc;
  if (status) return status;
  double J = 0.0;
  CUDA_TRY(cudaMemcpy(&J, A.J, 8, cudaMemcpyDeviceToHost));
  if (J_out) *J_out = J;
  A.fwd = true;
  return SPH_OK;
}

int sph_adjoint_backward(sph_ctx *c, double *grad_out, int32_t n_theta) {
  if (!c) return fail(SPH_ERR_ARG, "ctx is NULL");
  sph_ctx::Adj &A = c->adj;
  if (!A.fwd) return fail(SPH_ERR_STATE, "sph_adjoint_backward needs a completed sph_adjoint_forward");
  if (grad_out && n_theta != A.d.n_theta) return fail(SPH_ERR_ARG, "n_theta differs from the forward window");
  const size_t b8 = 8 * (size_t)c->cap;
  for (int k = 0; k < 8; ++k) CUDA_TRY(cudaMemsetAsync(A.lam[k], 0, b8, c->stream));
  CUDA_TRY(cudaMemsetAsync(A.grad, 0, 8 * (size_t)A.d.n_theta, c->stream));
  set_freeze(c, 1);
  const int K = A.d.checkpoint_every, steps = A.d.steps;
  const int nseg = (int)A.ckpt.size();
  int rc = 0;
  if ((int)A.slots.size() < K) A.slots.resize(K);
  for (int q = 0; q < K && !rc; ++q) rc = slot_alloc(c, A.slots[q]);
  for (int seg = nseg - 1; seg >= 0 && !rc; --seg) {
    const int s0 = seg * K, s1 = std::min(s0 + K, steps);
    if ((rc = sph_restore_state(c, A.ckpt[seg]))) break;
    for (int n = s0; n < s1; ++n) enqueue_step_taped(c, A.slots[n - s0]);
    for (int n = s1 - 1; n >= s0; --n) enqueue_step_reverse(c, A.slots[n - s0]);
  }
  if (!rc) rc = sph_restore_state(c, A.end_slot);
  set_freeze(c, 0);
  if (rc) return rc;
  CUDA_TRY(cudaGetLastError());
  int32_t status = 0;
  if ((rc = read_status(c, &status))) return rc;
  if (status) return status;
  if (grad_out) CUDA_TRY(cudaMemcpy(grad_out, A.grad, 8 * (size_t)A.d.n_theta, cudaMemcpyDeviceToHost));
  return SPH_OK;
}

int sph_adjoint_release(sph_ctx *c) {
  if (!c) return fail(SPH_ERR_ARG, "ctx is NULL");
  adj_free(c);
  return SPH_OK;
}

// ------------------------------------------------------------------------
// autotuner of the sweep block sizes
// ------------------------------------------------------------------------
static std::string tune_key(sph_ctx *c) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  std::string name = "gpu";
  if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) {
    name = prop.name;
    sms = prop.multiProcessorCount;
  }
  for (char &ch : name)
    if (ch == ' ' || ch == '\t') ch = '_';
  Counters h;
  int64_t n = 0;
  if (cudaMemcpy(&h, c->cnt, sizeof(h), cudaMemcpyDeviceToHost) == cudaSuccess) n = h.m_pending - h.n_del_step;
  int rans = 0;
  for (const InstDev &I : c->inst) rans |= I.rans;
  return name + "|sm" + std::to_string(sms) + "|d" + std::to_string(c->dim) + "|p" + std::to_string(c->prec) +
         "|i" + std::to_string(c->ninst) + "|n" + std::to_string(n) + "|w" + std::to_string(c->nw) + "|r" +
         std::to_string(rans) + "|s" + std::to_string(c->n_ac_max);
}

int sph_autotune(sph_ctx *c, int32_t steps, const char *cache_path, int32_t block_out[4], int32_t *from_cache) {
  if (!c) return fail(SPH_ERR_ARG, "ctx is NULL");
  if (steps < 1) return fail(SPH_ERR_ARG, "steps must be >= 1");
  if (from_cache) *from_cache = 0;
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  const std::string key = tune_key(c);
  if (cache_path) {
    std::ifstream in(cache_path);
    std::string line;
    while (std::getline(in, line)) {
      std::istringstream ls(line);
      std::string k;
      int32_t b[4];
      if (!(ls >> k >> b[0] >> b[1] >> b[2] >> b[3]) || k != key) continue;
      int rc = sph_set_launch(c, b);
      if (rc) continue;
      if (block_out)
        for (int q = 0; q < 4; ++q) block_out[q] = b[q];
      if (from_cache) *from_cache = 1;
      return SPH_OK;
    }
  }
  if (!c->started) {
    int rc = upload_buffers(c);
    if (rc) return rc;
    c->started = true;
  }
  int32_t slot = -1;
  int rc = sph_save_state(c, &slot);
  if (rc) return rc;
  const bool prof = c->prof, graph = c->use_graph;
  // each trial times whole advection steps as they are normally run, replayed
  // from the step's CUDA graphs, so that the choice includes how the sweeps
  // share the GPU with the kernels around them; the sweeps are tuned in turn
  // (coordinate descent)
  const int cand[3] = {64, 128, 256};
  int32_t best[4];
  for (int q = 0; q < 4; ++q) best[q] = c->blk[q];
  c->prof = false;
  c->use_graph = true;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = fail(SPH_ERR_CUDA, "events");
  for (int q = 0; q < 4 && !rc; ++q) {
    double best_ms = 1e300;
    for (int t = 0; t < 3 && !rc; ++t) {
      int32_t trial[4];
      for (int u = 0; u < 4; ++u) trial[u] = best[u];
      trial[q] = cand[t];
      if ((rc = sph_set_launch(c, trial)) || (rc = sph_restore_state(c, slot))) break;
      // untimed: one uncaptured step, then both graphs captured and replayed
      if ((rc = enqueue_steps(c, 3))) break;
      int32_t st = 0;
      if ((rc = read_status(c, &st))) break;
      cudaEventRecord(e0, c->stream);
      if ((rc = enqueue_steps(c, steps))) break;
      cudaEventRecord(e1, c->stream);
      if ((rc = read_status(c, &st))) break;
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = fail(SPH_ERR_CUDA, "event timing");
        break;
      }
      if (ms < best_ms) {
        best_ms = ms;
        best[q] = cand[t];
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  c->prof = prof;
  c->use_graph = graph;
  int rc2 = sph_restore_state(c, slot);
  if (!rc) rc = rc2;
  rc2 = sph_drop_state(c, slot);
  if (!rc) rc = rc2;
  if (!rc) rc = sph_set_launch(c, best);
  if (rc) return rc;
  if (block_out)
    for (int q = 0; q < 4; ++q) block_out[q] = best[q];
  if (cache_path) {
    std::ofstream o(cache_path, std::ios::app);
    if (o) o << key << " " << best[0] << " " << best[1] << " " << best[2] << " " << best[3] << "\n";
  }
  return SPH_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------
// field transfer
// ------------------------------------------------------------------------
struct LiveView {
  std::vector<int64_t> rows;  // device index of each output row
};

static int live_rows(sph_ctx *c, LiveView &lv) {
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  Counters h;
  CUDA_TRY(cudaMemcpy(&h, c->cnt, sizeof(h), cudaMemcpyDeviceToHost));
  int64_t m = h.m_pending;
  std::vector<uint32_t> keys(m), uid(m);
  std::vector<uint16_t> inst(m);
  if (m) {
    CUDA_TRY(cudaMemcpy(keys.data(), c->K[0], 4 * m, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(uid.data(), c->M[c->cur].uid, 4 * m, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(inst.data(), c->M[c->cur].inst, 2 * m, cudaMemcpyDeviceToHost));
  }
  lv.rows.clear();
  for (int64_t i = 0; i < m; ++i)
    if (keys[i] != c->ncell) lv.rows.push_back(i);
  std::sort(lv.rows.begin(), lv.rows.end(), [&](int64_t a, int64_t b) {
    if (inst[a] != inst[b]) return inst[a] < inst[b];
    return uid[a] < uid[b];
  });
  return 0;
}

template <typename T>
static int pull(const T *dev, int64_t m, std::vector<T> &out) {
  out.resize((size_t)m);
  if (m) CUDA_TRY(cudaMemcpy(out.data(), dev, sizeof(T) * m, cudaMemcpyDeviceToHost));
  return 0;
}

static int store_out(void *dst, const void *src, size_t bytes, int on_device) {
  if (!dst) return fail(SPH_ERR_ARG, "destination array is NULL");
  if (bytes == 0) return 0;
  if (on_device) {
    CUDA_TRY(cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice));
  } else {
    memcpy(dst, src, bytes);
  }
  return 0;
}

extern "C" {

int sph_read_fields(sph_ctx *c, uint32_t mask, void *const *dst, int32_t dst_on_device, int64_t *n_out) {
  if (!c) return fail(SPH_ERR_ARG, "ctx is NULL");
  if (mask & ~SPH_F_ALL_READ) return fail(SPH_ERR_ARG, "unknown field bits");
  LiveView lv;
  int rc = live_rows(c, lv);
  if (rc) return rc;
  const int64_t n = (int64_t)lv.rows.size();
  if (n_out) *n_out = n;
  if (!dst) return SPH_OK;
  Counters h;
  CUDA_TRY(cudaMemcpy(&h, c->cnt, sizeof(h), cudaMemcpyDeviceToHost));
  const int64_t m = h.m_pending;
  const Masters &M = c->M[c->cur];
  int slot = 0;
  for (int bit = 0; bit < 15; ++bit) {
    uint32_t f = 1u << bit;
    if (!(mask & f)) continue;
    void *out = dst[slot++];
    if (f == SPH_F_POS || f == SPH_F_VEL || f == SPH_F_ACC_NU) {
      double *const *src = f == SPH_F_POS ? M.x : (f == SPH_F_VEL ? M.v : c->der.an);
      std::vector<double> comp[3], buf(3 * n);
      for (int a = 0; a < 3; ++a)
        if ((rc = pull(src[a], m, comp[a]))) return rc;
      for (int64_t r = 0; r < n; ++r)
        for (int a = 0; a < 3; ++a) buf[3 * r + a] = (a < c->dim) ? comp[a][lv.rows[r]] : 0.0;
      if ((rc = store_out(out, buf.data(), sizeof(double) * 3 * n, dst_on_device))) return rc;
    } else if (f == SPH_F_B) {
      std::vector<double> comp[6], buf(9 * n);
      for (int q = 0; q < 6; ++q)
        if ((rc = pull(c->der.B[q], m, comp[q]))) return rc;
      for (int64_t r = 0; r < n; ++r) {
        int64_t i = lv.rows[r];
        const bool d3 = c->dim == 3;  // a 2D step writes xx, yy, xy only
        double xx = comp[0][i], yy = comp[1][i], xy = comp[3][i];
        double zz = d3 ? comp[2][i] : 0.0, xz = d3 ? comp[4][i] : 0.0, yz = d3 ? comp[5][i] : 0.0;
        double B9[9] = {xx, xy, xz, xy, yy, yz, xz, yz, zz};
        memcpy(&buf[9 * r], B9, sizeof(B9));
      }
      if ((rc = store_out(out, buf.data(), sizeof(double) * 9 * n, dst_on_device))) return rc;
    } else if (f == SPH_F_LABEL || f == SPH_F_UID) {
      std::vector<uint32_t> v, buf(n);
      if ((rc = pull(f == SPH_F_LABEL ? (const uint32_t *)M.label : M.uid, m, v))) return rc;
      for (int64_t r = 0; r < n; ++r) buf[r] = v[lv.rows[r]];
      if ((rc = store_out(out, buf.data(), 4 * n, dst_on_device))) return rc;
    } else if (f == SPH_F_INST) {
      std::vector<uint16_t> v;
      std::vector<int32_t> buf(n);
      if ((rc = pull(M.inst, m, v))) return rc;
      for (int64_t r = 0; r < n; ++r) buf[r] = v[lv.rows[r]];
      if ((rc = store_out(out, buf.data(), 4 * n, dst_on_device))) return rc;
    } else if (f == SPH_F_KEY) {
      std::vector<uint32_t> v;
      std::vector<uint16_t> ins;
      std::vector<int64_t> buf(n);
      if ((rc = pull(c->K[0], m, v)) || (rc = pull(M.inst, m, ins))) return rc;
      for (int64_t r = 0; r < n; ++r) buf[r] = (int64_t)v[lv.rows[r]] - (int64_t)c->inst[ins[lv.rows[r]]].cell_base;
      if ((rc = store_out(out, buf.data(), 8 * n, dst_on_device))) return rc;
    } else {
      const double *src = nullptr;
      switch (f) {
        case SPH_F_RHO: src = M.rho; break;
        case SPH_F_MASS: src = M.mass; break;
        case SPH_F_DRHO: src = M.drho; break;
        case SPH_F_P: src = M.p; break;
        case SPH_F_K: src = M.k; break;
        case SPH_F_EPS: src = M.eps; break;
        case SPH_F_NUT: src = M.nut; break;
      }
      std::vector<double> v, buf(n);
      if ((rc = pull(src, m, v))) return rc;
      for (int64_t r = 0; r < n; ++r) buf[r] = v[lv.rows[r]];
      if ((rc = store_out(out, buf.data(), 8 * n, dst_on_device))) return rc;
    }
  }
  return SPH_OK;
}

int sph_write_fields(sph_ctx *c, uint32_t mask, const void *const *src, int32_t src_on_device, int64_t n) {
  if (!c || !src) return fail(SPH_ERR_ARG, "NULL argument");
  if (mask & ~SPH_F_ALL_WRITE) return fail(SPH_ERR_ARG, "only pos, vel, rho, mass, drho, k, eps are writable");
  LiveView lv;
  int rc = live_rows(c, lv);
  if (rc) return rc;
  if (n != (int64_t)lv.rows.size()) return fail(SPH_ERR_ARG, "row count differs from the live particle count");
  Counters h;
  CUDA_TRY(cudaMemcpy(&h, c->cnt, sizeof(h), cudaMemcpyDeviceToHost));
  const int64_t m = h.m_pending;
  const Masters &M = c->M[c->cur];
  int slot = 0;
  for (int bit = 0; bit < 15; ++bit) {
    uint32_t f = 1u << bit;
    if (!(mask & f)) continue;
    const void *in = src[slot++];
    if (!in) return fail(SPH_ERR_ARG, "source array is NULL");
    int width = (f == SPH_F_POS || f == SPH_F_VEL) ? 3 : 1;
    std::vector<double> hin((size_t)(width * n));
    if (n) {
      if (src_on_device)
        CUDA_TRY(cudaMemcpy(hin.data(), in, sizeof(double) * width * n, cudaMemcpyDeviceToHost));
      else
        memcpy(hin.data(), in, sizeof(double) * width * n);
    }
    if (width == 3) {
      double *const *dstv = f == SPH_F_POS ? M.x : M.v;
      for (int a = 0; a < 3; ++a) {
        std::vector<double> cur;
        if ((rc = pull(dstv[a], m, cur))) return rc;
        for (int64_t r = 0; r < n; ++r) cur[lv.rows[r]] = (a < c->dim) ? hin[3 * r + a] : 0.0;
        if (m) CUDA_TRY(cudaMemcpy(dstv[a], cur.data(), 8 * m, cudaMemcpyHostToDevice));
      }
    } else {
      double *dstp = nullptr;
      switch (f) {
        case SPH_F_RHO: dstp = M.rho; break;
        case SPH_F_MASS: dstp = M.mass; break;
        case SPH_F_DRHO: dstp = M.drho; break;
        case SPH_F_K: dstp = M.k; break;
        case SPH_F_EPS: dstp = M.eps; break;
      }
      std::vector<double> cur;
      if ((rc = pull(dstp, m, cur))) return rc;
      for (int64_t r = 0; r < n; ++r) cur[lv.rows[r]] = hin[r];
      if (m) CUDA_TRY(cudaMemcpy(dstp, cur.data(), 8 * m, cudaMemcpyHostToDevice));
    }
  }
  if (mask & SPH_F_POS) {
    launch_keys(c->topo(), (int)c->cap, 0, c->stream);
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    CUDA_TRY(cudaGetLastError());
  }
  return SPH_OK;
}

int sph_get_stats(sph_ctx *c, sph_stats *out) {
  if (!c || !out) return fail(SPH_ERR_ARG, "NULL argument");
  // two copies into pinned staging on the context's stream, one wait
  CUDA_TRY(cudaMemcpyAsync(&c->pin->cnt, c->cnt, sizeof(Counters), cudaMemcpyDeviceToHost, c->stream));
  // dt_ad, dt_ac, dt, t, n_ac are the trailing fields of the instance record
  const size_t tail = offsetof(InstDev, dt_ad);
  CUDA_TRY(cudaMemcpyAsync(c->pin->inst_tail + tail, (const char *)c->d_inst + tail, sizeof(InstDev) - tail,
                           cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  c->prof_collect();
  const Counters h = c->pin->cnt;
  InstDev i0;
  memcpy((char *)&i0 + tail, c->pin->inst_tail + tail, sizeof(InstDev) - tail);
  memset(out, 0, sizeof(*out));
  out->n = (int64_t)h.m_pending - (int64_t)h.n_del_step;
  out->step = c->step;
  out->t = i0.t;
  out->dt_ad = i0.dt_ad;
  out->dt_ac = i0.dt_ac;
  out->n_ac = i0.n_ac;
  out->n_instances = c->ninst;
  out->spawned = (int64_t)h.spawned;
  out->deleted = (int64_t)h.deleted;
  out->capacity = c->cap;
  out->device_bytes = (int64_t)c->bytes;
  out->kernel_launches = c->launches;
  out->status = h.status;
  return SPH_OK;
}

// bring the live particles into cell order, then restore a pending state
// equal to that order (keys sorted, identity indices), so that the next
// step sorts nothing new
static int debug_topology(sph_ctx *c) {
  if (!c->started) {
    int rc = upload_buffers(c);
    if (rc) return rc;
    c->started = true;
  }
  enqueue_topology(c);
  if (c->sorted_keys != c->K[0])
    CUDA_TRY(cudaMemcpyAsync(c->K[0], c->sorted_keys, 4 * (size_t)c->cap, cudaMemcpyDeviceToDevice, c->stream));
  c->sorted_keys = c->K[0];
  CUDA_TRY(cudaMemcpyAsync(&c->cnt->m_pending, &c->cnt->n_live, 4, cudaMemcpyDeviceToDevice, c->stream));
  launch_iota(c->Vv[0], (int)c->cap, c->stream);
  CUDA_TRY(cudaMemsetAsync(c->pair_counter, 0, 8, c->stream));
  return 0;
}

}  // extern "C"

// rows of a debug read: run `emit` into a temporary device buffer (test aid,
// not on the stepping path) and copy the first max rows out
template <typename F>
static int debug_rows(sph_ctx *c, int64_t *out, int64_t max, int64_t *count, const char *what, F &&emit) {
  int64_t *dout = nullptr;
  if (max > 0 && cudaMalloc(&dout, sizeof(int64_t) * 4 * (size_t)max) != cudaSuccess)
    return fail(SPH_ERR_ALLOC, std::string(what) + " buffer");
  emit(dout);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  unsigned long long n = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&n, c->pair_counter, 8, cudaMemcpyDeviceToHost);
  int64_t k = std::min<int64_t>((int64_t)n, max);
  if (e == cudaSuccess && dout && out && k > 0)
    e = cudaMemcpy(out, dout, sizeof(int64_t) * 4 * k, cudaMemcpyDeviceToHost);
  if (dout) cudaFree(dout);
  if (e != cudaSuccess) return fail(SPH_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  *count = (int64_t)n;
  return SPH_OK;
}

extern "C" {

int sph_debug_pairs(sph_ctx *c, int64_t *out, int64_t max, int64_t *count) {
  if (!c || !count) return fail(SPH_ERR_ARG, "NULL argument");
  int rc = debug_topology(c);
  if (rc) return rc;
  return debug_rows(c, out, max, count, "debug pairs", [&](int64_t *dout) {
    launch_debug_pairs(c->sweep(0, 0), c->wx[0], c->wx[1], c->wx[2], c->wall_index, dout, max, c->pair_counter,
                       (int)c->cap, c->stream);
  });
}

int sph_debug_list(sph_ctx *c, int64_t *out, int64_t max, int64_t *count) {
  if (!c || !count) return fail(SPH_ERR_ARG, "NULL argument");
  if (c->kinematic) return fail(SPH_ERR_STATE, "a kinematic context builds no neighbour list");
  int rc = debug_topology(c);
  if (rc) return rc;
  // the list builder of the stepping path, in the context's precision and
  // launch shape, without the time step its first block takes when stepping
  SweepArgs la = c->sweep(0, 0);
  la.with_time_step = 0;
  launch_neighbour_list(la, c->packs(), c->prec, c->dim, (int)c->cap, c->stream);
  rc = debug_rows(c, out, max, count, "debug list", [&](int64_t *dout) {
    launch_debug_list(c->sweep(0, 0), c->wall_index, dout, max, c->pair_counter, (int)c->cap, c->stream);
  });
  if (rc) return rc;
  int32_t status = 0;
  rc = read_status(c, &status);
  return rc ? rc : status;
}

}  // extern "C"

// ------------------------------------------------------------------------
// test aid: a grid barrier whose wait runs out
// ------------------------------------------------------------------------
namespace {
// every block waits at barrier 2 first, whose target (2 x gridDim.x
// arrivals) the launch never reaches: each wait ends at its poll limit or
// at the abort flag the first block to run out sets, then every block
// leaves, and the last one resets the barrier words
__global__ void k_barrier_timeout(sphk::GridBarrier *gb, int32_t *status, uint32_t spin_limit) {
  __shared__ int s_ok;
  sphk::grid_sync(gb, 2u, status, &s_ok, spin_limit);
  sphk::grid_leave(gb);
}
}  // namespace

extern "C" int sph_debug_barrier_timeout(sph_ctx *c, int32_t *status_out, uint32_t *words_after) {
  if (!c || !status_out) return fail(SPH_ERR_ARG, "NULL argument");
  int32_t *d_status = nullptr;
  if (cudaMalloc(&d_status, sizeof(int32_t)) != cudaSuccess) return fail(SPH_ERR_ALLOC, "status word");
  cudaError_t e = cudaMemsetAsync(d_status, 0, sizeof(int32_t), c->stream);
  if (e == cudaSuccess) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(2);
    cfg.blockDim = dim3(32);
    cfg.stream = c->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // a short limit: about 2^14 polls per wait
    e = cudaLaunchKernelEx(&cfg, k_barrier_timeout, c->gbar, d_status, 1u << 14);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  int32_t st = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&st, d_status, sizeof(st), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && words_after) e = cudaMemcpy(words_after, c->gbar, sizeof(sphk::GridBarrier), cudaMemcpyDeviceToHost);
  cudaFree(d_status);
  if (e != cudaSuccess) return fail(SPH_ERR_CUDA, std::string("debug barrier: ") + cudaGetErrorString(e));
  *status_out = st;
  return SPH_OK;
}

// ------------------------------------------------------------------------
// test aid: the integer-pipe binary64 <-> binary32 conversions
// ------------------------------------------------------------------------
namespace {
__global__ void k_debug_convert(const double *in64, float *out32, const float *in32, double *out64, int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  if (in64) out32[k] = f64_to_f32(in64[k]);
  if (in32) out64[k] = f32_to_f64(in32[k]);
}
}  // namespace

extern "C" int sph_debug_convert(const double *in64, float *out32, const float *in32, double *out64, int64_t n) {
  if (n < 0 || n > ((int64_t)1 << 24)) return fail(SPH_ERR_ARG, "n must be 0..2^24");
  if ((in64 && !out32) || (in32 && !out64)) return fail(SPH_ERR_ARG, "output missing");
  if (n == 0 || (!in64 && !in32)) return SPH_OK;
  // test aid, not on the stepping path: temporary device buffers
  char *d = nullptr;
  const size_t b8 = 8 * (size_t)n, b4 = 4 * (size_t)n;
  if (cudaMalloc(&d, 2 * (b8 + b4)) != cudaSuccess) return fail(SPH_ERR_ALLOC, "convert buffers");
  double *d_in64 = (double *)d, *d_out64 = (double *)(d + b8);
  float *d_in32 = (float *)(d + 2 * b8), *d_out32 = (float *)(d + 2 * b8 + b4);
  cudaError_t e = cudaSuccess;
  if (in64) e = cudaMemcpy(d_in64, in64, b8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && in32) e = cudaMemcpy(d_in32, in32, b4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_debug_convert<<<(unsigned)((n + 255) / 256), 256>>>(in64 ? d_in64 : nullptr, d_out32, in32 ? d_in32 : nullptr,
                                                           d_out64, n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && in64) e = cudaMemcpy(out32, d_out32, b4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && in32) e = cudaMemcpy(out64, d_out64, b8, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return fail(SPH_ERR_CUDA, cudaGetErrorString(e));
  return SPH_OK;
}

// ------------------------------------------------------------------------
// FP64 mass and momentum of every instance (deterministic order)
// ------------------------------------------------------------------------
namespace {
constexpr int kRedThreads = 256;

// blocks per instance: about two per SM in all.  Every FP64 operation is
// costly on this GPU (about 1.4 per clock and SM): with more, thinner
// blocks the shuffle trees that sum the threads outweigh the five
// operations per particle (1024 blocks: 32 us for 480k particles, FP64
// pipe 57 % busy).  Fixed per context (the first call), so the summation
// order is fixed too.
static int red_slices(int ninst) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
  cudaGetLastError();
  return std::max(1, (2 * sms + ninst - 1) / ninst);
}

// first index in [lo, hi) whose instance is >= q (instances non-decreasing
// there), found by the 32 lanes of a warp together: each round probes 32
// evenly spaced rows and keeps the interval between the last probe below q
// and the first at or above it, so a search over n rows takes about
// log32(n) dependent loads
__device__ int inst_lower_bound_warp(const uint16_t *inst, int lo, int hi, int q) {
  const int lane = threadIdx.x & 31;
  while (hi - lo > 32) {
    const int step = (hi - lo + 31) / 32;
    const int probe = lo + lane * step;
    const unsigned below = __ballot_sync(0xffffffffu, probe < hi && (int)inst[probe] < q);
    const int t = __popc(below);  // lanes 0 .. t-1 probe rows below q
    const int nlo = t == 0 ? lo : lo + (t - 1) * step + 1;
    const int nhi = t == 32 ? hi : min(hi, lo + t * step);
    lo = nlo;
    hi = nhi;
  }
  const int probe = lo + lane;
  const unsigned below = __ballot_sync(0xffffffffu, probe < hi && (int)inst[probe] < q);
  return lo + __popc(below);
}

// block (q, s): slice s of instance q's rows, which are one run in
// [0, n_live) (the sorted particles) and one in [n_live, m_pending) (the
// copies appended by the last buffer update); deleted rows carry the
// sentinel key.  Each thread sums a fixed strided subset (momentum by
// FMA), the block sums its threads in a fixed order (block_sum).  The last
// of an instance's blocks to finish then sums its slices in a fixed order
// (thread t takes slices t, t + 256, ... in turn, then the same block sum)
// into out[q][4] (instances in parallel; out may be page-locked host
// memory): the result does not depend on timing.
__global__ void __launch_bounds__(kRedThreads) k_reduce(Masters m, const uint32_t *keys, uint32_t sentinel,
                                                        const Counters *cnt, int dim, int slices, int ninst,
                                                        double *partial, uint32_t *done, double *out) {
  const int q = blockIdx.x / slices, sl = blockIdx.x % slices;
  const int n1 = cnt->n_live, n2 = cnt->m_pending;
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  __shared__ int s_r[4];
  __shared__ bool s_last;
  __shared__ double s_v[4][kRedThreads];
  __shared__ double s_w[4];
  if (ninst == 1) {
    // one instance: its rows are all of [0, n_live) and [n_live, m_pending)
    if (threadIdx.x < 4) s_r[threadIdx.x] = threadIdx.x < 2 ? (threadIdx.x == 0 ? 0 : n1) : (threadIdx.x == 2 ? n1 : n2);
  } else if (wq < 4) {
    // the four run bounds, one warp each
    const int lo = wq < 2 ? 0 : n1, hi = wq < 2 ? n1 : n2;
    const int r = inst_lower_bound_warp(m.inst, lo, hi, q + (wq & 1));
    if (lane == 0) s_r[wq] = r;
  }
  __syncthreads();
  const int a0 = s_r[0], la = s_r[1] - s_r[0], b0 = s_r[2], L = la + (s_r[3] - s_r[2]);
  const int64_t k0 = (int64_t)L * sl / slices, k1 = (int64_t)L * (sl + 1) / slices;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  // four rows per round, their loads issued together; a deleted row adds
  // nothing (its terms are skipped, not multiplied by zero)
  constexpr int U = 4;
  for (int64_t kb = k0 + threadIdx.x; kb < k1; kb += (int64_t)U * kRedThreads) {
    double mu[U], vu[U][3];
    bool live[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t k = kb + (int64_t)u * kRedThreads;
      const int i = k < k1 ? (k < la ? a0 + (int)k : b0 + (int)(k - la)) : 0;
      live[u] = k < k1 && keys[i] != sentinel;
      mu[u] = m.mass[i];
#pragma unroll
      for (int d = 0; d < 3; ++d) vu[u][d] = d < dim ? m.v[d][i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!live[u]) continue;
      acc[0] = sphk::dadd(acc[0], mu[u]);
      for (int d = 0; d < dim; ++d) acc[1 + d] = __fma_rn(mu[u], vu[u][d], acc[1 + d]);
    }
  }
  // the block's sum in a fixed order, one warp per component (every FP64
  // operation counts here): lane l sums threads l, l + 32, ..., l + 224 in
  // turn, then a shuffle tree over the lanes
  auto block_sum = [&]() {
    for (int c = 0; c < 4; ++c) s_v[c][threadIdx.x] = acc[c];
    __syncthreads();
    if (wq < 4) {
      double x = s_v[wq][lane];
#pragma unroll
      for (int k = 1; k < kRedThreads / 32; ++k) x = sphk::dadd(x, s_v[wq][lane + 32 * k]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x = sphk::dadd(x, __shfl_down_sync(0xffffffffu, x, o));
      if (lane == 0) s_w[wq] = x;
    }
    __syncthreads();
    if (threadIdx.x < 4) acc[threadIdx.x] = s_w[threadIdx.x];
  };
  block_sum();
  if (threadIdx.x < 4) {
    partial[(size_t)blockIdx.x * 4 + threadIdx.x] = acc[threadIdx.x];
    __threadfence();  // the partial is visible before the block counts itself done
  }
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&done[q], 1u) == (unsigned)slices - 1u;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int c = 0; c < 4; ++c) acc[c] = 0.0;
  for (int t = threadIdx.x; t < slices; t += kRedThreads)
    for (int c = 0; c < 4; ++c) acc[c] = sphk::dadd(acc[c], __ldcg(&partial[((size_t)q * slices + t) * 4 + c]));
  block_sum();
  if (threadIdx.x < 4) out[(size_t)q * 4 + threadIdx.x] = acc[threadIdx.x];
  if (threadIdx.x == 0) done[q] = 0u;
}
}  // namespace

// the reduction launch on the context's stream, results [ninst][4] (mass,
// momentum x y z) into out (device memory or page-locked host memory the
// device can address); NULL: the context's device result buffer, whose
// address *res receives
static int enqueue_mass_momentum(sph_ctx *c, double *out, double **res) {
  if (!c->red) c->red_slices = red_slices(c->ninst);
  const int slices = c->red_slices;
  if (!c->red) {
    // partial sums [ninst * slices][4], results [ninst][4] and the
    // instances' block completion counters, owned by the context from the
    // first call on
    const size_t words = 4 * ((size_t)c->ninst * slices + c->ninst) + ((size_t)c->ninst + 1) / 2;
    c->red = (double *)c->dalloc(sizeof(double) * words);
    if (!c->red) return fail(SPH_ERR_ALLOC, "reduction buffers");
    CUDA_TRY(cudaMemsetAsync(c->red, 0, sizeof(double) * words, c->stream));
  }
  double *partial = c->red;
  double *dres = c->red + 4 * (size_t)c->ninst * slices;
  uint32_t *done = reinterpret_cast<uint32_t *>(dres + 4 * (size_t)c->ninst);
  if (res) *res = dres;
  k_reduce<<<c->ninst * slices, kRedThreads, 0, c->stream>>>(c->M[c->cur], c->K[0], c->ncell, c->cnt, c->dim, slices,
                                                              c->ninst, partial, done, out ? out : dres);
  CUDA_TRY(cudaGetLastError());
  return 0;
}

extern "C" int sph_reduce_mass_momentum_async(sph_ctx *c, double *out) {
  if (!c || !out) return fail(SPH_ERR_ARG, "NULL argument");
  // page-locked host memory the device can write: the reduction's last
  // block writes the totals there; other memory takes a copy
  cudaPointerAttributes pa{};
  void *dev = nullptr;
  if (cudaPointerGetAttributes(&pa, out) == cudaSuccess &&
      (pa.type == cudaMemoryTypeHost || pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged))
    dev = pa.devicePointer;
  cudaGetLastError();
  double *res = nullptr;
  const int rc = enqueue_mass_momentum(c, (double *)dev, &res);
  if (rc) return rc;
  if (!dev)
    CUDA_TRY(cudaMemcpyAsync(out, res, sizeof(double) * 4 * (size_t)c->ninst, cudaMemcpyDeviceToHost, c->stream));
  return SPH_OK;
}

extern "C" int sph_reduce_mass_momentum(sph_ctx *c, double *mass, double *momentum) {
  if (!c || (!mass && !momentum)) return fail(SPH_ERR_ARG, "NULL argument");
  double *res = nullptr;
  const int rc = enqueue_mass_momentum(c, nullptr, &res);
  if (rc) return rc;
  std::vector<double> h(4 * (size_t)c->ninst);
  CUDA_TRY(cudaMemcpyAsync(h.data(), res, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  for (int q = 0; q < c->ninst; ++q) {
    if (mass) mass[q] = h[4 * (size_t)q];
    if (momentum)
      for (int d = 0; d < 3; ++d) momentum[3 * (size_t)q + d] = h[4 * (size_t)q + 1 + d];
  }
  return SPH_OK;
}
