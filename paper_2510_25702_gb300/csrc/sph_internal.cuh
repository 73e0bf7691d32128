// sph_internal.cuh -- device-side data layout and helpers of the GB300 SPH
// step library (the C ABI is include/sph.h).
//
// Layout in HBM (one context):
//  * master particle state, FP64 structure-of-arrays, two copies (the cell
//    sort gathers one into the other every advection step);
//  * per-sweep neighbour records in the sweep precision R (float or double):
//    one record per particle holding what one sweep reads of a neighbour,
//    written by the kernel that runs before that sweep (layout at Packs);
//  * sorted cell keys, cell offsets (exclusive prefix over all cells of
//    all instances) and the same for the fixed wall dummies;
//  * a device status word (first error wins) and counters.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sph.h"
#include "sph_grid.cuh"

namespace sphk {

constexpr uint32_t kSubRecycle = 0xFFFFFFFFu;
constexpr int kBlock = 128;     // topology kernels
constexpr int kMaxBlock = 256;  // largest block size of the sweeps

// k-epsilon constants (App. A table)
constexpr double kC1 = 1.44, kC2 = 1.92, kCmu = 0.09, kSigK = 1.0, kSigE = 1.3;
constexpr double kFloor = 1e-12;

// constants of the pair sweeps in the sweep precision, converted once on
// the host (the conversions match the ones the device would make)
template <typename R>
struct SweepConst {
  R L[3], g[3];
  R cut2, inv_h, c5, reg;  // c5 = -5 alpha_d / h^2: F = c5 (1 - q/2)^3
  R rho0, nu_l, c0, eta, muR_k, inv_c0sq, inv_rc0, c0sq;
};

struct InstDev {
  int32_t dim, rans, dt_mode, n_ac_fixed;
  int32_t kinematic;
  int32_t freeze_turb;  // k, eps, nu_t held (differentiated windows)
  int32_t periodic[3];
  int32_t nc[3];
  int32_t nbuf, buf0;
  uint32_t seed;
  uint32_t cell_base;  // first global cell key of this instance
  uint32_t ncell;
  int32_t obc;  // SPH_OBC_*: open-boundary treatment (Sec. 4.1 ablation cases)
  int32_t density_sum;  // density reinitialised by kernel summation each advection step
  int32_t tvf;          // transport-velocity shift on
  int32_t wall_fn;      // step-wise wall function at the walls (RANS)
  int32_t tvf_pbuf;     // the shift also moves pressure-buffer particles (across n_b)
  double wf_cmu34;      // C_mu^(3/4) of the wall value of eps
  double tvf_k;         // -2 alpha h^2: shift = tvf_k sum_j V_j grad_i W_ij
  double dsum_k;        // rho0 alpha_d / sigma_0: rho = dsum_k (1 + sum_j w^4 (5 - 4 w))
  double dp, h, rho0, c0, nu_l, eta, U_ref, dt_ad_fixed;
  double g[3], lo[3], hi[3], L[3];
  double cs;       // cell size 2h
  double cut2;     // (2h)^2
  double alpha_h;  // Wendland normalisation / h
  double Vw;       // wall dummy volume dp^dim
  double rc0;      // rho0 * c0
  double eos_k;    // rho0 * c0^2
  double muR_k;    // 0.5 * rho0 * h
  double reg;      // 0.01 h
  double inv_h;    // 1 / h
  double inv_cs;   // 1 / (2h)
  double inv_rc0;  // 1 / (rho0 c0)
  double c0sq;     // c0^2: p = c0^2 (rho - rho0), the stiff EOS of Sec. 2.1
  SweepConst<float> kf;
  SweepConst<double> kd;
  float lo_f[3], inv_cs_f;  // FP32 copies for the cell-index prefilter
  // FP32 form: record positions in fixed point, X = rint((x - lo) / q) with
  // q a power of two between dp 2^-20 and dp 2^-19 (int32 bit patterns in
  // the records), so that the difference of two positions and its FP32
  // value are exact: a pair vector is rounded only in its positions
  float fx_q;
  int32_t fx_Lu[3];   // periodic lengths in units of q
  double fx_inv_q;    // 1 / q
  // 1.5 2^52 - lo / q rounded to an integer (the encoding origin o = lo to
  // within q / 2): fma(x, 1 / q, fx_c) is 1.5 2^52 + X, X = round((x - o) / q)
  double fx_c[3];
  float fx_o[3];      // the origin o in FP32, for decoding
  // written every advection step by the time-step kernel
  double dt_ad, dt_ac, dt, t;
  int32_t n_ac;
  int32_t pad1;
};

template <typename R>
__host__ __device__ __forceinline__ const SweepConst<R> &sweep_const(const InstDev &I);
template <>
__host__ __device__ __forceinline__ const SweepConst<float> &sweep_const<float>(const InstDev &I) {
  return I.kf;
}
template <>
__host__ __device__ __forceinline__ const SweepConst<double> &sweep_const<double>(const InstDev &I) {
  return I.kd;
}

struct BufDev {
  int32_t type, turb, inst, local_id;
  double origin[3];
  double frame[9];
  double length, half[2];
  double p_ob, rho_ob, noise, k_in, eps_in, nut_in;
  double gen_line;  // length + 0.5 dp (Sec. 3.1)
  // FP32 bounding sphere of the box, widened for FP32 rounding (a point
  // outside it is outside the box; inside it the exact test decides)
  float cen[3], rad2;
  // the inlet profile, n_theta directly before theta so that one copy
  // moves both
  int32_t n_theta, pad0;
  double theta[SPH_MAX_THETA];
};

// master state (FP64 SoA)
struct Masters {
  double *x[3], *v[3];
  double *rho, *mass, *drho, *p, *k, *eps, *nut;
  int32_t *label;
  uint32_t *uid;
  uint16_t *inst;
};

// per-step derived masters (not permuted)
struct Derived {
  double *B[6];  // xx, yy, zz, xy, xz, yz
  double *an[3]; // viscous acceleration
};

template <typename R>
struct alignas(4 * sizeof(R)) V4 {
  R x, y, z, w;
};

// Neighbour records: what one sweep reads of a neighbour j, packed into
// RV consecutive 4-vectors (32 B per record in 2D FP32, one sector), so
// that a neighbour costs one gather.  Written by the kernel before the
// sweep that reads them:
//   adv  (permute -> advection sweep)   2D (x y V vx)(vy k eps nut)
//                                       3D (x y z V)(vx vy vz k), with
//                                          (eps nut - -) in adv_b
//   mom  (advection / continuity -> momentum)
//                                       2D (x y V p)(Bxx Bxy Byy kw)
//                                       3D (x y z V)(p kw Bxx Byy), with
//                                          (Bzz Bxy Bxz Byz) in mom_b: the
//                                          first 32 bytes stay one aligned
//                                          256-bit load and one sector
//   cont (momentum -> continuity)       2D (x y V p)(vx vy - -)
//                                       3D (x y z V)(p vx vy vz)
// kw = 2/3 k (effective pressure); Bxx < 0 marks a pressure-buffer
// particle whose neighbours use their own B (the condition B_k = B_i).
template <typename R>
struct Packs {
  V4<R> *adv, *mom, *cont;  // records, RV 4-vectors per particle
  V4<R> *lpos;              // FP32 form: (x y z 0) in FP32 for the list builder
  V4<R> *WPf;               // FP32 form: walls (x y z 0) in FP32 for the list builder
  V4<R> *mom_b;             // 3D: the momentum record's B tail (Bzz Bxy Bxz Byz)
  V4<R> *adv_b;             // 3D: the advection record's k-epsilon tail (eps nut - -)
  V4<R> *Ap;                // a_nu + g of the advection step
  V4<R> *WP, *WV;           // walls: (x, y, z, V) and (vx, vy, vz, 0)
};

template <int D>
struct RecLayout {
  static constexpr int adv = 2;
  static constexpr int mom = 2;
  static constexpr int cont = 2;
};

struct Counters {
  int32_t status;
  int32_t n_live;     // live real particles after the sort
  int32_t m_pending;  // entries to sort (live + spawned copies, deleted keyed out)
  int32_t n_spawn;    // copies appended by the last buffer update
  int32_t overflow;
  int32_t n_del_step;  // entries deleted by the last buffer update
  int32_t n_ac_all;    // largest sub-step count of any instance this step
  int32_t pad2;
  unsigned long long spawned, deleted;
  // advection steps completed (the Philox step counter of the boundary
  // noise); advanced by the buffer update, which keeps the index of the step
  // it closes in spawn_step for the recycled particles
  long long step, spawn_step;
};

// ------------------------------------------------------------------------
// exact FP64 operations for every floating-point decision that sets an
// integer (cell index, cut-off, box containment, generation line): no
// contraction, same operation order as the plain definition
// ------------------------------------------------------------------------
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }

// ------------------------------------------------------------------------
// binary64 <-> binary32 conversions with 32-bit integer operations.  On
// GB300 the conversion instructions issue on the FP64 pipe (a small
// fraction of the FP32 rate), and the FP32 form converts every field it
// gathers or writes back; these run on the integer pipe instead.  Both
// follow the IEEE 754 encodings (1 sign, 11 / 8 exponent bits with biases
// 1023 / 127, 52 / 23 fraction bits) and give the same results as the
// conversion instructions:
//  * binary64 -> binary32, round to nearest, ties to even: for a value in
//    the normal binary32 range the exponent is rebased by 1023 - 127 = 896
//    and the 52-bit fraction keeps its top 23 bits, plus one unit when the
//    29 dropped bits exceed half a unit or equal it with an odd result (a
//    carry into the exponent is the correct next binade, at the top the
//    correct overflow to infinity);
//  * binary32 -> binary64 is exact: exponent rebased, fraction shifted.
// Zeros take a direct path; subnormals, infinities and NaNs (rare here) use
// the conversion instruction.
// ------------------------------------------------------------------------
__device__ __forceinline__ float f64_to_f32(double d) {
  const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
  const uint32_t mag = hi & 0x7FFFFFFFu;
  const uint32_t e = mag >> 20;
  if (e - 897u > 253u) {  // binary32 exponent field outside 1..254
    if ((mag | lo) == 0u) return __uint_as_float(hi);  // +-0
    return __double2float_rn(d);
  }
  uint32_t f = ((mag - (896u << 20)) << 3) | (lo >> 29);
  const uint32_t rem = lo & 0x1FFFFFFFu;
  f += (uint32_t)(rem > 0x10000000u) | ((uint32_t)(rem == 0x10000000u) & f);
  return __uint_as_float(f | (hi & 0x80000000u));
}

__device__ __forceinline__ double f32_to_f64(float x) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t mag = u & 0x7FFFFFFFu;
  const uint32_t e = mag >> 23;
  if (e - 1u > 253u) {  // zero, subnormal, infinity, NaN
    if (mag == 0u) return __hiloint2double((int)u, 0);  // +-0
    return (double)x;
  }
  return __hiloint2double((int)((u & 0x80000000u) | ((mag >> 3) + (896u << 20))), (int)(u << 29));
}

// fixed-point record coordinate of x along axis a (FP32 form): the integer
// X nearest to (x - o) / q, modulo 2^32 (a difference of two coordinates is
// exact modulo 2^32 all the same), as a float bit pattern.  One FMA: q being
// a power of two, x / q is exact and the sum with fx_c is rounded once, to
// an integer (its magnitude lies in [2^52, 2^53)), whose bit pattern is that
// of 1.5 2^52 (low word 0) plus X while |X| < 2^51
__device__ __forceinline__ float fx_encode(const InstDev &I, double x, int a) {
  return __int_as_float(__double2loint(__fma_rn(x, I.fx_inv_q, I.fx_c[a])));
}

// conversions into and out of the sweep precision R
template <typename R>
__device__ __forceinline__ R to_R(double d) {
  if constexpr (sizeof(R) == 4)
    return f64_to_f32(d);
  else
    return d;
}
template <typename R>
__device__ __forceinline__ double from_R(R x) {
  if constexpr (sizeof(R) == 4)
    return f32_to_f64(x);
  else
    return x;
}

// floor((x - lo) / (2h)) with the correctly rounded quotient, clamped.  The
// product with 1/(2h) is within 3.4e-10 cells of that quotient for grids of
// up to 1e6 cells per axis, so when it lies more than 1e-9 away from an
// integer both have the same floor; only then is the division skipped.
__device__ __forceinline__ int32_t cell_coord(const InstDev &I, double x, int a) {
  const double t = dsub(x, I.lo[a]);
  const double qa = dmul(t, I.inv_cs);
  double f = floor(qa);
  const double frac = qa - f;
  if (!(frac > 1e-9 && frac < 1.0 - 1e-9)) f = floor(ddiv(t, I.cs));
  if (!(f >= 0.0)) return 0;
  if (f >= (double)I.nc[a]) return I.nc[a] - 1;
  return (int32_t)f;
}

// the same cell index from an FP32 estimate of (x - lo) / (2h) where that
// estimate lies farther from a cell boundary than its rounding error can
// reach (then both floors agree); the exact FP64 path otherwise.  The bound
// adds the FP32 roundings of x, lo, their difference, 1/(2h) and the
// product, with a factor 2 to spare.
__device__ __forceinline__ int32_t cell_coord_fast(const InstDev &I, double x, int a) {
  const float xf = (float)x, lof = I.lo_f[a], ics = I.inv_cs_f;
  const float q = (xf - lof) * ics;
  const float fq = floorf(q), fr = q - fq;
  const float err = (fabsf(xf) + fabsf(lof)) * 1.2e-7f * ics + fabsf(q) * 4.8e-7f + 1e-6f;
  if (q >= 0.0f && q < (float)I.nc[a] && fr > err && fr < 1.0f - err) return (int32_t)fq;
  return cell_coord(I, x, a);
}

__device__ __forceinline__ uint32_t cell_key(const InstDev &I, double x, double y, double z) {
  uint32_t cx = (uint32_t)cell_coord_fast(I, x, 0);
  uint32_t cy = (uint32_t)cell_coord_fast(I, y, 1);
  uint32_t cz = I.dim == 3 ? (uint32_t)cell_coord_fast(I, z, 2) : 0u;
  return I.cell_base + (cz * (uint32_t)I.nc[1] + cy) * (uint32_t)I.nc[0] + cx;
}

// buffer-local coordinate k: (x - o) . frame row k, left-to-right sum
__device__ __forceinline__ double local_coord(const BufDev &b, int dim, double x, double y, double z, int k) {
  const double *f = &b.frame[3 * k];
  double s = dmul(dsub(x, b.origin[0]), f[0]);
  s = dadd(s, dmul(dsub(y, b.origin[1]), f[1]));
  if (dim == 3) s = dadd(s, dmul(dsub(z, b.origin[2]), f[2]));
  return s;
}

// region-constrained containment (Sec. 3.2)
__device__ __forceinline__ bool box_contains(const BufDev &b, int dim, double x, double y, double z) {
  double s0 = local_coord(b, dim, x, y, z, 0);
  if (!(s0 >= 0.0 && s0 < b.length)) return false;
  double s1 = local_coord(b, dim, x, y, z, 1);
  if (!(fabs(s1) <= b.half[0])) return false;
  if (dim == 3) {
    double s2 = local_coord(b, dim, x, y, z, 2);
    if (!(fabs(s2) <= b.half[1])) return false;
  }
  return true;
}

// Philox4x32-10 (Salmon et al., SC'11)
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
    uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
    uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// 53-bit uniform in [-1, 1) from two words (top 27 + 26 bits)
__device__ __forceinline__ double uniform_pm1(uint32_t a, uint32_t b) {
  double m = dadd(dmul((double)(a >> 5), 67108864.0), (double)(b >> 6));
  return dsub(dmul(2.0, dmul(m, 1.0 / 9007199254740992.0)), 1.0);
}

__device__ __forceinline__ void set_status(int32_t *status, int32_t code) {
  atomicCAS(status, 0, code);
}

// a4 dual-criteria time step of one instance (Sec. 2.3): advection step
// from max |v| (or U_ref) and the viscous limit with nu_l + max nu_t,
// acoustic step from c0 + max |v|, sub-step count ceil(dt_ad / dt_ac)
// (fixed or single-step modes override); folds the count into n_ac_all
struct StepArgs {
  InstDev *inst;
  const unsigned long long *v2max, *nutmax;  // per instance, from the permute
  Counters *cnt;
  int32_t ninst, n_ac_max;
};

__device__ __forceinline__ void time_step_instance(const StepArgs &a, int ii) {
  InstDev &I = a.inst[ii];
  double v2max = __longlong_as_double((long long)a.v2max[ii]);
  double nutmax = __longlong_as_double((long long)a.nutmax[ii]);
  double vmax = __dsqrt_rn(v2max);
  double u = (vmax > I.U_ref) ? vmax : I.U_ref;
  double dt_adv = ddiv(dmul(0.25, I.h), u);
  double nu_eff = dadd(I.nu_l, nutmax);
  double dt_visc = ddiv(dmul(dmul(0.125, I.h), I.h), nu_eff);
  double dt_ad = (dt_adv < dt_visc) ? dt_adv : dt_visc;
  double dt_ac = ddiv(dmul(0.6, I.h), dadd(I.c0, vmax));
  int n;
  if (I.dt_mode == SPH_DT_FIXED) {
    dt_ad = I.dt_ad_fixed;
    n = I.n_ac_fixed;
  } else if (I.dt_mode == SPH_DT_SINGLE) {
    if (dt_ac < dt_ad) dt_ad = dt_ac;
    n = 1;
  } else {
    double f = ceil(ddiv(dt_ad, dt_ac));
    n = (f >= 1.0) ? (int)fmin(f, 1.0e9) : 1;
  }
  if (n > a.n_ac_max) {
    set_status(&a.cnt->status, SPH_ERR_STATE);
    n = a.n_ac_max;
  }
  I.dt_ad = dt_ad;
  I.dt_ac = dt_ac;
  I.n_ac = n;
  I.dt = ddiv(dt_ad, (double)n);
  I.t = dadd(I.t, dt_ad);
  atomicMax(&a.cnt->n_ac_all, n);
}

// velocity-profile value at transverse coordinate s1 (linear in theta)
__device__ __forceinline__ double profile_U(const BufDev &b, double s1) {
  if (b.n_theta <= 1) return b.theta[0];
  double w = b.half[0];
  double u = dmul(ddiv(dadd(s1, w), dmul(2.0, w)), (double)(b.n_theta - 1));
  if (!(u > 0.0)) return b.theta[0];
  if (u >= (double)(b.n_theta - 1)) return b.theta[b.n_theta - 1];
  int k = (int)floor(u);
  double f = dsub(u, (double)k);
  return dadd(b.theta[k], dmul(f, dsub(b.theta[k + 1], b.theta[k])));
}

// Buffer boundary values on particle i (Sec. 2.4.2, buffer table of
// Sec. 4.3), in the plain operation order (no contraction).
__device__ __forceinline__ void apply_bc(const InstDev &I, const BufDev &b, const Masters &m, int i,
                                         int64_t step, uint32_t sub) {
  if (b.type == SPH_BUF_VELOCITY) {
    double s1 = local_coord(b, I.dim, m.x[0][i], m.x[1][i], I.dim == 3 ? m.x[2][i] : 0.0, 1);
    double U = profile_U(b, s1);
    double xi[3] = {0.0, 0.0, 0.0};
    if (b.noise != 0.0) {
      uint32_t c[4] = {(uint32_t)step, sub, 0u, 0u};
      philox4x32_10(c, I.seed, m.uid[i]);
      xi[0] = uniform_pm1(c[0], c[1]);
      xi[1] = uniform_pm1(c[2], c[3]);
      if (I.dim == 3) {
        uint32_t c2[4] = {(uint32_t)step, sub, 1u, 0u};
        philox4x32_10(c2, I.seed, m.uid[i]);
        xi[2] = uniform_pm1(c2[0], c2[1]);
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (a < I.dim) m.v[a][i] = dadd(dmul(U, b.frame[a]), dmul(dmul(b.noise, U), xi[a]));
  } else {
    m.p[i] = b.p_ob;
    m.rho[i] = b.rho_ob;
  }
  if (I.rans && !I.freeze_turb && b.turb == SPH_TURB_FREESTREAM) {
    m.k[i] = b.k_in;
    m.eps[i] = b.eps_in;
    m.nut[i] = b.nut_in;
  }
}

// record msg as this thread's sph_last_error() message and return code
int set_error(int code, const char *msg);

// ------------------------------------------------------------------------
// host-side launch wrappers implemented in the .cu files
// ------------------------------------------------------------------------
struct SortTemp {
  uint32_t *hist;  // digit histograms [1 << digit bits][tiles] + scan chunk totals
  int max_blocks;
};


// radix sort of (keys, vals) over *d_count entries (device count); bits of
// key to sort; results in keys_out / vals_out.  Uses keys_tmp/vals_tmp.
void radix_sort(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                const int32_t *d_count, int max_count, int bits, const SortTemp &tmp,
                cudaStream_t st, uint32_t **keys_result, uint32_t **vals_result);
// cell offsets (lower bounds) for cells [0, ncell] over sorted keys
void cell_offsets(const uint32_t *keys, const int32_t *d_count, uint32_t ncell, uint32_t *off,
                  int32_t *d_nlive, cudaStream_t st);

// The cell sort of the stepping path: one cooperative launch that sorts
// (key, index) pairs stably by key, writes the count of keys below the
// sentinel and zeroes two optional word ranges.  The plan fixes the digit
// width, the passes and the grid (co-resident blocks); scratch holds
// cell_sort_words(plan) words, zeroed once when allocated.
constexpr int kCellSortBlocksPerSm = 1;
struct CellSortPlan {
  int rb, passes, grid;
};
int cell_sort_plan(int bits, CellSortPlan *plan);
size_t cell_sort_words(const CellSortPlan &plan);
struct ClearSpans {
  uint32_t *p[3];  // word ranges the sort launch zeroes (NULL: unused)
  int n[3];
};
void cell_sort(const CellSortPlan &plan, uint32_t *scratch, uint32_t *keys[2], uint32_t *vals[2],
               const int32_t *d_count, int max_count, uint32_t sentinel, int32_t *d_below, int32_t *status,
               const ClearSpans &clear, cudaStream_t st, uint32_t **keys_result, uint32_t **vals_result);

struct TopoArgs {
  const InstDev *inst;
  const BufDev *buf;
  Masters src, dst;
  Derived der;
  uint32_t *keys, *idx;
  const uint32_t *sorted_vals;
  const uint32_t *sorted_keys;  // permute: keys in sorted order, for the cell offsets
  uint32_t *off;                // permute: cell offsets out (NULL: not written)
  int32_t carry_p;              // permute: move the pressure master (kinematic stepping)
  Counters *cnt;
  unsigned long long *v2max, *nutmax;  // per instance
  uint32_t *next_uid;                  // per instance
  int32_t *inst_spawn;                 // per instance spawn counts / bases
  uint8_t *flag;
  int32_t *block_cnt;
  uint32_t sentinel;
  int32_t ninst, n_ac_max;
  int64_t capacity;
  int32_t *spawn_dst;  // optional: index of the copy each injecting particle made
};

void launch_permute(const TopoArgs &a, int max_n, int prec, cudaStream_t st, void *packs);
void launch_time_step(const TopoArgs &a, cudaStream_t st);
StepArgs step_args(const TopoArgs &a);  // the time-step fields of a
// flags_done: the continuity sweep already wrote the flags, the per-instance
// inject counts and the per-128-block inject counts (zeroed by the sort)
void launch_buffer_update(const TopoArgs &a, int max_n, int flags_done, cudaStream_t st);

// buffer-update flag of a particle (inject / delete / keep), Sec. 2.4.2,
// 2.4.3, 3.1: inject when its local x'_0 has crossed the generation line
// L_b + 0.5 dp, delete when x'_0 < 0 (behind the buffer)
enum : uint8_t { kKeep = 0, kInject = 1, kDelete = 2 };
__device__ __forceinline__ uint8_t buffer_flag(const BufDev &B, int dim, double x, double y, double z) {
  const double x0 = local_coord(B, dim, x, y, z, 0);
  return x0 >= B.gen_line ? kInject : (x0 < 0.0 ? kDelete : kKeep);
}
void launch_keys(const TopoArgs &a, int max_n, int all_live, cudaStream_t st);
void launch_iota(uint32_t *idx, int max_n, cudaStream_t st);

// Neighbour list of the frozen configuration (rebuilt every advection
// step), in warp tiles of 4-entry chunks: the entries of the 32 particles of
// warp tile w form one contiguous block; in it, chunk c (entries 4c..4c+3)
// of lane l is the 16-byte word at (c * 32 + l), so a warp reads four
// entries of all its particles with one 512-byte load and its whole list is
// one contiguous range.  The n_real[i] real neighbours come first, then
// n_wall[i] wall dummies; rows[w] is the longest list of tile w (the part
// worth prefetching).
struct NbrList {
  uint32_t *nbr;
  uint16_t *n_real, *n_wall;
  uint16_t *rows;
  int32_t stride;  // particle capacity
  int32_t kmax;    // entries per particle, a multiple of 8
};

constexpr int kListTile = 32;

// first entry of particle i; entry k is at list_at(p, k)
__host__ __device__ __forceinline__ uint32_t *list_of(const NbrList &nl, int i) {
  return nl.nbr + ((size_t)(i / kListTile) * (size_t)(nl.kmax / 4) * kListTile + (size_t)(i % kListTile)) * 4;
}
__host__ __device__ __forceinline__ size_t list_off(int k) { return (size_t)(k >> 2) * (4 * kListTile) + (k & 3); }
__device__ __forceinline__ uint32_t list_at(const uint32_t *p, int k) { return p[list_off(k)]; }
// chunk c (entries 4c..4c+3) of the particle whose first entry is p
__device__ __forceinline__ uint4 list_chunk(const uint32_t *p, int c) {
  return reinterpret_cast<const uint4 *>(p)[(size_t)c * kListTile];
}

// asynchronous L2 prefetch of the list tile that particle i belongs to
__device__ __forceinline__ void prefetch_list_tile(const NbrList &nl, int i) {
  const int w = i / kListTile;
  const unsigned rows = nl.rows[w];
  if (rows == 0) return;
  const uint32_t *p = nl.nbr + (size_t)w * (size_t)nl.kmax * kListTile;
  const unsigned bytes = ((rows + 3u) / 4u) * kListTile * 16u;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

struct SweepArgs {
  const InstDev *inst;
  const BufDev *buf;
  Masters m;
  Derived der;
  NbrList nl;
  const uint32_t *keys;  // sorted cell keys of the live particles
  const uint32_t *off;   // cell offsets
  const uint32_t *woff;  // wall cell offsets
  const Counters *cnt;
  int32_t *status;
  int32_t sub;
  int32_t any_periodic;  // some instance has a periodic axis
  int32_t any_extra;     // some instance takes the transport shift or the density reinitialisation
  int32_t block;         // threads per block of the launch
  double *tape_S;        // optional: momentum sums S1, Cb, S2, Ct per sub-step
  StepArgs ts;           // list builder: time step of every instance by block 0
  int32_t with_time_step;
  // continuity sweep, last sub-step of an instance: the buffer-update flags
  // of its particles (NULL flag: the buffer update computes them)
  uint8_t *flag;
  int32_t *inst_spawn, *block_cnt;
  GridBarrier *gbar;     // sub-step launch: grid barrier words (zeroed once)
  const double *wx[3];   // FP64 wall positions in wall cell order (FP32 list: the
                         // exact test of candidates near the cut-off)
};

// sweeps: prec 0 -> double packs, 1 -> float packs; dim 2 / 3
void launch_neighbour_list(const SweepArgs &a, void *packs, int prec, int dim, int max_n, cudaStream_t st);
void launch_advection_sweep(const SweepArgs &a, void *packs, int prec, int dim, int max_n,
                            cudaStream_t st);
void launch_momentum_sweep(const SweepArgs &a, void *packs, int prec, int dim, int max_n, int sub,
                           cudaStream_t st);
void launch_continuity_sweep(const SweepArgs &a, void *packs, int prec, int dim, int max_n, int sub,
                             cudaStream_t st);
// acoustic sub-steps 1 .. n_ac_all - 1 (momentum, continuity) in one
// cooperative launch that ends at once when no instance takes them (2D
// contexts; 3D contexts launch the two sweeps per sub-step)
void launch_substeps(const SweepArgs &a, void *packs, int prec, int dim, int max_n, cudaStream_t st);
// ------------------------------------------------------------------------
// adjoint of the step (differentiated windows, FP64 contexts)
// ------------------------------------------------------------------------
// What the reverse pass needs of one advection step, recorded while the
// step is recomputed: the start-of-step state in cell order, per sub-step
// the density of the first half, the velocity after the kick, the position
// at the boundary-value time and the continuity rate, the sort permutation
// and the copies of the buffer update.
struct AdjTape {
  double *x0[3], *v0[3], *rho0, *drho0;
  double *S;  // momentum sums [sub][12][cap]: S1, Cb, S2, Ct
  double *rho_s, *drho_s, *v1[3], *xbc[3];  // [sub * cap + i]
  uint32_t *perm;                           // cell-order index -> pending index
  int32_t *spawn_dst;                       // injecting particle -> its copy
  int64_t cap;
};

struct AdjArgs {
  const InstDev *inst;
  const BufDev *buf;
  Masters m;    // masters after the recomputed step (cell order of the step)
  Derived der;  // B and viscous acceleration of the step
  NbrList nl;
  const uint32_t *off, *woff, *pending_keys;
  const double *wx[3];
  const V4<double> *WV;  // wall velocities
  const Counters *cnt;
  const uint8_t *flag;  // buffer-update decisions of the step
  AdjTape T;
  double *lx[3], *lv[3], *lrho, *ldrho;  // adjoint of the particle state
  double *lxg[3];                        // adjoint of the start position (pair geometry)
  double *lxs[3], *lrhos;                // mirror-term contributions (scattered)
  double *lB[6], *lan[3];
  double *sd[12];                        // per-particle scratch of one pair reverse
  V4<double> *rc, *rm, *rs, *ra;         // per-particle records of the pair reverses
  double *out[8];                        // pending-order result of the permutation reverse
  double *grad;                          // dJ/dtheta
  double *J;                             // objective accumulator
  const uint8_t *region;                 // per uid of the objective instance: buffer + 1
  int64_t n_region;
  int32_t g_inst, g_buf, o_inst;
  int32_t sub;
  uint32_t sentinel;
  double w_s, dt_obj;
};

void launch_adj_tape_start(const AdjArgs &a, int max_n, cudaStream_t st);
void launch_adj_tape_sub(const AdjArgs &a, int sub, int max_n, cudaStream_t st);
void launch_adj_tape_drho(const AdjArgs &a, int sub, int max_n, cudaStream_t st);
void launch_adj_region(const AdjArgs &a, uint8_t *region, const int32_t *obj_buf_mask, int max_n,
                       cudaStream_t st);
void launch_adj_objective(const AdjArgs &a, int seed, int max_n, cudaStream_t st);
void launch_adj_buffer_rev(const AdjArgs &a, int max_n, cudaStream_t st);
void launch_adj_substep_rev(const AdjArgs &a, int dim, int any_periodic, int sub, int max_n, cudaStream_t st);
void launch_adj_adv_rev(const AdjArgs &a, int dim, int any_periodic, int max_n, cudaStream_t st);
void launch_adj_perm_rev(const AdjArgs &a, int max_n, cudaStream_t st);

void launch_debug_list(const SweepArgs &a, const uint32_t *wall_index, int64_t *out, int64_t max,
                       unsigned long long *counter, int max_n, cudaStream_t st);
void launch_debug_pairs(const SweepArgs &a, const double *wx, const double *wy, const double *wz,
                        const uint32_t *wall_index, int64_t *out, int64_t max, unsigned long long *counter,
                        int max_n, cudaStream_t st);

}  // namespace sphk
