// sph_pair.cuh -- pair geometry and small linear algebra shared by the
// forward sweeps and their adjoint: exact/fast arithmetic per precision,
// the Wendland C2 kernel factor, minimum-image pair vectors, cell-range
// visiting, symmetric 2x2 / 3x3 helpers and the guarded inverse of B.
#pragma once

#include "sph_internal.cuh"

namespace sphk {

// A neighbour's two consecutive record 4-vectors.  FP32: one 256-bit load
// (the 32 bytes start on a 32-byte boundary: record arrays are 256-byte
// aligned and the record stride is 32 bytes), so that a scattered gather
// costs one L1 wavefront per lane instead of two.  Not volatile: the
// address depends on a list entry loaded after any barrier that orders the
// record's writes.  FP64 records (64 bytes) keep plain vector loads.
template <typename R>
__device__ __forceinline__ void ld_rec2(const V4<R> *p, V4<R> &a, V4<R> &b) {
  a = p[0];
  b = p[1];
}
template <>
__device__ __forceinline__ void ld_rec2<float>(const V4<float> *p, V4<float> &a, V4<float> &b) {
  asm("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
      : "l"(p));
}

template <typename R>
struct Ex;
template <>
struct Ex<double> {
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double div(double a, double b) { return a / b; }
  static __device__ __forceinline__ void len(double rr, double &r) { r = sqrt(rr); }
  // 1 / |r| given |r|^2 and |r|
  static __device__ __forceinline__ double inv_len(double rr, double r) { return 1.0 / r; }
};
template <>
struct Ex<float> {
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
  static __device__ __forceinline__ void len(float rr, float &r) { r = rr * rsqrtf(rr); }
  // 1 / |r| given |r|^2 and |r|: the reciprocal square root len already took
  static __device__ __forceinline__ float inv_len(float rr, float r) { return rsqrtf(rr); }
};

template <typename R>
struct Geo;
template <typename R, int D, bool PER>
__device__ __forceinline__ R pair_vec_abs(const Geo<R> &g, const V4<R> &pi, const V4<R> &pj, R d[3]);

// per-thread copy of the instance geometry in sweep precision
template <typename R>
struct Geo {
  R L[3];
  int per[3];
  R cut2, inv_h, c5, reg;
  R q;        // FP32 form: the fixed-point unit of the record positions
  int Lu[3];  // FP32 form: periodic lengths in units
};

template <typename R, int D>
__device__ __forceinline__ Geo<R> make_geo(const InstDev &I) {
  const SweepConst<R> &k = sweep_const<R>(I);
  Geo<R> g;
  for (int a = 0; a < 3; ++a) {
    g.L[a] = k.L[a];
    g.per[a] = (a < D) ? I.periodic[a] : 0;
    g.Lu[a] = I.fx_Lu[a];
  }
  g.cut2 = k.cut2;
  g.inv_h = k.inv_h;
  g.c5 = k.c5;
  g.reg = k.reg;
  g.q = (R)I.fx_q;
  return g;
}

// r_ij = x_i - x_j (minimum image when PER) from the leading 4-vectors of two
// records, whose first D components are the position; returns |r_ij|^2.
// FP64 form: FP64 positions, the plain left-to-right sum without
// contraction.  FP32 form: fixed-point positions; the difference of the two
// integers is exact (wrapped by the periodic length in units), and for a
// listed pair (|r| < 2h, under 2^22 units) it converts to FP32 exactly by the
// 2^23 + 2^22 offset; q being a power of two, the component di q comes out
// of one FMA exactly, and the sum of squares is contracted.
template <typename R, int D, bool PER>
__device__ __forceinline__ R pair_vec(const Geo<R> &g, const V4<R> &pi, const V4<R> &pj, R d[3]) {
  if constexpr (sizeof(R) == 4) {
    const float xi[3] = {pi.x, pi.y, pi.z}, xj[3] = {pj.x, pj.y, pj.z};
    float rr = 0.0f;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      int di = __float_as_int(xi[a]) - __float_as_int(xj[a]);
      if (PER && g.per[a]) {
        const int hu = g.Lu[a] >> 1;
        if (di > hu)
          di -= g.Lu[a];
        else if (di < -hu)
          di += g.Lu[a];
      }
      // q is a power of two: f q - (2^23 + 2^22) q = di q exactly, one FMA
      const float v = fmaf(__int_as_float(0x4B400000 + di), (float)g.q, -12582912.0f * (float)g.q);
      d[a] = (R)v;
      rr = (a == 0) ? v * v : fmaf(v, v, rr);
    }
    if (D == 2) d[2] = (R)0;
    return (R)rr;
  } else {
    return pair_vec_abs<R, D, PER>(g, pi, pj, d);
  }
}

// the absolute coordinate of axis a of a record position (the FP32 form
// decodes its fixed point; the FP64 form stores it)
template <typename R>
__device__ __forceinline__ R rec_abs(const InstDev &I, R x, int a) {
  if constexpr (sizeof(R) == 4)
    return I.fx_o[a] + (float)__float_as_int(x) * I.fx_q;
  else
    return x;
}

// r_ij = x_i - x_j (minimum image when PER) from absolute positions in R,
// |r_ij|^2 summed left to right (FP32: contracted); the list builder's
// candidate test in both forms and the FP64 form's pair vector
template <typename R, int D, bool PER>
__device__ __forceinline__ R pair_vec_abs(const Geo<R> &g, const V4<R> &pi, const V4<R> &pj, R d[3]) {
  R xi[3] = {pi.x, pi.y, pi.z}, xj[3] = {pj.x, pj.y, pj.z};
  R rr = (R)0;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    R v = Ex<R>::sub(xi[a], xj[a]);
    if (PER && g.per[a]) {
      R h = (R)0.5 * g.L[a];
      if (v > h)
        v = Ex<R>::sub(v, g.L[a]);
      else if (v < -h)
        v = Ex<R>::add(v, g.L[a]);
    }
    d[a] = v;
    if (sizeof(R) == 4)
      rr = (a == 0) ? v * v : fmaf((float)v, (float)v, (float)rr);  // FP32: contracted
    else
      rr = (a == 0) ? Ex<R>::mul(v, v) : Ex<R>::add(rr, Ex<R>::mul(v, v));
  }
  if (D == 2) d[2] = (R)0;
  return rr;
}

// volume slot of a record's leading 4-vector: (x y V .) in 2D, (x y z V) in 3D
template <typename R, int D>
__device__ __forceinline__ R vol(const V4<R> &r0) {
  return (D == 2) ? r0.z : r0.w;
}

// Wendland C2 (Sec. 2.2 kernel, support 2h): F = (dW/dr) / r
// = -5 (alpha / h^2) (1 - q/2)^3, evaluated without a division
template <typename R>
__device__ __forceinline__ R kernel_F(const Geo<R> &g, R r) {
  R w = (R)1 - (R)0.5 * (r * g.inv_h);
  return g.c5 * w * w * w;
}

// Wendland C2 divided by its normalisation, W / alpha_d = w^4 (1 + 2q) with
// w = 1 - q/2, i.e. w^4 (5 - 4w) (1 at r = 0)
template <typename R>
__device__ __forceinline__ R kernel_u(const Geo<R> &g, R r) {
  const R w = (R)1 - (R)0.5 * (r * g.inv_h);
  const R w2 = w * w;
  return w2 * w2 * ((R)5 - (R)4 * w);
}

// Friction velocity of the step-wise (two-layer) wall law for the
// tangential speed ut at wall distance y (FP64): the viscous sublayer
// ut = u_tau^2 y / nu while y+ = u_tau y / nu <= 11.225, else the log law
// ut = (u_tau / kappa) ln(E y u_tau / nu) by 8 Newton steps from the
// sublayer value (the residual is convex and increasing in u_tau and that
// value lies below its root); kappa = 0.4187 and E = 9.793 make the two
// laws meet at y+ = 11.225
constexpr double kWfKappa = 0.4187, kWfE = 9.793, kWfYplus = 11.225;
__device__ __forceinline__ double wall_utau(double ut, double y, double nu, bool &log_layer) {
  log_layer = false;
  if (!(ut > 0.0) || !(y > 0.0)) return 0.0;
  double u = sqrt(nu * ut / y);
  if (u * y / nu <= kWfYplus) return u;
  for (int it = 0; it < 8; ++it) {
    const double L = log(kWfE * y * u / nu);
    const double f = u * L / kWfKappa - ut;
    const double fp = (L + 1.0) / kWfKappa;
    u = u - f / fp;
  }
  log_layer = true;
  return u;
}

// buffer-frame coordinate 0 of a point, in sweep precision, plain order
template <typename R, int D>
__device__ __forceinline__ R local0(const R o[3], const R n[3], R x, R y, R z) {
  R s = Ex<R>::mul(Ex<R>::sub(x, o[0]), n[0]);
  s = Ex<R>::add(s, Ex<R>::mul(Ex<R>::sub(y, o[1]), n[1]));
  if (D == 3) s = Ex<R>::add(s, Ex<R>::mul(Ex<R>::sub(z, o[2]), n[2]));
  return s;
}

// The cells of visit_cells (span 1, no periodic axes) without those that
// cannot hold a point within the cut-off of a particle at offset o (o in
// [0, cs)^d from its cell's low corner): a row (dy, dz) is left out when
// its distance from the particle in y and z alone reaches the cut-off, and
// the row's first or last cell when the distance to that cell's box does.
// Only the ends of a row's index range move, so the candidates that remain
// come in the same order.  The test keeps a margin of 1e-3 cs for the FP32
// offsets: a cell it drops has no point closer than 1.001 cut-offs.
template <int D, typename F>
__device__ __forceinline__ void visit_cells_trimmed(const InstDev &I, int cx, int cy, int cz, const float o[3],
                                                    float cs, const uint32_t *__restrict__ off, F &&f) {
  const int nx = I.nc[0], ny = I.nc[1];
  const int nz = (D == 3) ? I.nc[2] : 1;
  const float far2 = (1.001f * cs) * (1.001f * cs);  // cut-off = cs = 2h
  const float lx = o[0], rx = cs - o[0];              // distances to the x faces
  const int a0 = max(cx - 1, 0), a1 = min(cx + 1, nx - 1);
  for (int dz = (D == 3 ? -1 : 0); dz <= (D == 3 ? 1 : 0); ++dz) {
    const int zz = cz + dz;
    if (zz < 0 || zz >= nz) continue;
    const float pz = dz == 0 ? 0.0f : (dz < 0 ? o[2] : cs - o[2]);
    for (int dy = -1; dy <= 1; ++dy) {
      const int yy = cy + dy;
      if (yy < 0 || yy >= ny) continue;
      const float py = dy == 0 ? 0.0f : (dy < 0 ? o[1] : cs - o[1]);
      const float b2 = py * py + pz * pz;
      if (b2 > far2) continue;
      const int c0 = (a0 < cx && lx * lx + b2 > far2) ? cx : a0;
      const int c1 = (a1 > cx && rx * rx + b2 > far2) ? cx : a1;
      const uint32_t row = I.cell_base + ((uint32_t)zz * (uint32_t)ny + (uint32_t)yy) * (uint32_t)nx;
      f(off[row + c0], off[row + c1 + 1]);
    }
  }
}

// visit the index ranges of the cells within +-span of (cx, cy, cz): the
// clamped part of each x row is one contiguous range; periodic axes hold at
// least 2 span + 1 cells (checked at creation), so wrapped coordinates are
// distinct and the wrapped x cells of a row form at most two more ranges.
// f has one call site so that it stays inlined.
template <int D, bool PER, typename F>
__device__ __forceinline__ void visit_cells(const InstDev &I, int cx, int cy, int cz, int span,
                                            const uint32_t *__restrict__ off, F &&f) {
  const int nx = I.nc[0], ny = I.nc[1];
  const int nz = (D == 3) ? I.nc[2] : 1;
  const int zspan = (D == 3) ? span : 0;
  const int a0 = max(cx - span, 0), a1 = min(cx + span, nx - 1);
  const int nparts = (PER && I.periodic[0]) ? 3 : 1;
  for (int dz = -zspan; dz <= zspan; ++dz) {
    int zz = cz + dz;
    if (zz < 0 || zz >= nz) {
      if (!PER || D != 3 || !I.periodic[2]) continue;
      zz = zz < 0 ? zz + nz : zz - nz;
    }
    for (int dy = -span; dy <= span; ++dy) {
      int yy = cy + dy;
      if (yy < 0 || yy >= ny) {
        if (!PER || !I.periodic[1]) continue;
        yy = yy < 0 ? yy + ny : yy - ny;
      }
      const uint32_t row = I.cell_base + ((uint32_t)zz * (uint32_t)ny + (uint32_t)yy) * (uint32_t)nx;
      for (int part = 0; part < nparts; ++part) {
        int c0 = a0, c1 = a1;
        if (part == 1) {  // cells wrapped from the left edge
          if (cx - span >= 0) continue;
          c0 = cx - span + nx;
          c1 = nx - 1;
        } else if (part == 2) {  // cells wrapped from the right edge
          if (cx + span < nx) continue;
          c0 = 0;
          c1 = cx + span - nx;
        }
        f(off[row + c0], off[row + c1 + 1]);
      }
    }
  }
}

// |r|^2 of i with two candidates at once on paired FP32 operations: the
// same roundings as pair_vec's FP32 path (difference, square, contracted
// sum), two lanes per instruction
template <int D>
__device__ __forceinline__ void rr_pairs_f32x2(const V4<float> &pi, const V4<float> &a, const V4<float> &b,
                                               float &ra, float &rb) {
  unsigned long long xi, xj, dx, yi, yj, dy, r;
  asm("mov.b64 %0, {%1, %1};" : "=l"(xi) : "f"(pi.x));
  asm("mov.b64 %0, {%1, %2};" : "=l"(xj) : "f"(a.x), "f"(b.x));
  asm("mov.b64 %0, {%1, %1};" : "=l"(yi) : "f"(pi.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(yj) : "f"(a.y), "f"(b.y));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dx) : "l"(xi), "l"(xj));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dy) : "l"(yi), "l"(yj));
  asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(r) : "l"(dx));
  asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(r) : "l"(dy), "l"(r));
  if (D == 3) {
    unsigned long long zi, zj, dz;
    asm("mov.b64 %0, {%1, %1};" : "=l"(zi) : "f"(pi.z));
    asm("mov.b64 %0, {%1, %2};" : "=l"(zj) : "f"(a.z), "f"(b.z));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dz) : "l"(zi), "l"(zj));
    asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(r) : "l"(dz), "l"(r));
  }
  asm("mov.b64 {%0, %1}, %2;" : "=f"(ra), "=f"(rb) : "l"(r));
}

// candidates j in [jb, je) whose position leads the 4-vector P[j * stride],
// four loads in flight; hit(j) is called, in increasing j, for every j with
// 0 < |r_ij|^2 < (2h)^2.  In FP64 (lo = hi = (2h)^2) that test is the
// definition itself.  In FP32 a candidate is a pair outright when its FP32
// |r|^2 lies in (0, lo), is not one at or beyond hi, and in between (or at
// zero) exact(j) decides with the FP64 test of the definition on the FP64
// positions; [lo, hi) brackets the cut-off by more than the rounding of the
// FP32 positions and sum can move |r|^2, so the FP32 list holds exactly the
// pairs of the FP64 test.  The decisions of up to 32 candidates are gathered
// in one mask before hit() runs on its set bits: the lanes of a warp then
// diverge once per 32 candidates, not once per four.
template <typename R, int D, bool PER, typename H, typename X>
__device__ __forceinline__ void scan_range(const Geo<R> &g, const V4<R> &Pi, const V4<R> *__restrict__ P,
                                           int stride, uint32_t jb, uint32_t je, R lo, R hi, H &&hit,
                                           X &&exact) {
  for (uint32_t j0 = jb; j0 < je; j0 += 32u) {
    const uint32_t j1 = min(je, j0 + 32u);
    uint32_t acc = 0u;
    for (uint32_t j = j0; j < j1; j += 4) {
      const unsigned tail = (j1 - j >= 4u) ? 0xFu : ((1u << (j1 - j)) - 1u);
      R rr[4];
      if constexpr (sizeof(R) == 4 && !PER) {
        // FP32 candidate arrays are padded by four entries: the loads need
        // no bounds, the tail mask drops the entries past the range
        const V4<R> q0 = P[j], q1 = P[j + 1], q2 = P[j + 2], q3 = P[j + 3];
        rr_pairs_f32x2<D>(Pi, q0, q1, rr[0], rr[1]);
        rr_pairs_f32x2<D>(Pi, q2, q3, rr[2], rr[3]);
      } else {
        const V4<R> q0 = P[(size_t)j * stride];
        const V4<R> q1 = (j + 1 < j1) ? P[(size_t)(j + 1) * stride] : q0;
        const V4<R> q2 = (j + 2 < j1) ? P[(size_t)(j + 2) * stride] : q0;
        const V4<R> q3 = (j + 3 < j1) ? P[(size_t)(j + 3) * stride] : q0;
        R d[3];
        rr[0] = pair_vec_abs<R, D, PER>(g, Pi, q0, d);
        rr[1] = pair_vec_abs<R, D, PER>(g, Pi, q1, d);
        rr[2] = pair_vec_abs<R, D, PER>(g, Pi, q2, d);
        rr[3] = pair_vec_abs<R, D, PER>(g, Pi, q3, d);
      }
      unsigned sure = ((rr[0] > (R)0 && rr[0] < lo) ? 1u : 0u) | ((rr[1] > (R)0 && rr[1] < lo) ? 2u : 0u) |
                      ((rr[2] > (R)0 && rr[2] < lo) ? 4u : 0u) | ((rr[3] > (R)0 && rr[3] < lo) ? 8u : 0u);
      sure &= tail;
      if (sizeof(R) == 4) {
        // candidates the FP32 test cannot decide (rare): the FP64 test, out
        // of the common path
        const unsigned maybe = ((rr[0] < hi) ? 1u : 0u) | ((rr[1] < hi) ? 2u : 0u) |
                               ((rr[2] < hi) ? 4u : 0u) | ((rr[3] < hi) ? 8u : 0u);
        unsigned amb = maybe & tail & ~sure;
        if (__builtin_expect(amb != 0u, 0)) {
          while (amb) {
            const int k = __ffs(amb) - 1;
            amb &= amb - 1;
            if (exact(j + (uint32_t)k)) sure |= 1u << k;
          }
        }
      }
      acc |= sure << (j - j0);
    }
    while (acc) {
      const int k = __ffs(acc) - 1;
      acc &= acc - 1;
      hit(j0 + (uint32_t)k);
    }
  }
}

// The FP64 test of the definition, 0 < |x_i - x_j|^2 < (2h)^2 summed left to
// right without contraction (minimum image on periodic axes), on the FP64
// positions of i (xi) and j (xj[c][j]): the decision for the rare FP32
// candidates within the band of the cut-off.  Not inlined, so that the
// FP64 work stays off the candidate loop.
static __device__ __noinline__ bool exact_pair_test(const InstDev &I, int dim, const double xi[3],
                                             const double *const xj[3], uint32_t j) {
  double rr = 0.0;
  for (int c = 0; c < dim; ++c) {
    double v = dsub(xi[c], xj[c][j]);
    if (I.periodic[c]) {
      const double hl = 0.5 * I.L[c];
      if (v > hl)
        v = dsub(v, I.L[c]);
      else if (v < -hl)
        v = dadd(v, I.L[c]);
    }
    rr = (c == 0) ? dmul(v, v) : dadd(rr, dmul(v, v));
  }
  return rr > 0.0 && rr < I.cut2;
}

// Half-width of the FP32 band around the cut-off within which the FP32
// |r|^2 cannot decide the pair (see scan_range).  With u = 2^-24, each FP32
// coordinate is within u |x| of the FP64 one and the FP32 difference adds
// u |x_i - x_j| (and u L when it is wrapped across a periodic length L, the
// shift itself being exact); near the cut-off |x_j| <= |x_i| + 2h, so each
// component of r is within u (2 M + 2 cs + L) of the FP64 one (M the
// largest |coordinate| of i, cs = 2h the cut-off), which moves |r|^2 by at
// most 2 sqrt(D) cs u (2 M + 2 cs + L) plus the rounding of the contracted
// sum (3 u cs^2) and of the FP32 cut-off itself (u cs^2).  The band is four
// times that bound: cs 2^-20 (D (M + cs + L) + cs).
__device__ __forceinline__ float cutoff_band(int D, float cs, float M, float L) {
  return cs * 9.5367431640625e-07f * ((float)D * (M + cs + L) + cs);
}

__device__ __forceinline__ void decode_cell(const InstDev &I, uint32_t key, int &cx, int &cy, int &cz) {
  uint32_t l = key - I.cell_base;
  cx = (int)(l % (uint32_t)I.nc[0]);
  uint32_t r = l / (uint32_t)I.nc[0];
  cy = (int)(r % (uint32_t)I.nc[1]);
  cz = (int)(r / (uint32_t)I.nc[1]);
}

// symmetric 3x3 stored as (xx, yy, zz, xy, xz, yz)
template <typename R, int D>
__device__ __forceinline__ void sym_add_outer(R A[6], const R d[3], R s) {
  // A += s d (x) d; with s = -F V this is -r_ij (x) grad W V
  A[0] += s * d[0] * d[0];
  A[1] += s * d[1] * d[1];
  A[3] += s * d[0] * d[1];
  if (D == 3) {
    A[2] += s * d[2] * d[2];
    A[4] += s * d[0] * d[2];
    A[5] += s * d[1] * d[2];
  }
}

// B = A^-1 in FP64 with the guard det A <= 1e-3 (tr A / d)^d -> I
template <int D>
__device__ __forceinline__ void invert_guarded(const double A[6], double B[6]) {
  for (int c = 0; c < 6; ++c) B[c] = 0.0;
  if (D == 2) {
    double t = 0.5 * (A[0] + A[1]);
    double det = A[0] * A[1] - A[3] * A[3];
    if (!(det > 1e-3 * t * t)) {
      B[0] = B[1] = 1.0;
      return;
    }
    double inv = 1.0 / det;
    B[0] = A[1] * inv;
    B[1] = A[0] * inv;
    B[3] = -A[3] * inv;
  } else {
    const double xx = A[0], yy = A[1], zz = A[2], xy = A[3], xz = A[4], yz = A[5];
    double c00 = yy * zz - yz * yz;
    double c01 = yz * xz - xy * zz;
    double c02 = xy * yz - yy * xz;
    double det = xx * c00 + xy * c01 + xz * c02;
    double t = (xx + yy + zz) * (1.0 / 3.0);
    if (!(det > 1e-3 * t * t * t)) {
      B[0] = B[1] = B[2] = 1.0;
      return;
    }
    double inv = 1.0 / det;
    B[0] = c00 * inv;
    B[1] = (xx * zz - xz * xz) * inv;
    B[2] = (xx * yy - xy * xy) * inv;
    B[3] = c01 * inv;
    B[4] = c02 * inv;
    B[5] = (xz * xy - xx * yz) * inv;
  }
}

// the same guarded inverse in the sweep precision (fast reciprocal in FP32)
template <typename R, int D>
__device__ __forceinline__ void invert_guarded_fast(const R A[6], R B[6]) {
  for (int c = 0; c < 6; ++c) B[c] = (R)0;
  if (D == 2) {
    const R t = (R)0.5 * (A[0] + A[1]);
    const R det = A[0] * A[1] - A[3] * A[3];
    if (!(det > (R)1e-3 * t * t)) {
      B[0] = B[1] = (R)1;
      return;
    }
    const R inv = Ex<R>::div((R)1, det);
    B[0] = A[1] * inv;
    B[1] = A[0] * inv;
    B[3] = -A[3] * inv;
  } else {
    const R xx = A[0], yy = A[1], zz = A[2], xy = A[3], xz = A[4], yz = A[5];
    const R c00 = yy * zz - yz * yz, c01 = yz * xz - xy * zz, c02 = xy * yz - yy * xz;
    const R det = xx * c00 + xy * c01 + xz * c02;
    const R t = (xx + yy + zz) * (R)(1.0 / 3.0);
    if (!(det > (R)1e-3 * t * t * t)) {
      B[0] = B[1] = B[2] = (R)1;
      return;
    }
    const R inv = Ex<R>::div((R)1, det);
    B[0] = c00 * inv;
    B[1] = (xx * zz - xz * xz) * inv;
    B[2] = (xx * yy - xy * xy) * inv;
    B[3] = c01 * inv;
    B[4] = c02 * inv;
    B[5] = (xz * xy - xx * yz) * inv;
  }
}

template <typename R, int D>
__device__ __forceinline__ void sym_matvec(const R B[6], const R x[3], R y[3]) {
  if (D == 2) {
    y[0] = B[0] * x[0] + B[3] * x[1];
    y[1] = B[3] * x[0] + B[1] * x[1];
    y[2] = (R)0;
  } else {
    y[0] = B[0] * x[0] + B[3] * x[1] + B[4] * x[2];
    y[1] = B[3] * x[0] + B[1] * x[1] + B[5] * x[2];
    y[2] = B[4] * x[0] + B[5] * x[1] + B[2] * x[2];
  }
}

// B, kw = 2/3 k and (3D) p from a momentum record; false for the marker of a
// pressure-buffer particle, whose B is then not in the record
template <typename R, int D>
__device__ __forceinline__ bool mom_B(const V4<R> &m1, const V4<R> &m2, R B[6], R &kw, R &p) {
  if (D == 2) {
    // (x y V p)(Bxx Bxy Byy kw)
    B[0] = m1.x;
    B[3] = m1.y;
    B[1] = m1.z;
    B[2] = B[4] = B[5] = (R)0;
    kw = m1.w;
    return m1.x >= (R)0;
  } else {
    // (x y z V)(p kw Bxx Byy)(Bzz Bxy Bxz Byz)
    p = m1.x;
    kw = m1.y;
    B[0] = m1.z;
    B[1] = m1.w;
    B[2] = m2.x;
    B[3] = m2.y;
    B[4] = m2.z;
    B[5] = m2.w;
    return m1.z >= (R)0;
  }
}

// effective pressure p + 2/3 rho k (Table 1) with rho = rho0 + p / c0^2,
// the stiff EOS of Sec. 2.1 solved for the density
template <typename R>
__device__ __forceinline__ R p_eff(R p, R kw, R rho0, R inv_c0sq) {
  return p + kw * (rho0 + p * inv_c0sq);
}

}  // namespace sphk
