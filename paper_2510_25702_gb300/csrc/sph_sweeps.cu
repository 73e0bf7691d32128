// sph_sweeps.cu -- the pair sweeps of one advection step.
//
//  k_adv  (once per advection step): correction matrix B_i with the mirror
//         condition at pressure buffers (a5; Sec. 2.2, 3.3), ARD viscous
//         acceleration (a6; Sec. 2.2), k-epsilon sources and diffusion with
//         the explicit update (a7; Sec. 2.1, 2.2, App. A), then the first
//         half of sub-step 0 (a8).
//  k_mom  (per acoustic sub-step): RKGC pressure acceleration with the
//         compensated open-boundary term (a9; Sec. 2.2, final Eq. of 3.3),
//         velocity kick and half position update.
//  k_cont (per acoustic sub-step): Riemann continuity (a10; Sec. 2.2),
//         density half update, buffer boundary values (a11) and the first
//         half of the next sub-step.
//
// One thread per particle in cell order; the neighbours of a particle are
// the particles of the 3^d cells around its cell, and because particles
// are sorted by cell key the cells of one row form one contiguous index
// range, so a 2D sweep walks three ranges (nine in 3D) of the packs.
// Neighbouring threads read overlapping ranges, which L1/L2 serve.
// R is the sweep precision (float or double); every accumulation that ends
// in a master field is converted to FP64 in the epilogue.
#include "sph_internal.cuh"

namespace sphk {

template <typename R>
struct Ex;
template <>
struct Ex<double> {
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
};
template <>
struct Ex<float> {
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
};

// per-thread copy of the instance geometry in sweep precision
template <typename R>
struct Geo {
  R L[3];
  int per[3];
  R cut2, inv_h, alpha_h, reg;
};

template <typename R, int D>
__device__ __forceinline__ Geo<R> make_geo(const InstDev &I) {
  Geo<R> g;
  for (int a = 0; a < 3; ++a) {
    g.L[a] = (R)I.L[a];
    g.per[a] = (a < D) ? I.periodic[a] : 0;
  }
  g.cut2 = (R)I.cut2;
  g.inv_h = (R)(1.0 / I.h);
  g.alpha_h = (R)I.alpha_h;
  g.reg = (R)I.reg;
  return g;
}

// r_ij = x_i - x_j with the minimum image; returns |r_ij|^2 summed left to
// right without contraction (the cut-off test decides membership)
template <typename R, int D>
__device__ __forceinline__ R pair_vec(const Geo<R> &g, const V4<R> &pi, const V4<R> &pj, R d[3]) {
  R xi[3] = {pi.x, pi.y, pi.z}, xj[3] = {pj.x, pj.y, pj.z};
  R rr = (R)0;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    R v = Ex<R>::sub(xi[a], xj[a]);
    if (g.per[a]) {
      R h = (R)0.5 * g.L[a];
      if (v > h)
        v = Ex<R>::sub(v, g.L[a]);
      else if (v < -h)
        v = Ex<R>::add(v, g.L[a]);
    }
    d[a] = v;
    rr = (a == 0) ? Ex<R>::mul(v, v) : Ex<R>::add(rr, Ex<R>::mul(v, v));
  }
  if (D == 2) d[2] = (R)0;
  return rr;
}

// Wendland C2 derivative dW/dr (Sec. 2.2 kernel, support 2h)
template <typename R>
__device__ __forceinline__ R kernel_dW(const Geo<R> &g, R r) {
  R q = r * g.inv_h;
  R w = (R)1 - (R)0.5 * q;
  return g.alpha_h * ((R)-5 * q) * w * w * w;
}

// buffer-frame coordinate 0 of a point, in sweep precision, plain order
template <typename R, int D>
__device__ __forceinline__ R local0(const R o[3], const R n[3], R x, R y, R z) {
  R s = Ex<R>::mul(Ex<R>::sub(x, o[0]), n[0]);
  s = Ex<R>::add(s, Ex<R>::mul(Ex<R>::sub(y, o[1]), n[1]));
  if (D == 3) s = Ex<R>::add(s, Ex<R>::mul(Ex<R>::sub(z, o[2]), n[2]));
  return s;
}

// distinct cell coordinates c-span..c+span along one axis (wrapped when
// periodic, dropped when outside a non-periodic grid)
__device__ __forceinline__ int axis_list(int c, int span, int n, int per, int out[5]) {
  int cnt = 0;
  for (int cc = c - span; cc <= c + span; ++cc) {
    int w = cc;
    if (cc < 0 || cc >= n) {
      if (!per) continue;
      w = ((cc % n) + n) % n;
    }
    bool dup = false;
    for (int t = 0; t < cnt; ++t) dup |= (out[t] == w);
    if (!dup) out[cnt++] = w;
  }
  return cnt;
}

// visit the index ranges of the cells within +-span of (cx, cy, cz); the
// clamped part of each x row is one contiguous range, wrapped x cells are
// extra single-cell ranges
template <int D, typename F>
__device__ __forceinline__ void visit_cells(const InstDev &I, int cx, int cy, int cz, int span,
                                            const uint32_t *__restrict__ off, F &&f) {
  const int nx = I.nc[0], ny = I.nc[1];
  int ys[5], zs[5];
  const int nys = axis_list(cy, span, ny, I.periodic[1], ys);
  int nzs = 1;
  zs[0] = 0;
  if (D == 3) nzs = axis_list(cz, span, I.nc[2], I.periodic[2], zs);
  const int a0 = max(cx - span, 0), a1 = min(cx + span, nx - 1);
  int xw[4], nxw = 0;
  if (I.periodic[0]) {
    for (int xx = cx - span; xx <= cx + span; ++xx) {
      if (xx >= 0 && xx < nx) continue;
      int w = ((xx % nx) + nx) % nx;
      if (w >= a0 && w <= a1) continue;
      bool dup = false;
      for (int t = 0; t < nxw; ++t) dup |= (xw[t] == w);
      if (!dup && nxw < 4) xw[nxw++] = w;
    }
  }
  for (int zi = 0; zi < nzs; ++zi)
    for (int yi = 0; yi < nys; ++yi) {
      const uint32_t row = I.cell_base + ((uint32_t)zs[zi] * (uint32_t)ny + (uint32_t)ys[yi]) * (uint32_t)nx;
      f(off[row + a0], off[row + a1 + 1]);
      for (int t = 0; t < nxw; ++t) f(off[row + xw[t]], off[row + xw[t] + 1]);
    }
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
__device__ __forceinline__ void sym_add_outer(R A[6], const R d[3], const R gw[3], R V) {
  // A += -d (x) gw V; the product is symmetric in exact arithmetic, the
  // upper triangle is accumulated
  A[0] += -d[0] * gw[0] * V;
  A[1] += -d[1] * gw[1] * V;
  A[3] += -d[0] * gw[1] * V;
  if (D == 3) {
    A[2] += -d[2] * gw[2] * V;
    A[4] += -d[0] * gw[2] * V;
    A[5] += -d[1] * gw[2] * V;
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
    B[0] = A[1] / det;
    B[1] = A[0] / det;
    B[3] = -A[3] / det;
  } else {
    const double xx = A[0], yy = A[1], zz = A[2], xy = A[3], xz = A[4], yz = A[5];
    double c00 = yy * zz - yz * yz;
    double c01 = yz * xz - xy * zz;
    double c02 = xy * yz - yy * xz;
    double det = xx * c00 + xy * c01 + xz * c02;
    double t = (xx + yy + zz) / 3.0;
    if (!(det > 1e-3 * t * t * t)) {
      B[0] = B[1] = B[2] = 1.0;
      return;
    }
    B[0] = c00 / det;
    B[1] = (xx * zz - xz * xz) / det;
    B[2] = (xx * yy - xy * xy) / det;
    B[3] = c01 / det;
    B[4] = c02 / det;
    B[5] = (xz * xy - xx * yz) / det;
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

// =========================================================================
// advection sweep: B (+ mirror), viscous acceleration, k-epsilon, half 1
// =========================================================================
template <typename R, int D>
__global__ void __launch_bounds__(kBlock) k_adv(SweepArgs a, Packs<R> pk) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.cnt->n_live) return;
  const Masters m = a.m;
  const int ii = m.inst[i];
  const InstDev &I = a.inst[ii];
  const Geo<R> g = make_geo<R, D>(I);
  int cx, cy, cz;
  decode_cell(I, a.keys[i], cx, cy, cz);
  const V4<R> Pi = pk.P[0][i];
  const V4<R> Qi = pk.Q[0][i];
  const bool rans = I.rans != 0;
  const R rho0 = (R)I.rho0, nu_l = (R)I.nu_l, c0 = (R)I.c0, eta = (R)I.eta, muRk = (R)I.muR_k;
  const R nut_i = rans ? (R)m.nut[i] : (R)0;
  const R k_i = rans ? (R)m.k[i] : (R)0, e_i = rans ? (R)m.eps[i] : (R)0;
  const R mu_i = rho0 * (nu_l + nut_i);
  const R Dk_i = nu_l + nut_i / (R)kSigK, De_i = nu_l + nut_i / (R)kSigE;

  const int lab = m.label[i];
  const BufDev *mb = (lab > 0 && lab <= I.nbuf) ? &a.buf[I.buf0 + lab - 1] : nullptr;
  const bool mirror = mb && mb->type == SPH_BUF_PRESSURE;
  R mo[3] = {0, 0, 0}, mn[3] = {0, 0, 0};
  if (mirror)
    for (int c = 0; c < 3; ++c) {
      mo[c] = (R)mb->origin[c];
      mn[c] = (R)mb->frame[c];
    }

  R A[6] = {0, 0, 0, 0, 0, 0};
  R sv[3] = {0, 0, 0};
  R G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  R dk = 0, de = 0;

  auto real_range = [&](uint32_t jb, uint32_t je) {
    for (uint32_t j = jb; j < je; ++j) {
      if ((int)j == i) continue;
      const V4<R> Pj = pk.P[0][j];
      R d[3];
      const R rr = pair_vec<R, D>(g, Pi, Pj, d);
      if (!(rr > (R)0 && rr < g.cut2)) continue;
      const R r = sqrt(rr);
      const R dw = kernel_dW(g, r);
      const R inv_r = (R)1 / r;
      R gw[3] = {dw * d[0] * inv_r, dw * d[1] * inv_r, dw * d[2] * inv_r};
      const R V = Pj.w;
      if (!mirror || !(local0<R, D>(mo, mn, Pj.x, Pj.y, Pj.z) < (R)0)) sym_add_outer<R, D>(A, d, gw, V);
      const V4<R> Qj = pk.Q[0][j];
      R vij[3] = {Qi.x - Qj.x, Qi.y - Qj.y, Qi.z - Qj.z};
      R nut_j = (R)0, k_j = (R)0, e_j = (R)0;
      if (rans) {
        const V4<R> Tj = pk.T[j];
        k_j = Tj.x;
        e_j = Tj.y;
        nut_j = Tj.z;
      }
      const R mu_j = rho0 * (nu_l + nut_j);
      const R mut = (R)2 * mu_i * mu_j / (mu_i + mu_j);
      R mu_ad = mut;
      if (rans) {
        R ve = -(vij[0] * d[0] + vij[1] * d[1] + vij[2] * d[2]) * inv_r;
        R lim = eta * (ve > (R)0 ? ve : (R)0);
        R muR = muRk * (lim < c0 ? lim : c0);
        mu_ad = mut > muR ? mut : muR;
      }
      const R f = dw / (r + g.reg) * V;
#pragma unroll
      for (int c = 0; c < D; ++c) sv[c] += mu_ad * f * vij[c];
      if (rans) {
#pragma unroll
        for (int p = 0; p < D; ++p)
#pragma unroll
          for (int q = 0; q < D; ++q) G[p][q] += vij[p] * gw[q] * V;
        const R Dk_j = nu_l + nut_j / (R)kSigK, De_j = nu_l + nut_j / (R)kSigE;
        dk += rho0 * ((R)2 * Dk_i * Dk_j / (Dk_i + Dk_j)) * (k_i - k_j) * f;
        de += rho0 * ((R)2 * De_i * De_j / (De_i + De_j)) * (e_i - e_j) * f;
      }
    }
  };
  visit_cells<D>(I, cx, cy, cz, 1, a.off, real_range);

  auto wall_range = [&](uint32_t jb, uint32_t je) {
    for (uint32_t w = jb; w < je; ++w) {
      const V4<R> Wp = pk.WP[w];
      R d[3];
      const R rr = pair_vec<R, D>(g, Pi, Wp, d);
      if (!(rr > (R)0 && rr < g.cut2)) continue;
      const R r = sqrt(rr);
      const R dw = kernel_dW(g, r);
      const R inv_r = (R)1 / r;
      R gw[3] = {dw * d[0] * inv_r, dw * d[1] * inv_r, dw * d[2] * inv_r};
      const R V = Wp.w;
      if (!mirror || !(local0<R, D>(mo, mn, Wp.x, Wp.y, Wp.z) < (R)0)) sym_add_outer<R, D>(A, d, gw, V);
      const V4<R> Wv = pk.WV[w];
      // no-slip: the dummy carries 2 v_wall - v_i
      R vij[3] = {(R)2 * (Qi.x - Wv.x), (R)2 * (Qi.y - Wv.y), (R)2 * (Qi.z - Wv.z)};
      R mu_ad = mu_i;
      if (rans) {
        R ve = -(vij[0] * d[0] + vij[1] * d[1] + vij[2] * d[2]) * inv_r;
        R lim = eta * (ve > (R)0 ? ve : (R)0);
        R muR = muRk * (lim < c0 ? lim : c0);
        mu_ad = mu_i > muR ? mu_i : muR;
      }
      const R f = dw / (r + g.reg) * V;
#pragma unroll
      for (int c = 0; c < D; ++c) sv[c] += mu_ad * f * vij[c];
      if (rans) {
#pragma unroll
        for (int p = 0; p < D; ++p)
#pragma unroll
          for (int q = 0; q < D; ++q) G[p][q] += vij[p] * gw[q] * V;
      }
    }
  };
  visit_cells<D>(I, cx, cy, cz, 1, a.woff, wall_range);

  if (mirror) {
    // images m_j = x_j - 2 x'_0(x_j) n_b of every particle on the fluid side
    // of the open face; searched around the image of x_i (two-cell margin)
    const R si = local0<R, D>(mo, mn, Pi.x, Pi.y, Pi.z);
    const double q0 = (double)Pi.x - 2.0 * (double)si * mb->frame[0];
    const double q1 = (double)Pi.y - 2.0 * (double)si * mb->frame[1];
    const double q2 = (double)Pi.z - 2.0 * (double)si * mb->frame[2];
    const int qx = cell_coord(I, q0, 0), qy = cell_coord(I, q1, 1), qz = D == 3 ? cell_coord(I, q2, 2) : 0;
    auto mirror_one = [&](const V4<R> &Pj) {
      const R sj = local0<R, D>(mo, mn, Pj.x, Pj.y, Pj.z);
      if (sj < (R)0) return;
      const R two_s = Ex<R>::mul((R)2, sj);
      R xj[3] = {Pj.x, Pj.y, Pj.z}, xi[3] = {Pi.x, Pi.y, Pi.z};
      R d[3] = {0, 0, 0};
      R dd = 0;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        R img = Ex<R>::sub(xj[c], Ex<R>::mul(two_s, mn[c]));
        d[c] = Ex<R>::sub(xi[c], img);
        dd = (c == 0) ? Ex<R>::mul(d[c], d[c]) : Ex<R>::add(dd, Ex<R>::mul(d[c], d[c]));
      }
      if (!(dd > (R)0 && dd < g.cut2)) return;
      const R r = sqrt(dd);
      const R dw = kernel_dW(g, r);
      const R inv_r = (R)1 / r;
      R gw[3] = {dw * d[0] * inv_r, dw * d[1] * inv_r, dw * d[2] * inv_r};
      sym_add_outer<R, D>(A, d, gw, Pj.w);
    };
    visit_cells<D>(I, qx, qy, qz, 2, a.off, [&](uint32_t jb, uint32_t je) {
      for (uint32_t j = jb; j < je; ++j) mirror_one(pk.P[0][j]);
    });
    visit_cells<D>(I, qx, qy, qz, 2, a.woff, [&](uint32_t jb, uint32_t je) {
      for (uint32_t w = jb; w < je; ++w) mirror_one(pk.WP[w]);
    });
  }

  // ---------------- epilogue (FP64) ----------------
  double Ad[6], B[6];
  for (int c = 0; c < 6; ++c) Ad[c] = (double)A[c];
  invert_guarded<D>(Ad, B);
  for (int c = 0; c < 6; ++c) a.der.B[c][i] = B[c];
  const double rho_i = m.rho[i], mass_i = m.mass[i];
  for (int c = 0; c < 3; ++c) a.der.an[c][i] = (c < D) ? 2.0 * (double)sv[c] / rho_i : 0.0;

  double kap = 0.0;
  if (rans) {
    // grad v = -(sum v_ij (x) grad W V) B^T, (p, q) = dv_p / dx_q
    double Bf[3][3] = {{B[0], B[3], B[4]}, {B[3], B[1], B[5]}, {B[4], B[5], B[2]}};
    double gv[3][3];
    for (int p = 0; p < D; ++p)
      for (int q = 0; q < D; ++q) {
        double s = 0.0;
        for (int c = 0; c < D; ++c) s += (double)G[p][c] * Bf[q][c];
        gv[p][q] = -s;
      }
    double tr = 0.0, prod = 0.0;
    for (int p = 0; p < D; ++p) {
      tr += gv[p][p];
      for (int q = 0; q < D; ++q) prod += (gv[p][q] + gv[q][p]) * gv[p][q];
    }
    const double kd = m.k[i], ed = m.eps[i], nutd = m.nut[i];
    const double Gk = nutd * prod - (2.0 / 3.0) * kd * tr;
    const double dkdt = Gk - ed + 2.0 * (double)dk / rho_i;
    const double dedt = kC1 * (ed / kd) * Gk - kC2 * ed * ed / kd + 2.0 * (double)de / rho_i;
    double k1 = kd + I.dt_ad * dkdt, e1 = ed + I.dt_ad * dedt;
    k1 = k1 > kFloor ? k1 : kFloor;
    e1 = e1 > kFloor ? e1 : kFloor;
    m.k[i] = k1;
    m.eps[i] = e1;
    m.nut[i] = kCmu * k1 * k1 / e1;
    kap = (2.0 / 3.0) * k1 * mass_i;
  }
  // neighbour-facing B pack; pressure-buffer particles are marked so that
  // neighbours use their own B_i (the condition B_k = B_i, Sec. 3.3)
  if (D == 2) {
    V4<R> b0 = {(R)B[0], (R)B[3], (R)B[1], (R)kap};
    if (mirror) b0.x = (R)-1;
    pk.Bm0[i] = b0;
  } else {
    V4<R> b0 = {(R)B[0], (R)B[1], (R)B[2], (R)kap};
    V4<R> b1 = {(R)B[3], (R)B[4], (R)B[5], (R)0};
    if (mirror) b0.x = (R)-1;
    pk.Bm0[i] = b0;
    pk.Bm1[i] = b1;
  }
  // first half of sub-step 0 (a8)
  const double dt = I.dt;
  double rho = rho_i + 0.5 * dt * m.drho[i];
  double p = I.eos_k * (rho / I.rho0 - 1.0);
  m.rho[i] = rho;
  m.p[i] = p;
  for (int c = 0; c < D; ++c) m.x[c][i] = m.x[c][i] + 0.5 * dt * m.v[c][i];
  V4<R> P1 = {Pi.x, Pi.y, Pi.z, (R)(mass_i / rho)};
  V4<R> Q1 = {Qi.x, Qi.y, Qi.z, (R)p};
  pk.P[1][i] = P1;
  pk.Q[1][i] = Q1;
}

// =========================================================================
// momentum sweep (a9)
// =========================================================================
template <typename R, int D>
__global__ void __launch_bounds__(kBlock) k_mom(SweepArgs a, Packs<R> pk, int pin, int qin, int qout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.cnt->n_live) return;
  const Masters m = a.m;
  const int ii = m.inst[i];
  const InstDev &I = a.inst[ii];
  if (a.sub >= I.n_ac) return;
  const Geo<R> g = make_geo<R, D>(I);
  int cx, cy, cz;
  decode_cell(I, a.keys[i], cx, cy, cz);
  const V4<R> *__restrict__ P = pk.P[pin];
  const V4<R> *__restrict__ Q = pk.Q[qin];
  const V4<R> Pi = P[i];
  const R p_i = Q[i].w;
  const bool rans = I.rans != 0;
  const double rho_i = m.rho[i];
  double Bd[6];
  for (int c = 0; c < 6; ++c) Bd[c] = a.der.B[c][i];
  R Bi[6];
  for (int c = 0; c < 6; ++c) Bi[c] = (R)Bd[c];
  const R pe_i = rans ? p_i + (R)((2.0 / 3.0) * m.k[i] * m.mass[i]) / Pi.w : p_i;

  R S1[3] = {0, 0, 0}, Cb[3] = {0, 0, 0}, S2[3] = {0, 0, 0}, Ct[3] = {0, 0, 0};
  visit_cells<D>(I, cx, cy, cz, 1, a.off, [&](uint32_t jb, uint32_t je) {
    for (uint32_t j = jb; j < je; ++j) {
      if ((int)j == i) continue;
      const V4<R> Pj = P[j];
      R d[3];
      const R rr = pair_vec<R, D>(g, Pi, Pj, d);
      if (!(rr > (R)0 && rr < g.cut2)) continue;
      const R r = sqrt(rr);
      const R dw = kernel_dW(g, r) / r;
      const R V = Pj.w;
      R gw[3] = {dw * d[0], dw * d[1], dw * d[2]};
      const R p_j = Q[j].w;
      const V4<R> b0 = pk.Bm0[j];
      const R pe_j = rans ? p_j + b0.w / V : p_j;
      if (b0.x < (R)0) {
#pragma unroll
        for (int c = 0; c < D; ++c) Cb[c] += V * gw[c];
      } else {
        R Bj[6];
        if (D == 2) {
          Bj[0] = b0.x; Bj[3] = b0.y; Bj[1] = b0.z;
          Bj[2] = Bj[4] = Bj[5] = (R)0;
        } else {
          const V4<R> b1 = pk.Bm1[j];
          Bj[0] = b0.x; Bj[1] = b0.y; Bj[2] = b0.z;
          Bj[3] = b1.x; Bj[4] = b1.y; Bj[5] = b1.z;
        }
        R bg[3];
        sym_matvec<R, D>(Bj, gw, bg);
#pragma unroll
        for (int c = 0; c < D; ++c) S1[c] += V * bg[c];
      }
#pragma unroll
      for (int c = 0; c < D; ++c) {
        S2[c] += V * pe_j * gw[c];
        Ct[c] += V * gw[c];
      }
    }
  });
  visit_cells<D>(I, cx, cy, cz, 1, a.woff, [&](uint32_t jb, uint32_t je) {
    for (uint32_t w = jb; w < je; ++w) {
      const V4<R> Wp = pk.WP[w];
      R d[3];
      const R rr = pair_vec<R, D>(g, Pi, Wp, d);
      if (!(rr > (R)0 && rr < g.cut2)) continue;
      const R r = sqrt(rr);
      const R dw = kernel_dW(g, r) / r;
      const R V = Wp.w;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const R gv = V * dw * d[c];
        Cb[c] += gv;       // wall dummy: B^_j = B_i
        S2[c] += pe_i * gv; // wall dummy: p_j = p_i
        Ct[c] += gv;
      }
    }
  });
  double acc[3] = {0, 0, 0};
  {
    double s1[3], cb[3], s2[3], ct[3], bcb[3], bs2[3], bct[3];
    for (int c = 0; c < 3; ++c) {
      s1[c] = (double)S1[c];
      cb[c] = (double)Cb[c];
      s2[c] = (double)S2[c];
      ct[c] = (double)Ct[c];
    }
    sym_matvec<double, D>(Bd, cb, bcb);
    sym_matvec<double, D>(Bd, s2, bs2);
    sym_matvec<double, D>(Bd, ct, bct);
    const double pe = (double)pe_i;
    for (int c = 0; c < D; ++c) acc[c] = -(pe * (s1[c] + bcb[c]) + bs2[c]) / rho_i;
    const int lab = m.label[i];
    if (lab > 0 && lab <= I.nbuf) {
      const BufDev &b = a.buf[I.buf0 + lab - 1];
      if (b.type == SPH_BUF_PRESSURE) {
        double pob = b.p_ob;
        if (rans) pob += (2.0 / 3.0) * rho_i * m.k[i];
        for (int c = 0; c < D; ++c) acc[c] += 2.0 * pob / rho_i * bct[c];
      }
    }
  }
  const double dt = I.dt;
  double v[3];
  for (int c = 0; c < 3; ++c) v[c] = m.v[c][i];
  for (int c = 0; c < D; ++c) {
    v[c] = v[c] + dt * (acc[c] + a.der.an[c][i] + I.g[c]);
    m.v[c][i] = v[c];
    m.x[c][i] = m.x[c][i] + 0.5 * dt * v[c];
  }
  V4<R> Qo = {(R)v[0], (R)v[1], (R)v[2], p_i};
  pk.Q[qout][i] = Qo;
}

// =========================================================================
// continuity sweep (a10) + density update + boundary values (a11) + next
// half step (a8)
// =========================================================================
template <typename R, int D>
__global__ void __launch_bounds__(kBlock) k_cont(SweepArgs a, Packs<R> pk, int pin, int qin, int pout,
                                                 int qout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.cnt->n_live) return;
  const Masters m = a.m;
  const int ii = m.inst[i];
  const InstDev &I = a.inst[ii];
  if (a.sub >= I.n_ac) return;
  const Geo<R> g = make_geo<R, D>(I);
  int cx, cy, cz;
  decode_cell(I, a.keys[i], cx, cy, cz);
  const V4<R> *__restrict__ P = pk.P[pin];
  const V4<R> *__restrict__ Q = pk.Q[qin];
  const V4<R> Pi = P[i];
  const V4<R> Qi = Q[i];
  const R inv_rc = (R)(1.0 / I.rc0);
  R sum = 0;
  visit_cells<D>(I, cx, cy, cz, 1, a.off, [&](uint32_t jb, uint32_t je) {
    for (uint32_t j = jb; j < je; ++j) {
      if ((int)j == i) continue;
      const V4<R> Pj = P[j];
      R d[3];
      const R rr = pair_vec<R, D>(g, Pi, Pj, d);
      if (!(rr > (R)0 && rr < g.cut2)) continue;
      const R r = sqrt(rr);
      const R dw = kernel_dW(g, r);
      const V4<R> Qj = Q[j];
      const R vd = (Qi.x - Qj.x) * d[0] + (Qi.y - Qj.y) * d[1] + (Qi.z - Qj.z) * d[2];
      sum += (vd / r + (Qi.w - Qj.w) * inv_rc) * dw * Pj.w;
    }
  });
  visit_cells<D>(I, cx, cy, cz, 1, a.woff, [&](uint32_t jb, uint32_t je) {
    for (uint32_t w = jb; w < je; ++w) {
      const V4<R> Wp = pk.WP[w];
      R d[3];
      const R rr = pair_vec<R, D>(g, Pi, Wp, d);
      if (!(rr > (R)0 && rr < g.cut2)) continue;
      const R r = sqrt(rr);
      const R dw = kernel_dW(g, r);
      const V4<R> Wv = pk.WV[w];
      // dummy velocity 2 v_wall - v_i, dummy pressure p_i
      const R vd = (R)2 * ((Qi.x - Wv.x) * d[0] + (Qi.y - Wv.y) * d[1] + (Qi.z - Wv.z) * d[2]);
      sum += vd / r * dw * Wp.w;
    }
  });
  const double dt = I.dt;
  const double drho = m.rho[i] * (double)sum;
  m.drho[i] = drho;
  double rho = m.rho[i] + 0.5 * dt * drho;
  m.rho[i] = rho;
  const int lab = m.label[i];
  if (lab > 0 && lab <= I.nbuf) {
    const BufDev &b = a.buf[I.buf0 + lab - 1];
    apply_bc(I, b, m, i, a.step, (uint32_t)a.sub);
    rho = m.rho[i];
    if (I.rans && b.turb == SPH_TURB_FREESTREAM) {
      V4<R> b0 = pk.Bm0[i];
      b0.w = (R)((2.0 / 3.0) * b.k_in * m.mass[i]);
      pk.Bm0[i] = b0;
    }
  }
  double v0 = m.v[0][i], v1 = m.v[1][i], v2 = m.v[2][i];
  if (!isfinite(rho) || !isfinite(v0) || !isfinite(v1) || !isfinite(v2)) set_status(a.status, SPH_ERR_NONFINITE);
  if (a.sub + 1 < I.n_ac) {
    // first half of the next sub-step
    rho = rho + 0.5 * dt * drho;
    const double p = I.eos_k * (rho / I.rho0 - 1.0);
    m.rho[i] = rho;
    m.p[i] = p;
    double v[3] = {v0, v1, v2};
    for (int c = 0; c < D; ++c) m.x[c][i] = m.x[c][i] + 0.5 * dt * v[c];
    V4<R> Po = {Pi.x, Pi.y, Pi.z, (R)(m.mass[i] / rho)};
    V4<R> Qo = {(R)v0, (R)v1, (R)v2, (R)p};
    pk.P[pout][i] = Po;
    pk.Q[qout][i] = Qo;
  }
}

// =========================================================================
// neighbour pairs of the current configuration (FP64 masters), test aid
// =========================================================================
__global__ void __launch_bounds__(kBlock) k_pairs(SweepArgs a, const double *__restrict__ wx,
                                                  const double *__restrict__ wy, const double *__restrict__ wz,
                                                  const uint32_t *__restrict__ wall_index, int64_t *out, int64_t max,
                                                  unsigned long long *counter) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.cnt->n_live) return;
  const Masters m = a.m;
  const int ii = m.inst[i];
  const InstDev &I = a.inst[ii];
  int cx, cy, cz;
  decode_cell(I, a.keys[i], cx, cy, cz);
  const double xi[3] = {m.x[0][i], m.x[1][i], m.x[2][i]};
  auto test = [&](const double xj[3]) -> bool {
    double rr = 0.0;
    for (int c = 0; c < I.dim; ++c) {
      double v = dsub(xi[c], xj[c]);
      if (I.periodic[c]) {
        double h = 0.5 * I.L[c];
        if (v > h)
          v = dsub(v, I.L[c]);
        else if (v < -h)
          v = dadd(v, I.L[c]);
      }
      rr = (c == 0) ? dmul(v, v) : dadd(rr, dmul(v, v));
    }
    return rr > 0.0 && rr < I.cut2;
  };
  auto emit = [&](int64_t uj, int64_t wall) {
    unsigned long long t = atomicAdd(counter, 1ull);
    if ((int64_t)t < max) {
      out[4 * t + 0] = m.uid[i];
      out[4 * t + 1] = uj;
      out[4 * t + 2] = wall;
      out[4 * t + 3] = ii;
    }
  };
  auto body = [&](uint32_t jb, uint32_t je) {
    for (uint32_t j = jb; j < je; ++j) {
      if ((int)j == i) continue;
      const double xj[3] = {m.x[0][j], m.x[1][j], m.x[2][j]};
      if (test(xj)) emit(m.uid[j], 0);
    }
  };
  auto wbody = [&](uint32_t jb, uint32_t je) {
    for (uint32_t w = jb; w < je; ++w) {
      const double xj[3] = {wx[w], wy[w], wz[w]};
      if (test(xj)) emit(wall_index[w], 1);
    }
  };
  if (I.dim == 2) {
    visit_cells<2>(I, cx, cy, cz, 1, a.off, body);
    visit_cells<2>(I, cx, cy, cz, 1, a.woff, wbody);
  } else {
    visit_cells<3>(I, cx, cy, cz, 1, a.off, body);
    visit_cells<3>(I, cx, cy, cz, 1, a.woff, wbody);
  }
}

// ------------------------------------------------------------------------
// launch wrappers
// ------------------------------------------------------------------------
static inline int grid_for(int max_n) {
  int g = (max_n + kBlock - 1) / kBlock;
  return g < 1 ? 1 : g;
}

template <typename R>
static void adv_dispatch(const SweepArgs &a, void *packs, int dim, int max_n, cudaStream_t st) {
  Packs<R> &pk = *(Packs<R> *)packs;
  if (dim == 2)
    k_adv<R, 2><<<grid_for(max_n), kBlock, 0, st>>>(a, pk);
  else
    k_adv<R, 3><<<grid_for(max_n), kBlock, 0, st>>>(a, pk);
}

void launch_advection_sweep(const SweepArgs &a, void *packs, int prec, int dim, int max_n, cudaStream_t st) {
  if (prec == SPH_PREC_FP32)
    adv_dispatch<float>(a, packs, dim, max_n, st);
  else
    adv_dispatch<double>(a, packs, dim, max_n, st);
}

// Pack ping-pong: the advection sweep leaves P[1], Q[1].  Sub-step s reads
// P[pc] with pc = 1 for even s, 0 for odd s; momentum reads Q[1] and writes
// Q[0]; continuity reads Q[0], writes P[1 - pc] and Q[1].
template <typename R>
static void mom_dispatch(const SweepArgs &a, void *packs, int dim, int max_n, int sub, cudaStream_t st) {
  Packs<R> &pk = *(Packs<R> *)packs;
  const int pc = (sub % 2 == 0) ? 1 : 0;
  if (dim == 2)
    k_mom<R, 2><<<grid_for(max_n), kBlock, 0, st>>>(a, pk, pc, 1, 0);
  else
    k_mom<R, 3><<<grid_for(max_n), kBlock, 0, st>>>(a, pk, pc, 1, 0);
}

template <typename R>
static void cont_dispatch(const SweepArgs &a, void *packs, int dim, int max_n, int sub, cudaStream_t st) {
  Packs<R> &pk = *(Packs<R> *)packs;
  const int pc = (sub % 2 == 0) ? 1 : 0;
  if (dim == 2)
    k_cont<R, 2><<<grid_for(max_n), kBlock, 0, st>>>(a, pk, pc, 0, 1 - pc, 1);
  else
    k_cont<R, 3><<<grid_for(max_n), kBlock, 0, st>>>(a, pk, pc, 0, 1 - pc, 1);
}

void launch_momentum_sweep(const SweepArgs &a, void *packs, int prec, int dim, int max_n, int sub,
                           cudaStream_t st) {
  if (prec == SPH_PREC_FP32)
    mom_dispatch<float>(a, packs, dim, max_n, sub, st);
  else
    mom_dispatch<double>(a, packs, dim, max_n, sub, st);
}

void launch_continuity_sweep(const SweepArgs &a, void *packs, int prec, int dim, int max_n, int sub,
                             cudaStream_t st) {
  if (prec == SPH_PREC_FP32)
    cont_dispatch<float>(a, packs, dim, max_n, sub, st);
  else
    cont_dispatch<double>(a, packs, dim, max_n, sub, st);
}

void launch_debug_pairs(const SweepArgs &a, const double *wx, const double *wy, const double *wz,
                        const uint32_t *wall_index, int64_t *out, int64_t max, unsigned long long *counter,
                        int max_n, cudaStream_t st) {
  k_pairs<<<grid_for(max_n), kBlock, 0, st>>>(a, wx, wy, wz, wall_index, out, max, counter);
}

}  // namespace sphk
