// sph_adjoint.cu -- reverse (adjoint) of one advection step for
// differentiated windows, FP64.
//
// The differentiated map is the step as the forward kernels compute it,
// with the discrete decisions of that step held: cell order, neighbour
// lists, labels, the buffer-update decisions, the guard of the B inverse,
// the time step (fixed) and, in RANS instances, k, eps and nu_t (held over
// the window).  Everything continuous is differentiated: positions enter
// through the pair geometry of every sweep (kernel gradient, the
// correction matrix B with dB = -B dA B, the mirror images at pressure
// buffers), densities through volumes and pressures, velocities through
// the viscous, momentum and continuity sums, and the inlet profile theta
// through the velocity boundary values and the recycling of injected
// particles (Sec. 2.4.2, 3.1).
//
// Reverse of a pair sum O_i = sum_j T(q_i, q_j, x_i - x_j) in gather form:
// thread i adds, over its list, the derivative of its own term T_ij with
// respect to its quantities (seeded by the adjoint of O_i) and of the
// neighbour's term T_ji (seeded by the adjoint of O_j), so no two threads
// write the same particle.  The mirror images of the B sum are not in the
// lists; their source terms are scattered with atomics into separate
// arrays.
#include "sph_pair.cuh"

namespace sphk {

namespace {

using G = Geo<double>;

// F = W'(r) / r and its r derivative
__device__ __forceinline__ void kernel_FF(const G &g, double r, double &F, double &Fr) {
  const double w = 1.0 - 0.5 * (r * g.inv_h);
  F = g.c5 * w * w * w;
  Fr = -1.5 * g.c5 * g.inv_h * w * w;
}

__device__ __forceinline__ double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// symmetric (xx, yy, zz, xy, xz, yz) -> full
__device__ __forceinline__ void sym_full(const double s[6], double M[3][3]) {
  M[0][0] = s[0];
  M[1][1] = s[1];
  M[2][2] = s[2];
  M[0][1] = M[1][0] = s[3];
  M[0][2] = M[2][0] = s[4];
  M[1][2] = M[2][1] = s[5];
}

// add the symmetric part of u (x) w to the stored symmetric adjoint
__device__ __forceinline__ void sym_acc(double s[6], const double u[3], const double w[3], double c) {
  s[0] += c * u[0] * w[0];
  s[1] += c * u[1] * w[1];
  s[2] += c * u[2] * w[2];
  s[3] += c * 0.5 * (u[0] * w[1] + u[1] * w[0]);
  s[4] += c * 0.5 * (u[0] * w[2] + u[2] * w[0]);
  s[5] += c * 0.5 * (u[1] * w[2] + u[2] * w[1]);
}

__device__ __forceinline__ int buffer_of(const AdjArgs &a, const InstDev &I, int i) {
  const int lab = a.m.label[i];
  return (lab > 0 && lab <= I.nbuf) ? I.buf0 + lab - 1 : -1;
}

__device__ __forceinline__ bool is_pressure(const AdjArgs &a, const InstDev &I, int i) {
  const int b = buffer_of(a, I, i);
  return b >= 0 && a.buf[b].type == SPH_BUF_PRESSURE;
}

__device__ __forceinline__ double rho_s(const AdjArgs &a, int s, int i) { return a.T.rho_s[(size_t)s * a.T.cap + i]; }

__device__ __forceinline__ void load_x0(const AdjArgs &a, int i, double x[3]) {
  x[0] = a.T.x0[0][i];
  x[1] = a.T.x0[1][i];
  x[2] = a.T.x0[2][i];
}

__device__ __forceinline__ void load_B(const AdjArgs &a, int i, int dim, double B[6]) {
  B[0] = a.der.B[0][i];
  B[1] = a.der.B[1][i];
  B[3] = a.der.B[3][i];
  if (dim == 3) {
    B[2] = a.der.B[2][i];
    B[4] = a.der.B[4][i];
    B[5] = a.der.B[5][i];
  } else {
    B[2] = B[4] = B[5] = 0.0;
  }
}

// minimum-image pair vector in FP64 (same rule as the forward)
template <int D, bool PER>
__device__ __forceinline__ double pvec(const G &g, const double xi[3], const double xj[3], double d[3]) {
  V4<double> pi{xi[0], xi[1], xi[2], 0.0}, pj{xj[0], xj[1], xj[2], 0.0};
  return pair_vec<double, D, PER>(g, pi, pj, d);
}

// velocity profile U(s1) of a buffer with its theta and s1 derivatives
__device__ __forceinline__ double profile_dU(const BufDev &b, double s1, int &k0, double &w0, int &k1, double &w1,
                                             double &dU_ds1) {
  k0 = 0;
  w0 = 1.0;
  k1 = 0;
  w1 = 0.0;
  dU_ds1 = 0.0;
  if (b.n_theta <= 1) return b.theta[0];
  const double w = b.half[0];
  const double u = (s1 + w) / (2.0 * w) * (double)(b.n_theta - 1);
  if (!(u > 0.0)) return b.theta[0];
  if (u >= (double)(b.n_theta - 1)) {
    k0 = b.n_theta - 1;
    return b.theta[k0];
  }
  const int k = (int)floor(u);
  const double f = u - (double)k;
  k0 = k;
  w0 = 1.0 - f;
  k1 = k + 1;
  w1 = f;
  dU_ds1 = (b.theta[k + 1] - b.theta[k]) * (double)(b.n_theta - 1) / (2.0 * w);
  return b.theta[k] + f * (b.theta[k + 1] - b.theta[k]);
}

// reverse of the velocity boundary value v = U(s1(x)) (n_b + noise xi) at
// position x: theta gradient (profile of the differentiated buffer only),
// position adjoint, and the velocity adjoint is consumed
__device__ void velocity_bc_rev(const AdjArgs &a, const InstDev &I, int bidx, int i, const double x[3],
                                int64_t step, uint32_t sub, double lv[3], double lx[3]) {
  const BufDev &b = a.buf[bidx];
  const double s1 = local_coord(b, I.dim, x[0], x[1], x[2], 1);
  int k0, k1;
  double w0, w1, dU;
  profile_dU(b, s1, k0, w0, k1, w1, dU);
  double xi[3] = {0.0, 0.0, 0.0};
  if (b.noise != 0.0) {
    uint32_t c[4] = {(uint32_t)step, sub, 0u, 0u};
    philox4x32_10(c, I.seed, a.m.uid[i]);
    xi[0] = uniform_pm1(c[0], c[1]);
    xi[1] = uniform_pm1(c[2], c[3]);
    if (I.dim == 3) {
      uint32_t c2[4] = {(uint32_t)step, sub, 1u, 0u};
      philox4x32_10(c2, I.seed, a.m.uid[i]);
      xi[2] = uniform_pm1(c2[0], c2[1]);
    }
  }
  double ld = 0.0;
  for (int c = 0; c < I.dim; ++c) ld += lv[c] * (b.frame[c] + b.noise * xi[c]);
  const int ii = a.m.inst[i];
  if (ii == a.g_inst && bidx == I.buf0 + a.g_buf) {
    atomicAdd(&a.grad[k0], ld * w0);
    if (w1 != 0.0) atomicAdd(&a.grad[k1], ld * w1);
  }
  for (int c = 0; c < I.dim; ++c) {
    lx[c] += ld * dU * b.frame[3 + c];
    lv[c] = 0.0;
  }
}

}  // namespace

// ------------------------------------------------------------------------
// tape kernels (run inside the recomputed forward step)
// ------------------------------------------------------------------------
__global__ void k_adj_tape_start(AdjArgs a) {
  const int n = a.cnt->n_live;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    for (int c = 0; c < 3; ++c) {
      a.T.x0[c][i] = a.m.x[c][i];
      a.T.v0[c][i] = a.m.v[c][i];
    }
    a.T.rho0[i] = a.m.rho[i];
    a.T.drho0[i] = a.m.drho[i];
  }
}

__global__ void k_adj_tape_sub(AdjArgs a, int s) {
  const int n = a.cnt->n_live;
  const size_t o = (size_t)s * a.T.cap;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    a.T.rho_s[o + i] = a.m.rho[i];
    for (int c = 0; c < 3; ++c) {
      a.T.v1[c][o + i] = a.m.v[c][i];
      a.T.xbc[c][o + i] = a.m.x[c][i];
    }
  }
}

__global__ void k_adj_tape_drho(AdjArgs a, int s) {
  const int n = a.cnt->n_live;
  const size_t o = (size_t)s * a.T.cap;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    a.T.drho_s[o + i] = a.m.drho[i];
}

// ------------------------------------------------------------------------
// objective: J = sum over steps dt sum_{i in S} m_i v_i . n_out / w_s,
// S = particles of the objective instance labelled in one of the chosen
// buffers at window start (by uid), n_out = -n_b; evaluated on the state
// after each step's buffer update (deleted entries excluded)
// ------------------------------------------------------------------------
__global__ void k_adj_region(AdjArgs a, uint8_t *region, const int32_t *obj_mask) {
  const int n = a.cnt->m_pending;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (a.m.inst[i] != a.o_inst || a.pending_keys[i] == a.sentinel) continue;
    const InstDev &I = a.inst[a.o_inst];
    const int lab = a.m.label[i];
    if (lab < 1 || lab > I.nbuf || !obj_mask[lab - 1]) continue;
    const uint32_t u = a.m.uid[i];
    if ((int64_t)u < a.n_region) region[u] = (uint8_t)lab;
  }
}

__device__ __forceinline__ double member_weight(const AdjArgs &a, int i, double nout[3]) {
  if (a.m.inst[i] != a.o_inst || a.pending_keys[i] == a.sentinel) return 0.0;
  const uint32_t u = a.m.uid[i];
  if ((int64_t)u >= a.n_region) return 0.0;
  const int lab = a.region[u];
  if (!lab) return 0.0;
  const InstDev &I = a.inst[a.o_inst];
  const BufDev &b = a.buf[I.buf0 + lab - 1];
  for (int c = 0; c < 3; ++c) nout[c] = c < I.dim ? -b.frame[c] : 0.0;
  return a.dt_obj * a.m.mass[i] / a.w_s;
}

__global__ void k_adj_objective(AdjArgs a, int seed) {
  const int n = a.cnt->m_pending;
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double nout[3];
    const double w = member_weight(a, i, nout);
    if (w == 0.0) continue;
    if (seed) {
      for (int c = 0; c < 3; ++c) a.lv[c][i] += w * nout[c];
    } else {
      acc += w * (a.m.v[0][i] * nout[0] + a.m.v[1][i] * nout[1] + a.m.v[2][i] * nout[2]);
    }
  }
  if (!seed) {
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(a.J, acc);
  }
}

// ------------------------------------------------------------------------
// reverse of the buffer update: the injecting particle's copy inherited its
// pre-recycle state; the particle itself was shifted by -L_b n_b and given
// boundary values
// ------------------------------------------------------------------------
__global__ void k_adj_buffer_rev(AdjArgs a) {
  if (a.cnt->overflow) return;  // nothing was committed
  const int n = a.cnt->n_live;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (a.flag[i] != 1) continue;  // injection
    const InstDev &I = a.inst[a.m.inst[i]];
    const int b = buffer_of(a, I, i);
    if (b < 0) continue;
    double lv[3] = {a.lv[0][i], a.lv[1][i], a.lv[2][i]};
    double lx[3] = {a.lx[0][i], a.lx[1][i], a.lx[2][i]};
    if (a.buf[b].type == SPH_BUF_VELOCITY) {
      const double x[3] = {a.m.x[0][i], a.m.x[1][i], a.m.x[2][i]};
      velocity_bc_rev(a, I, b, i, x, a.cnt->spawn_step, kSubRecycle, lv, lx);
    } else {
      a.lrho[i] = 0.0;
    }
    const int d = a.T.spawn_dst[i];
    if (d < n || (int64_t)d >= a.T.cap) continue;
    for (int c = 0; c < 3; ++c) {
      a.lv[c][i] = lv[c] + a.lv[c][d];
      a.lx[c][i] = lx[c] + a.lx[c][d];
    }
    a.lrho[i] += a.lrho[d];
    a.ldrho[i] += a.ldrho[d];
  }
}

// ------------------------------------------------------------------------
// reverse of one acoustic sub-step
// ------------------------------------------------------------------------
// Per-particle records of the reverse pair passes (FP64, V4 units), written
// by the point kernel before each pass so that a neighbour costs one
// contiguous read:
//   C (continuity)  2D (x y V p)(vx vy ls -)        3D (x y z V)(p vx vy vz)(ls - - -)
//   M (momentum)    2D (x y V pe)(Bxx Bxy Byy mk)   3D (x y z V)(pe mk Bxx Byy)(Bzz Bxy Bxz Byz)
//   S (mom. seeds)  2D (a1 ab)(a2 at)               3D (a1 abx)(aby abz a2x a2y)(a2z at)
//   A (advection)   2D (x y V mu)(vx vy mir Lxx)(Lyy Lxy sx sy)
//                   3D (x y z V)(vx vy vz mu)(mir Lxx Lyy Lzz)(Lxy Lxz Lyz sx)(sy sz - -)
// with ls the continuity seed, mk 1 for pressure-buffer particles, a1..at
// the momentum seeds, L the adjoint of A and s the adjoint of the viscous
// sum, mir the buffer index of a pressure-buffer particle or -1.
template <int D>
struct RecW {
  static constexpr int C = D == 2 ? 2 : 3, M = D == 2 ? 2 : 3, S = D == 2 ? 2 : 3, A = D == 2 ? 3 : 5;
};

struct CRec {
  double x[3], V, p, v[3], ls;
};
struct MRec {
  double x[3], V, pe, B[6];
  bool mk;
};
struct SRec {
  double a1[3], ab[3], a2[3], at[3];
};
struct ARec {
  double x[3], V, v[3], mu, L[6], sg[3];
  int mir;
};

template <int D>
__device__ __forceinline__ void put_c(V4<double> *r, int i, const CRec &c) {
  V4<double> *p = r + (size_t)RecW<D>::C * i;
  if (D == 2) {
    p[0] = V4<double>{c.x[0], c.x[1], c.V, c.p};
    p[1] = V4<double>{c.v[0], c.v[1], c.ls, 0.0};
  } else {
    p[0] = V4<double>{c.x[0], c.x[1], c.x[2], c.V};
    p[1] = V4<double>{c.p, c.v[0], c.v[1], c.v[2]};
    p[2] = V4<double>{c.ls, 0.0, 0.0, 0.0};
  }
}
template <int D>
__device__ __forceinline__ CRec get_c(const V4<double> *r, int i) {
  const V4<double> *p = r + (size_t)RecW<D>::C * i;
  CRec c;
  const V4<double> q0 = p[0], q1 = p[1];
  if (D == 2) {
    c.x[0] = q0.x, c.x[1] = q0.y, c.x[2] = 0.0, c.V = q0.z, c.p = q0.w;
    c.v[0] = q1.x, c.v[1] = q1.y, c.v[2] = 0.0, c.ls = q1.z;
  } else {
    const V4<double> q2 = p[2];
    c.x[0] = q0.x, c.x[1] = q0.y, c.x[2] = q0.z, c.V = q0.w;
    c.p = q1.x, c.v[0] = q1.y, c.v[1] = q1.z, c.v[2] = q1.w, c.ls = q2.x;
  }
  return c;
}
template <int D>
__device__ __forceinline__ void put_m(V4<double> *r, int i, const MRec &m) {
  V4<double> *p = r + (size_t)RecW<D>::M * i;
  const double mk = m.mk ? 1.0 : 0.0;
  if (D == 2) {
    p[0] = V4<double>{m.x[0], m.x[1], m.V, m.pe};
    p[1] = V4<double>{m.B[0], m.B[3], m.B[1], mk};
  } else {
    p[0] = V4<double>{m.x[0], m.x[1], m.x[2], m.V};
    p[1] = V4<double>{m.pe, mk, m.B[0], m.B[1]};
    p[2] = V4<double>{m.B[2], m.B[3], m.B[4], m.B[5]};
  }
}
template <int D>
__device__ __forceinline__ MRec get_m(const V4<double> *r, int i) {
  const V4<double> *p = r + (size_t)RecW<D>::M * i;
  MRec m;
  const V4<double> q0 = p[0], q1 = p[1];
  if (D == 2) {
    m.x[0] = q0.x, m.x[1] = q0.y, m.x[2] = 0.0, m.V = q0.z, m.pe = q0.w;
    m.B[0] = q1.x, m.B[3] = q1.y, m.B[1] = q1.z, m.mk = q1.w != 0.0;
    m.B[2] = m.B[4] = m.B[5] = 0.0;
  } else {
    const V4<double> q2 = p[2];
    m.x[0] = q0.x, m.x[1] = q0.y, m.x[2] = q0.z, m.V = q0.w;
    m.pe = q1.x, m.mk = q1.y != 0.0, m.B[0] = q1.z, m.B[1] = q1.w;
    m.B[2] = q2.x, m.B[3] = q2.y, m.B[4] = q2.z, m.B[5] = q2.w;
  }
  return m;
}
template <int D>
__device__ __forceinline__ void put_s(V4<double> *r, int i, const SRec &s) {
  V4<double> *p = r + (size_t)RecW<D>::S * i;
  if (D == 2) {
    p[0] = V4<double>{s.a1[0], s.a1[1], s.ab[0], s.ab[1]};
    p[1] = V4<double>{s.a2[0], s.a2[1], s.at[0], s.at[1]};
  } else {
    p[0] = V4<double>{s.a1[0], s.a1[1], s.a1[2], s.ab[0]};
    p[1] = V4<double>{s.ab[1], s.ab[2], s.a2[0], s.a2[1]};
    p[2] = V4<double>{s.a2[2], s.at[0], s.at[1], s.at[2]};
  }
}
template <int D>
__device__ __forceinline__ SRec get_s(const V4<double> *r, int i) {
  const V4<double> *p = r + (size_t)RecW<D>::S * i;
  SRec s;
  const V4<double> q0 = p[0], q1 = p[1];
  if (D == 2) {
    s.a1[0] = q0.x, s.a1[1] = q0.y, s.ab[0] = q0.z, s.ab[1] = q0.w;
    s.a2[0] = q1.x, s.a2[1] = q1.y, s.at[0] = q1.z, s.at[1] = q1.w;
    s.a1[2] = s.ab[2] = s.a2[2] = s.at[2] = 0.0;
  } else {
    const V4<double> q2 = p[2];
    s.a1[0] = q0.x, s.a1[1] = q0.y, s.a1[2] = q0.z, s.ab[0] = q0.w;
    s.ab[1] = q1.x, s.ab[2] = q1.y, s.a2[0] = q1.z, s.a2[1] = q1.w;
    s.a2[2] = q2.x, s.at[0] = q2.y, s.at[1] = q2.z, s.at[2] = q2.w;
  }
  return s;
}
template <int D>
__device__ __forceinline__ void put_a(V4<double> *r, int i, const ARec &q) {
  V4<double> *p = r + (size_t)RecW<D>::A * i;
  const double mir = (double)q.mir;
  if (D == 2) {
    p[0] = V4<double>{q.x[0], q.x[1], q.V, q.mu};
    p[1] = V4<double>{q.v[0], q.v[1], mir, q.L[0]};
    p[2] = V4<double>{q.L[1], q.L[3], q.sg[0], q.sg[1]};
  } else {
    p[0] = V4<double>{q.x[0], q.x[1], q.x[2], q.V};
    p[1] = V4<double>{q.v[0], q.v[1], q.v[2], q.mu};
    p[2] = V4<double>{mir, q.L[0], q.L[1], q.L[2]};
    p[3] = V4<double>{q.L[3], q.L[4], q.L[5], q.sg[0]};
    p[4] = V4<double>{q.sg[1], q.sg[2], 0.0, 0.0};
  }
}
template <int D>
__device__ __forceinline__ ARec get_a(const V4<double> *r, int i) {
  const V4<double> *p = r + (size_t)RecW<D>::A * i;
  ARec q;
  const V4<double> q0 = p[0], q1 = p[1], q2 = p[2];
  if (D == 2) {
    q.x[0] = q0.x, q.x[1] = q0.y, q.x[2] = 0.0, q.V = q0.z, q.mu = q0.w;
    q.v[0] = q1.x, q.v[1] = q1.y, q.v[2] = 0.0, q.mir = (int)q1.z, q.L[0] = q1.w;
    q.L[1] = q2.x, q.L[3] = q2.y, q.sg[0] = q2.z, q.sg[1] = q2.w;
    q.L[2] = q.L[4] = q.L[5] = 0.0;
    q.sg[2] = 0.0;
  } else {
    const V4<double> q3 = p[3], q4 = p[4];
    q.x[0] = q0.x, q.x[1] = q0.y, q.x[2] = q0.z, q.V = q0.w;
    q.v[0] = q1.x, q.v[1] = q1.y, q.v[2] = q1.z, q.mu = q1.w;
    q.mir = (int)q2.x, q.L[0] = q2.y, q.L[1] = q2.z, q.L[2] = q2.w;
    q.L[3] = q3.x, q.L[4] = q3.y, q.L[5] = q3.z, q.sg[0] = q3.w;
    q.sg[1] = q4.x, q.sg[2] = q4.y;
  }
  return q;
}

// R1: boundary values and the density update of sub-step s; writes the
// continuity record
template <int D>
__global__ void k_adj_bc_density(AdjArgs a, int s) {
  const int n = a.cnt->n_live;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const InstDev &I = a.inst[a.m.inst[i]];
    if (s >= I.n_ac) continue;
    const double hdt = 0.5 * I.dt;
    const size_t o = (size_t)s * a.T.cap + i;
    const int b = buffer_of(a, I, i);
    if (b >= 0) {
      if (a.buf[b].type == SPH_BUF_VELOCITY) {
        double lv[3] = {a.lv[0][i], a.lv[1][i], a.lv[2][i]};
        double lx[3] = {a.lx[0][i], a.lx[1][i], a.lx[2][i]};
        const double x[3] = {a.T.xbc[0][o], a.T.xbc[1][o], a.T.xbc[2][o]};
        velocity_bc_rev(a, I, b, i, x, a.cnt->spawn_step, (uint32_t)s, lv, lx);
        for (int c = 0; c < 3; ++c) {
          a.lv[c][i] = lv[c];
          a.lx[c][i] = lx[c];
        }
      } else {
        a.lrho[i] = 0.0;
      }
    }
    // rho' = rho_s + hdt drho, drho = rho_s Sigma
    const double rs = a.T.rho_s[o];
    const double Sig = a.T.drho_s[o] / rs;
    const double ltot = a.ldrho[i] + hdt * a.lrho[i];
    a.lrho[i] += ltot * Sig;
    a.ldrho[i] = 0.0;
    CRec c;
    load_x0(a, i, c.x);
    c.V = a.m.mass[i] / rs;
    c.p = I.c0sq * (rs - I.rho0);
    for (int q = 0; q < 3; ++q) c.v[q] = a.T.v1[q][o];
    c.ls = ltot * rs;
    put_c<D>(a.rc, i, c);
  }
}

// R2: continuity sum  Sigma_i = sum_j [v_ij . r_ij + (p_i - p_j) r / (rho0 c0)] F V_j
template <int D, bool PER>
__global__ void k_adj_cont(AdjArgs a, int s) {
  const int n = a.cnt->n_live;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const InstDev &I = a.inst[a.m.inst[i]];
    if (s >= I.n_ac) continue;
    const G g = make_geo<double, D>(I);
    const double kap = I.inv_rc0;
    const CRec ci = get_c<D>(a.rc, i);
    const double lsi = ci.ls;
    double lvi[3] = {0, 0, 0}, lxi[3] = {0, 0, 0}, lpi = 0.0, lVi = 0.0;
    const int nr = a.nl.n_real[i], nw = a.nl.n_wall[i];
    const uint32_t *L = list_of(a.nl, i);
#pragma unroll 2
    for (int kk = 0; kk < nr; ++kk) {
      const int j = (int)list_at(L, kk);
      const CRec cj = get_c<D>(a.rc, j);
      double d[3];
      const double rr_ = pvec<D, PER>(g, ci.x, cj.x, d);
      const double ir = rsqrt(rr_), r = rr_ * ir;
      double F, Fr;
      kernel_FF(g, r, F, Fr);
      const double vv[3] = {ci.v[0] - cj.v[0], ci.v[1] - cj.v[1], ci.v[2] - cj.v[2]};
      const double vd = dot3(vv, d), dp = ci.p - cj.p;
      // own term (seed lsi)
      const double br = vd + dp * kap * r;
      // neighbour's term (seed lsj), i as its source
      const double br2 = vd - dp * kap * r;
      const double lsj = cj.ls;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        lvi[c] += (lsi * cj.V + lsj * ci.V) * F * d[c];
        lxi[c] += lsi * cj.V * (F * vv[c] + br * Fr * d[c] * ir + dp * kap * F * d[c] * ir) +
                  lsj * ci.V * (F * vv[c] + br2 * Fr * d[c] * ir - dp * kap * F * d[c] * ir);
      }
      lpi += (lsi * cj.V - lsj * ci.V) * kap * r * F;
      lVi += lsj * br2 * F;
    }
    for (int kk = nr; kk < nr + nw; ++kk) {
      const int w = (int)list_at(L, kk);
      const double xw[3] = {a.wx[0][w], a.wx[1][w], a.wx[2][w]};
      double d[3];
      const double rr_ = pvec<D, PER>(g, ci.x, xw, d);
      const double ir = rsqrt(rr_), r = rr_ * ir;
      double F, Fr;
      kernel_FF(g, r, F, Fr);
      const V4<double> Wv = a.WV[w];
      const double vv[3] = {ci.v[0] - Wv.x, ci.v[1] - Wv.y, ci.v[2] - Wv.z};
      const double vd = dot3(vv, d), Vw = I.Vw;
      for (int c = 0; c < D; ++c) {
        lvi[c] += lsi * 2.0 * F * Vw * d[c];
        lxi[c] += lsi * 2.0 * Vw * (F * vv[c] + vd * Fr * d[c] * ir);
      }
    }
    for (int c = 0; c < D; ++c) {
      a.lv[c][i] += lvi[c];
      a.lxg[c][i] += lxi[c];
    }
    a.lrho[i] += I.c0sq * lpi - (ci.V / a.T.rho_s[(size_t)s * a.T.cap + i]) * lVi;
  }
}

// R3a: reverse of the kick and half drift; writes the momentum record
template <int D>
__global__ void k_adj_mom_rec(AdjArgs a, int s) {
  const int n = a.cnt->n_live;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const InstDev &I = a.inst[a.m.inst[i]];
    if (s >= I.n_ac) continue;
    const double dt = I.dt, hdt = 0.5 * I.dt, c0sq = I.c0sq;
    for (int c = 0; c < D; ++c) {
      const double lv = a.lv[c][i] + hdt * a.lx[c][i];
      a.lv[c][i] = lv;
      a.sd[c][i] = dt * lv;  // adjoint of the pressure acceleration
      a.lan[c][i] += dt * lv;
    }
    MRec m;
    load_x0(a, i, m.x);
    const double rs = rho_s(a, s, i), p = c0sq * (rs - I.rho0);
    const double kw = I.rans ? (2.0 / 3.0) * a.m.k[i] : 0.0;
    m.V = a.m.mass[i] / rs;
    m.pe = I.rans ? p + kw * (I.rho0 + p / c0sq) : p;
    load_B(a, i, D, m.B);
    m.mk = is_pressure(a, I, i);
    put_m<D>(a.rm, i, m);
  }
}

// R3b: the seeds a1 (S1), ab (Cb), a2 (S2), at (Ct) from the momentum sums
// the forward step recorded, and the direct dependence on rho_i (1/rho_i,
// p_i, compensation) and B_i
template <int D>
__global__ void k_adj_mom_seed(AdjArgs a, int s) {
  const int n = a.cnt->n_live;
  const size_t cap = (size_t)a.T.cap;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const InstDev &I = a.inst[a.m.inst[i]];
    if (s >= I.n_ac) continue;
    const double c0sq = I.c0sq;
    const MRec mi = get_m<D>(a.rm, i);
    const double la[3] = {a.sd[0][i], a.sd[1][i], D == 3 ? a.sd[2][i] : 0.0};
    const double *t = a.T.S + (size_t)s * 12 * cap + i;
    double S1[3], Cb[3], S2[3], Ct[3];
    for (int c = 0; c < 3; ++c) {
      S1[c] = t[(0 + c) * cap];
      Cb[c] = t[(3 + c) * cap];
      S2[c] = t[(6 + c) * cap];
      Ct[c] = t[(9 + c) * cap];
    }
    const double rsi = rho_s(a, s, i);
    const double kwi = I.rans ? (2.0 / 3.0) * a.m.k[i] : 0.0;
    const bool comp = mi.mk;
    double pob = comp ? a.buf[buffer_of(a, I, i)].p_ob : 0.0;
    if (comp && I.rans) pob += (2.0 / 3.0) * rsi * a.m.k[i];
    double Bla[3], BCb[3], BS2[3], BCt[3];
    sym_matvec<double, D>(mi.B, la, Bla);
    sym_matvec<double, D>(mi.B, Cb, BCb);
    sym_matvec<double, D>(mi.B, S2, BS2);
    sym_matvec<double, D>(mi.B, Ct, BCt);
    const double inv = 1.0 / rsi;
    SRec sr;
    for (int c = 0; c < 3; ++c) {
      sr.a1[c] = c < D ? -mi.pe * inv * la[c] : 0.0;
      sr.ab[c] = c < D ? -mi.pe * inv * Bla[c] : 0.0;
      sr.a2[c] = c < D ? -inv * Bla[c] : 0.0;
      sr.at[c] = (c < D && comp) ? 2.0 * pob * inv * Bla[c] : 0.0;
    }
    put_s<D>(a.rs, i, sr);
    double accp = 0.0, accc = 0.0, lpe = 0.0;
    for (int c = 0; c < D; ++c) {
      accp += la[c] * (-(mi.pe * (S1[c] + BCb[c]) + BS2[c]) * inv);
      if (comp) accc += la[c] * 2.0 * pob * inv * BCt[c];
      lpe += -inv * la[c] * (S1[c] + BCb[c]);
    }
    double lrho = -(accp + accc) * inv + lpe * (c0sq + kwi);
    if (comp && I.rans) {
      double tt = 0.0;
      for (int c = 0; c < D; ++c) tt += la[c] * BCt[c];
      lrho += 2.0 * inv * (2.0 / 3.0) * a.m.k[i] * tt;
    }
    a.lrho[i] += lrho;
    double lB[6] = {0, 0, 0, 0, 0, 0};
    sym_acc(lB, la, Cb, -mi.pe * inv);
    sym_acc(lB, la, S2, -inv);
    if (comp) sym_acc(lB, la, Ct, 2.0 * pob * inv);
    for (int q = 0; q < 6; ++q) a.lB[q][i] += lB[q];
  }
}

// R4: momentum pair reverse
template <int D, bool PER>
__global__ void k_adj_mom(AdjArgs a, int s) {
  const int n = a.cnt->n_live;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const InstDev &I = a.inst[a.m.inst[i]];
    if (s >= I.n_ac) continue;
    const G g = make_geo<double, D>(I);
    const MRec mi = get_m<D>(a.rm, i);
    const SRec si = get_s<D>(a.rs, i);
    double lxi[3] = {0, 0, 0}, lB[6] = {0, 0, 0, 0, 0, 0}, lpe = 0.0, lVi = 0.0;
    const int nr = a.nl.n_real[i], nw = a.nl.n_wall[i];
    const uint32_t *L = list_of(a.nl, i);
#pragma unroll 2
    for (int kk = 0; kk < nr; ++kk) {
      const int j = (int)list_at(L, kk);
      const MRec mj = get_m<D>(a.rm, j);
      const SRec sj = get_s<D>(a.rs, j);
      double d[3];
      const double rr_ = pvec<D, PER>(g, mi.x, mj.x, d);
      const double ir = rsqrt(rr_), r = rr_ * ir;
      double F, Fr;
      kernel_FF(g, r, F, Fr);
      // own term: L = G . gw, gw = V_j F d
      double Gv[3];
      if (mj.mk) {
        for (int c = 0; c < 3; ++c) Gv[c] = si.ab[c];
      } else {
        sym_matvec<double, D>(mj.B, si.a1, Gv);
      }
      for (int c = 0; c < D; ++c) Gv[c] += mj.pe * si.a2[c] + si.at[c];
      // neighbour's term with i as its source: gw' = -V_i F d
      double Gp[3];
      if (mi.mk) {
        for (int c = 0; c < 3; ++c) Gp[c] = sj.ab[c];
      } else {
        sym_matvec<double, D>(mi.B, sj.a1, Gp);
      }
      for (int c = 0; c < D; ++c) Gp[c] += mi.pe * sj.a2[c] + sj.at[c];
      const double gwp[3] = {-mi.V * F * d[0], -mi.V * F * d[1], -mi.V * F * d[2]};
      if (!mi.mk) sym_acc(lB, sj.a1, gwp, 1.0);
      double Gd = 0.0, Gpd = 0.0, a2g = 0.0;
      for (int c = 0; c < D; ++c) {
        Gd += Gv[c] * d[c];
        Gpd += Gp[c] * d[c];
        a2g += sj.a2[c] * gwp[c];
      }
      lpe += a2g;
      lVi += -F * Gpd;
      for (int c = 0; c < D; ++c)
        lxi[c] += mj.V * (F * Gv[c] + Gd * Fr * d[c] * ir) - mi.V * (F * Gp[c] + Gpd * Fr * d[c] * ir);
    }
    for (int kk = nr; kk < nr + nw; ++kk) {
      const int w = (int)list_at(L, kk);
      const double xw[3] = {a.wx[0][w], a.wx[1][w], a.wx[2][w]};
      double d[3];
      const double rr_ = pvec<D, PER>(g, mi.x, xw, d);
      const double ir = rsqrt(rr_), r = rr_ * ir;
      double F, Fr;
      kernel_FF(g, r, F, Fr);
      double Gv[3], Gd = 0.0, a2g = 0.0;
      for (int c = 0; c < D; ++c) {
        Gv[c] = si.ab[c] + mi.pe * si.a2[c] + si.at[c];
        Gd += Gv[c] * d[c];
        a2g += si.a2[c] * I.Vw * F * d[c];
      }
      lpe += a2g;
      for (int c = 0; c < D; ++c) lxi[c] += I.Vw * (F * Gv[c] + Gd * Fr * d[c] * ir);
    }
    const double rsi = rho_s(a, s, i);
    const double kwi = I.rans ? (2.0 / 3.0) * a.m.k[i] : 0.0;
    for (int c = 0; c < D; ++c) a.lxg[c][i] += lxi[c];
    for (int q = 0; q < 6; ++q) a.lB[q][i] += lB[q];
    a.lrho[i] += lpe * (I.c0sq + kwi) - (mi.V / rsi) * lVi;
  }
}

// R5: reverse of the first half of sub-step s: rho_s = rho + hdt drho,
// x += hdt v
__global__ void k_adj_half1(AdjArgs a, int s) {
  const int n = a.cnt->n_live;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const InstDev &I = a.inst[a.m.inst[i]];
    if (s >= I.n_ac) continue;
    const double hdt = 0.5 * I.dt;
    a.ldrho[i] += hdt * a.lrho[i];
    for (int c = 0; c < I.dim; ++c) a.lv[c][i] += hdt * a.lx[c][i];
  }
}

// ------------------------------------------------------------------------
// reverse of the advection sweep: B (with mirror images) and the viscous
// acceleration, from the adjoints of B (lB) and a_nu (lan)
// ------------------------------------------------------------------------
template <int D>
__global__ void k_adj_adv_seed(AdjArgs a) {
  const int n = a.cnt->n_live;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const InstDev &I = a.inst[a.m.inst[i]];
    const double rho = a.T.rho0[i];
    ARec q;
    double t = 0.0;
    for (int c = 0; c < 3; ++c) {
      const double l = c < D ? a.lan[c][i] : 0.0;
      q.sg[c] = 2.0 * l / rho;
      if (c < D) t += a.der.an[c][i] * l;
    }
    a.lrho[i] -= t / rho;
    // lambda_A = -B Lambda_B B unless the guard replaced B by I
    double Bs[6];
    load_B(a, i, D, Bs);
    const bool guard = Bs[0] == 1.0 && Bs[1] == 1.0 && Bs[3] == 0.0 &&
                       (D == 2 || (Bs[2] == 1.0 && Bs[4] == 0.0 && Bs[5] == 0.0));
    for (int c = 0; c < 6; ++c) q.L[c] = 0.0;
    if (!guard) {
      double B[3][3], Lm[3][3], T[3][3], R[3][3];
      sym_full(Bs, B);
      const double lb[6] = {a.lB[0][i], a.lB[1][i], a.lB[2][i], a.lB[3][i], a.lB[4][i], a.lB[5][i]};
      sym_full(lb, Lm);
      for (int p = 0; p < 3; ++p)
        for (int r = 0; r < 3; ++r) T[p][r] = Lm[p][0] * B[0][r] + Lm[p][1] * B[1][r] + Lm[p][2] * B[2][r];
      for (int p = 0; p < 3; ++p)
        for (int r = 0; r < 3; ++r) R[p][r] = -(B[p][0] * T[0][r] + B[p][1] * T[1][r] + B[p][2] * T[2][r]);
      q.L[0] = R[0][0];
      q.L[1] = R[1][1];
      q.L[2] = R[2][2];
      q.L[3] = 0.5 * (R[0][1] + R[1][0]);
      q.L[4] = 0.5 * (R[0][2] + R[2][0]);
      q.L[5] = 0.5 * (R[1][2] + R[2][1]);
    }
    load_x0(a, i, q.x);
    q.V = a.m.mass[i] / rho;
    for (int c = 0; c < 3; ++c) q.v[c] = a.T.v0[c][i];
    q.mu = I.rho0 * (I.nu_l + (I.rans ? a.m.nut[i] : 0.0));
    const int b = buffer_of(a, I, i);
    q.mir = (b >= 0 && a.buf[b].type == SPH_BUF_PRESSURE) ? b : -1;
    put_a<D>(a.ra, i, q);
  }
}

// viscous coefficient of a pair and whether the ARD term is the active one
__device__ __forceinline__ double visc_mu(const InstDev &I, double mu_a, double mu_b, bool harmonic,
                                          const double vv[3], const double d[3], double ir, bool &ard) {
  ard = false;
  if (!I.rans) return mu_a;
  const double mut = harmonic ? 2.0 * mu_a * mu_b / (mu_a + mu_b) : mu_a;
  const double ve = -dot3(vv, d) * ir;
  const double lim = I.eta * (ve > 0.0 ? ve : 0.0);
  const double muR = I.muR_k * (lim < I.c0 ? lim : I.c0);
  if (mut > muR) return mut;
  ard = ve > 0.0 && lim < I.c0;
  return muR;
}

template <int D>
__device__ __forceinline__ void sym_apply(const double L[6], const double d[3], double u[3]) {
  u[0] = L[0] * d[0] + L[3] * d[1] + L[4] * d[2];
  u[1] = L[3] * d[0] + L[1] * d[1] + L[5] * d[2];
  u[2] = L[4] * d[0] + L[5] * d[1] + L[2] * d[2];
}

template <int D, bool PER>
__global__ void k_adj_adv(AdjArgs a) {
  const int n = a.cnt->n_live;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const InstDev &I = a.inst[a.m.inst[i]];
    const G g = make_geo<double, D>(I);
    const double reg = I.reg, kR = I.muR_k * I.eta;
    const ARec qi = get_a<D>(a.ra, i);
    const bool mir_i = qi.mir >= 0;
    double lvi[3] = {0, 0, 0}, lxi[3] = {0, 0, 0}, lVi = 0.0;
    const int nr = a.nl.n_real[i], nw = a.nl.n_wall[i];
    const uint32_t *L = list_of(a.nl, i);
#pragma unroll 2
    for (int kk = 0; kk < nr; ++kk) {
      const int j = (int)list_at(L, kk);
      const ARec qj = get_a<D>(a.ra, j);
      double d[3];
      const double rr_ = pvec<D, PER>(g, qi.x, qj.x, d);
      const double ir = rsqrt(rr_), r = rr_ * ir;
      double F, Fr;
      kernel_FF(g, r, F, Fr);
      const double vv[3] = {qi.v[0] - qj.v[0], qi.v[1] - qj.v[1], qi.v[2] - qj.v[2]};
      bool ard;
      const double mu = visc_mu(I, qi.mu, qj.mu, true, vv, d, ir, ard);
      const double irg = 1.0 / (r + reg);
      const double rf = r * irg, dfr = Fr * rf + F * reg * irg * irg;
      const double vd = dot3(vv, d);
      // ---- own terms (seeds of i) ----
      if (!mir_i || !(local_coord(a.buf[qi.mir], D, qj.x[0], qj.x[1], qj.x[2], 0) < 0.0)) {
        double u[3];
        sym_apply<D>(qi.L, d, u);
        const double q = dot3(d, u);
        for (int c = 0; c < D; ++c) lxi[c] += -qj.V * (Fr * q * d[c] * ir + 2.0 * F * u[c]);
      }
      {
        const double f = F * rf * qj.V, sv = dot3(qi.sg, vv);
        for (int c = 0; c < D; ++c) {
          lvi[c] += mu * f * qi.sg[c];
          lxi[c] += mu * sv * qj.V * dfr * d[c] * ir;
        }
        if (ard) {
          const double Lm = f * sv * kR;
          for (int c = 0; c < D; ++c) {
            lvi[c] += -Lm * d[c] * ir;
            lxi[c] += Lm * (-vv[c] * ir + vd * d[c] * (ir * ir * ir));
          }
        }
      }
      // ---- neighbour's terms (seeds of j), i as the source ----
      if (!(qj.mir >= 0) || !(local_coord(a.buf[qj.mir], D, qi.x[0], qi.x[1], qi.x[2], 0) < 0.0)) {
        double u[3];
        sym_apply<D>(qj.L, d, u);
        const double q = dot3(d, u);
        lVi += -F * q;
        for (int c = 0; c < D; ++c) lxi[c] += -qi.V * (Fr * q * d[c] * ir + 2.0 * F * u[c]);
      }
      {
        const double fp = F * rf * qi.V, svp = -dot3(qj.sg, vv);  // v_ji = -v_ij
        for (int c = 0; c < D; ++c) {
          lvi[c] += -mu * fp * qj.sg[c];
          lxi[c] += mu * svp * qi.V * dfr * d[c] * ir;
        }
        lVi += mu * F * rf * svp;
        if (ard) {
          const double Lm = fp * svp * kR;
          for (int c = 0; c < D; ++c) {
            lvi[c] += -Lm * d[c] * ir;
            lxi[c] += Lm * (-vv[c] * ir + vd * d[c] * (ir * ir * ir));
          }
        }
      }
    }
    for (int kk = nr; kk < nr + nw; ++kk) {
      const int w = (int)list_at(L, kk);
      const double xw[3] = {a.wx[0][w], a.wx[1][w], a.wx[2][w]};
      double d[3];
      const double rr_ = pvec<D, PER>(g, qi.x, xw, d);
      const double ir = rsqrt(rr_), r = rr_ * ir;
      double F, Fr;
      kernel_FF(g, r, F, Fr);
      const double Vw = I.Vw;
      if (!mir_i || !(local_coord(a.buf[qi.mir], D, xw[0], xw[1], xw[2], 0) < 0.0)) {
        double u[3];
        sym_apply<D>(qi.L, d, u);
        const double q = dot3(d, u);
        for (int c = 0; c < D; ++c) lxi[c] += -Vw * (Fr * q * d[c] * ir + 2.0 * F * u[c]);
      }
      const V4<double> Wv = a.WV[w];
      const double vv[3] = {2.0 * (qi.v[0] - Wv.x), 2.0 * (qi.v[1] - Wv.y), 2.0 * (qi.v[2] - Wv.z)};
      bool ard;
      const double mu = visc_mu(I, qi.mu, qi.mu, false, vv, d, ir, ard);
      const double irg = 1.0 / (r + reg);
      const double rf = r * irg, dfr = Fr * rf + F * reg * irg * irg;
      const double f = F * rf * Vw, sv = dot3(qi.sg, vv), vd = dot3(vv, d);
      for (int c = 0; c < D; ++c) {
        lvi[c] += 2.0 * mu * f * qi.sg[c];
        lxi[c] += mu * sv * Vw * dfr * d[c] * ir;
      }
      if (ard) {
        const double Lm = f * sv * kR;
        for (int c = 0; c < D; ++c) {
          lvi[c] += -2.0 * Lm * d[c] * ir;
          lxi[c] += Lm * (-vv[c] * ir + vd * d[c] * (ir * ir * ir));
        }
      }
    }
    if (mir_i) {
      // images m_k = x_k - 2 s_k n of every particle with s_k >= 0 around the
      // image of x_i (two-cell margin), as the forward sweep found them
      const BufDev &b = a.buf[qi.mir];
      const double nb[3] = {b.frame[0], b.frame[1], b.frame[2]};
      const double si = local_coord(b, D, qi.x[0], qi.x[1], qi.x[2], 0);
      const double q0 = qi.x[0] - 2.0 * si * nb[0], q1 = qi.x[1] - 2.0 * si * nb[1];
      const double q2 = D == 3 ? qi.x[2] - 2.0 * si * nb[2] : 0.0;
      const int qx = cell_coord(I, q0, 0), qy = cell_coord(I, q1, 1), qz = D == 3 ? cell_coord(I, q2, 2) : 0;
      for (int set = 0; set < 2; ++set) {
        visit_cells<D, PER>(I, qx, qy, qz, 2, set == 0 ? a.off : a.woff, [&](uint32_t jb, uint32_t je) {
          for (uint32_t k = jb; k < je; ++k) {
            double xk[3];
            double Vk;
            if (set == 0) {
              const ARec qk = get_a<D>(a.ra, (int)k);
              for (int c = 0; c < 3; ++c) xk[c] = qk.x[c];
              Vk = qk.V;
            } else {
              xk[0] = a.wx[0][k];
              xk[1] = a.wx[1][k];
              xk[2] = a.wx[2][k];
              Vk = I.Vw;
            }
            const double sk = local_coord(b, D, xk[0], xk[1], xk[2], 0);
            if (sk < 0.0) continue;
            double dd[3] = {0, 0, 0}, rr = 0.0;
            for (int c = 0; c < D; ++c) {
              dd[c] = qi.x[c] - (xk[c] - 2.0 * sk * nb[c]);
              rr += dd[c] * dd[c];
            }
            if (!(rr > 0.0 && rr < g.cut2)) continue;
            const double ir = rsqrt(rr), r = rr * ir;
            double F, Fr;
            kernel_FF(g, r, F, Fr);
            double u[3];
            sym_apply<D>(qi.L, dd, u);
            const double q = dot3(dd, u);
            double gd[3] = {0, 0, 0};
            for (int c = 0; c < D; ++c) {
              gd[c] = -Vk * (Fr * q * dd[c] * ir + 2.0 * F * u[c]);
              lxi[c] += gd[c];
            }
            if (set == 0) {
              double ng = 0.0;
              for (int c = 0; c < D; ++c) ng += nb[c] * gd[c];
              for (int c = 0; c < D; ++c) atomicAdd(&a.lxs[c][k], -(gd[c] - 2.0 * nb[c] * ng));
              atomicAdd(&a.lrhos[k], (-F * q) * (-Vk / a.T.rho0[k]));
            }
          }
        });
      }
    }
    for (int c = 0; c < D; ++c) {
      a.lv[c][i] += lvi[c];
      a.lxg[c][i] += lxi[c];
    }
    a.lrho[i] += -(qi.V / a.T.rho0[i]) * lVi;
  }
}

// ------------------------------------------------------------------------
// reverse of the cell sort: adjoint in the pending order of the step
// ------------------------------------------------------------------------
__global__ void k_adj_perm_rev(AdjArgs a) {
  const int n = a.cnt->n_live;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int s = (int)a.T.perm[t];
    for (int c = 0; c < 3; ++c) {
      a.out[c][s] = a.lx[c][t] + a.lxg[c][t] + a.lxs[c][t];
      a.out[3 + c][s] = a.lv[c][t];
    }
    a.out[6][s] = a.lrho[t] + a.lrhos[t];
    a.out[7][s] = a.ldrho[t];
  }
}

// ------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------
static int grid_of(int max_n, int block) {
  int g = (max_n + block - 1) / block;
  return g < 1 ? 1 : (g > 65535 ? 65535 : g);
}

void launch_adj_tape_start(const AdjArgs &a, int max_n, cudaStream_t st) {
  k_adj_tape_start<<<grid_of(max_n, 256), 256, 0, st>>>(a);
}
void launch_adj_tape_sub(const AdjArgs &a, int sub, int max_n, cudaStream_t st) {
  k_adj_tape_sub<<<grid_of(max_n, 256), 256, 0, st>>>(a, sub);
}
void launch_adj_tape_drho(const AdjArgs &a, int sub, int max_n, cudaStream_t st) {
  k_adj_tape_drho<<<grid_of(max_n, 256), 256, 0, st>>>(a, sub);
}
void launch_adj_region(const AdjArgs &a, uint8_t *region, const int32_t *obj_buf_mask, int max_n,
                       cudaStream_t st) {
  k_adj_region<<<grid_of(max_n, 256), 256, 0, st>>>(a, region, obj_buf_mask);
}
void launch_adj_objective(const AdjArgs &a, int seed, int max_n, cudaStream_t st) {
  k_adj_objective<<<grid_of(max_n, 256), 256, 0, st>>>(a, seed);
}
void launch_adj_buffer_rev(const AdjArgs &a, int max_n, cudaStream_t st) {
  k_adj_buffer_rev<<<grid_of(max_n, 256), 256, 0, st>>>(a);
}

template <int D, bool PER>
static void substep_rev(const AdjArgs &a, int s, int max_n, cudaStream_t st) {
  const int g = grid_of(max_n, kBlock);
  k_adj_bc_density<D><<<g, kBlock, 0, st>>>(a, s);
  k_adj_cont<D, PER><<<g, kBlock, 0, st>>>(a, s);
  k_adj_mom_rec<D><<<g, kBlock, 0, st>>>(a, s);
  k_adj_mom_seed<D><<<g, kBlock, 0, st>>>(a, s);
  k_adj_mom<D, PER><<<g, kBlock, 0, st>>>(a, s);
  k_adj_half1<<<g, kBlock, 0, st>>>(a, s);
}

void launch_adj_substep_rev(const AdjArgs &a, int dim, int any_periodic, int sub, int max_n, cudaStream_t st) {
  if (dim == 2)
    any_periodic ? substep_rev<2, true>(a, sub, max_n, st) : substep_rev<2, false>(a, sub, max_n, st);
  else
    any_periodic ? substep_rev<3, true>(a, sub, max_n, st) : substep_rev<3, false>(a, sub, max_n, st);
}

void launch_adj_adv_rev(const AdjArgs &a, int dim, int any_periodic, int max_n, cudaStream_t st) {
  const int g = grid_of(max_n, kBlock);
  if (dim == 2) {
    k_adj_adv_seed<2><<<g, kBlock, 0, st>>>(a);
    if (any_periodic)
      k_adj_adv<2, true><<<g, kBlock, 0, st>>>(a);
    else
      k_adj_adv<2, false><<<g, kBlock, 0, st>>>(a);
  } else {
    k_adj_adv_seed<3><<<g, kBlock, 0, st>>>(a);
    if (any_periodic)
      k_adj_adv<3, true><<<g, kBlock, 0, st>>>(a);
    else
      k_adj_adv<3, false><<<g, kBlock, 0, st>>>(a);
  }
}

void launch_adj_perm_rev(const AdjArgs &a, int max_n, cudaStream_t st) {
  k_adj_perm_rev<<<grid_of(max_n, 256), 256, 0, st>>>(a);
}

}  // namespace sphk
