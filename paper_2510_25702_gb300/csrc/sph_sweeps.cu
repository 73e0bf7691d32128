// sph_sweeps.cu -- the pair sweeps of one advection step.
//
//  k_list (first, once per advection step): the neighbour list of the frozen
//         configuration -- the dual-criteria scheme of Sec. 2.3 keeps the
//         configuration of an advection step -- read by all the sweeps.
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
// Work mapping: one thread per particle in cell order, grid-stride over a
// grid sized to the resident blocks of the GPU (a sub-step that no instance
// takes costs one pass over ~1k blocks).  The list builder visits the 3^d
// cells around a particle's cell; because particles are sorted by cell key
// the cells of one row form one contiguous index range; candidates are
// fetched four at a time and tested against the cut-off.  The sweeps walk the
// list (entry k of particle i at k * stride + i, so a warp's reads of one k
// are coalesced) and gather one record per neighbour: everything a sweep
// needs of neighbour j, written by the kernel before it (32 B in 2D FP32,
// one sector).
//
// Precision: R is the sweep precision.  Pair sums, forces, k-epsilon sources,
// volumes and pressures are evaluated in R; FP64 is used to update the FP64
// master state (x, v, rho, k, eps) and to invert B.  On GB300 FP64 issues at a
// small fraction of the FP32 rate, so with R = float the FP64 work per
// particle is a few adds and conversions, and divisions are the fast
// reciprocal form.  With R = double every operation is FP64 and IEEE.
#include <map>
#include <mutex>
#include <tuple>

#include "sph_pair.cuh"

namespace sphk {

// =========================================================================
// neighbour list of the frozen configuration (once per advection step)
// =========================================================================
template <typename R, int D, bool PER>
__device__ __forceinline__ int list_one(const SweepArgs &a, const Packs<R> &pk, const int i) {
  constexpr int RA = RecLayout<D>::adv;
  const InstDev &I = a.inst[a.m.inst[i]];
  const Geo<R> g = make_geo<R, D>(I);
  int cx, cy, cz;
  decode_cell(I, a.keys[i], cx, cy, cz);
  // candidate positions: the FP32 form tests absolute FP32 coordinates (its
  // records hold fixed point), the FP64 form its records' FP64 ones
  const bool f32 = sizeof(R) == 4;
  const V4<R> Pi = f32 ? pk.lpos[i] : pk.adv[RA * (size_t)i];
  uint32_t *__restrict__ out = list_of(a.nl, i);
  const int K = a.nl.kmax;
  int nr = 0, nw = 0;
  // offset of the particle from its cell's low corner (FP32, clamped to the
  // cell), for dropping cells out of reach
  const float cs = (float)I.cs;
  float o[3] = {0.0f, 0.0f, 0.0f};
  {
    const float p[3] = {(float)Pi.x, (float)Pi.y, (float)Pi.z};
    const int cc[3] = {cx, cy, cz};
#pragma unroll
    for (int q = 0; q < D; ++q) o[q] = fminf(fmaxf(p[q] - (I.lo_f[q] + (float)cc[q] * cs), 0.0f), cs);
  }
  // FP32: the band around the cut-off that the FP64 test decides
  R lo = g.cut2, hi = g.cut2;
  if (sizeof(R) == 4) {
    float M = fmaxf(fabsf((float)Pi.x), fabsf((float)Pi.y)), Lp = 0.0f;
    if (D == 3) M = fmaxf(M, fabsf((float)Pi.z));
    if (PER)
      for (int q = 0; q < D; ++q)
        if (g.per[q]) Lp = fmaxf(Lp, (float)g.L[q]);
    const float band = cutoff_band(D, cs, M, Lp);
    lo = (R)((float)g.cut2 - band);
    hi = (R)((float)g.cut2 + band);
  }
  // entries are collected four at a time and stored as one 16-byte chunk
  uint4 buf = make_uint4(0u, 0u, 0u, 0u);
  uint4 *__restrict__ out4 = reinterpret_cast<uint4 *>(out);
  // real neighbours, then wall dummies; 0 < |r|^2 < (2h)^2 excludes i itself
  for (int set = 0; set < 2; ++set) {
    const uint32_t *offs = set == 0 ? a.off : a.woff;
    if (!PER && set == 1) {
      // the cells of the block lie between the keys of its two extreme
      // corners: equal offsets there, no dummy in any of them
      const int x0 = max(cx - 1, 0), y0 = max(cy - 1, 0), z0 = D == 3 ? max(cz - 1, 0) : 0;
      const int x1 = min(cx + 1, I.nc[0] - 1), y1 = min(cy + 1, I.nc[1] - 1);
      const int z1 = D == 3 ? min(cz + 1, I.nc[2] - 1) : 0;
      const uint32_t k0 = I.cell_base + ((uint32_t)z0 * (uint32_t)I.nc[1] + (uint32_t)y0) * (uint32_t)I.nc[0] + (uint32_t)x0;
      const uint32_t k1 = I.cell_base + ((uint32_t)z1 * (uint32_t)I.nc[1] + (uint32_t)y1) * (uint32_t)I.nc[0] + (uint32_t)x1;
      if (offs[k0] == offs[k1 + 1]) break;
    }
    const V4<R> *recs = set == 0 ? (f32 ? pk.lpos : pk.adv) : (f32 ? pk.WPf : pk.WP);
    const int stride = (set == 0 && !f32) ? RA : 1;
    // the definition in FP64 on the masters (rare: candidates in the band)
    auto exact = [&](uint32_t j) -> bool {
      if (set == 0 && j == (uint32_t)i) return false;
      const double xi[3] = {a.m.x[0][i], a.m.x[1][i], D == 3 ? a.m.x[2][i] : 0.0};
      return exact_pair_test(I, D, xi, set == 0 ? a.m.x : a.wx, j);
    };
    auto scan = [&](uint32_t jb, uint32_t je) {
      scan_range<R, D, PER>(g, Pi, recs, stride, jb, je, lo, hi, [&](uint32_t j) {
        const int k = nr + nw;
        buf.x = buf.y;
        buf.y = buf.z;
        buf.z = buf.w;
        buf.w = j;
        if ((k & 3) == 3 && k < K) out4[(size_t)(k >> 2) * kListTile] = buf;
        if (set == 0)
          ++nr;
        else
          ++nw;
      }, exact);
    };
    if (PER)
      visit_cells<D, PER>(I, cx, cy, cz, 1, offs, scan);
    else
      visit_cells_trimmed<D>(I, cx, cy, cz, o, cs, offs, scan);
  }
  {
    // the last, partly filled chunk: its r entries are the newest in buf
    const int tot = nr + nw, r = tot & 3;
    if (r && tot <= K) {
      uint4 c = buf;
      if (r == 1) c = make_uint4(buf.w, 0u, 0u, 0u);
      if (r == 2) c = make_uint4(buf.z, buf.w, 0u, 0u);
      if (r == 3) c = make_uint4(buf.y, buf.z, buf.w, 0u);
      out4[(size_t)(tot >> 2) * kListTile] = c;
    }
  }
  if (nr + nw > K) {  // more neighbours than the list holds
    set_status(a.status, SPH_ERR_CAPACITY);
    nr = nr < K ? nr : K;
    nw = K - nr < nw ? K - nr : nw;
  }
  a.nl.n_real[i] = (uint16_t)nr;
  a.nl.n_wall[i] = (uint16_t)nw;
  return nr + nw;
}

// =========================================================================
// advection sweep: B (+ mirror), viscous acceleration, k-epsilon, half 1
// =========================================================================
// X: some instance of the context takes the transport-velocity shift or the
// density reinitialisation (their sums cost the pair loop a few percent, so
// contexts without them run a form that leaves them out)
template <typename R, int D, bool PER, bool X>
__device__ __forceinline__ void adv_one(const SweepArgs &a, const Packs<R> &pk, const int i) {
  constexpr int RA = RecLayout<D>::adv;
  const Masters &m = a.m;
  const int ii = m.inst[i];
  const InstDev &I = a.inst[ii];
  const Geo<R> g = make_geo<R, D>(I);
  const uint32_t *__restrict__ Lst = list_of(a.nl, i);
  const int nr = a.nl.n_real[i], nw = a.nl.n_wall[i];
  const bool rans = I.rans != 0;
  // own record: 2D (x y V vx)(vy k eps nut), 3D (x y z V)(vx vy vz k)(eps nut - -)
  const V4<R> A0 = pk.adv[RA * (size_t)i], A1 = pk.adv[RA * (size_t)i + 1];
  V4<R> A2 = A1;
  if (D == 3 && rans) A2 = pk.adv_b[i];
  const R vi[3] = {D == 2 ? A0.w : A1.x, D == 2 ? A1.x : A1.y, D == 2 ? (R)0 : A1.z};
  const SweepConst<R> &kc = sweep_const<R>(I);
  const R rho0 = kc.rho0, nu_l = kc.nu_l, c0 = kc.c0, eta = kc.eta, muRk = kc.muR_k;
  R k_i = (R)0, e_i = (R)0, nut_i = (R)0;
  if (rans) {
    k_i = D == 2 ? A1.y : A1.w;
    e_i = D == 2 ? A1.z : A2.x;
    nut_i = D == 2 ? A1.w : A2.y;
  }
  const R mu_i = rho0 * (nu_l + nut_i);
  const R Dk_i = nu_l + nut_i * (R)(1.0 / kSigK), De_i = nu_l + nut_i * (R)(1.0 / kSigE);
  // pair-invariant factors: the harmonic mean of mu_i, mu_j is
  // 2 rho0 nu_i nu_j / (nu_i + nu_j); mu_R = min(muRk eta max(v_e, 0), muRk c0);
  // the k and eps diffusion sums carry 2 rho0 D_i outside
  const R nu_i = nu_l + nut_i, mu2_i = (R)2 * mu_i;
  const R muR_eta = muRk * eta, muR_c0 = muRk * c0;

  const int lab = m.label[i];
  const BufDev *mb = (lab > 0 && lab <= I.nbuf) ? &a.buf[I.buf0 + lab - 1] : nullptr;
  // pressure-buffer particle: the mirror support completes its A (cases 3
  // and 4 of the open-boundary ablation), and its neighbours take B^ = B_i
  // (every case with the condition B_k = B_i)
  const bool pbuf = mb && mb->type == SPH_BUF_PRESSURE;
  const bool mirror = pbuf && (I.obc == SPH_OBC_IMPROVED || I.obc == SPH_OBC_VIPO_RKGC_MIRROR);
  const bool own_B = pbuf && I.obc != SPH_OBC_VIPO && I.obc != SPH_OBC_VIPO_RKGC;
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
  // transport-velocity shift: sum_j V_j grad_i W_ij (fluid particles, and
  // pressure-buffer particles when the instance asks for it); density
  // reinitialisation: sum_j W_ij / alpha_d = sum_j w^4 (5 - 4 w), w = 1 - q/2
  // (fluid particles)
  const bool tvf_b = X && I.tvf && I.tvf_pbuf && pbuf;
  const bool tvf = (X && I.tvf && lab == 0) || tvf_b, dsum = X && I.density_sum && lab == 0;
  R gsum[3] = {0, 0, 0};
  R sig = 0;

  // step-wise wall function (RANS, a fluid particle less than dp from the
  // wall surface): wall distance, normal and nearest dummy from a first pass
  // over the wall neighbours, then the friction velocity of the two-layer
  // wall law in FP64; its wall pairs then carry nu_w = u_tau^2 y / u_t
  bool wf = false, wf_log = false;
  double wf_y = 0.0, wf_utau = 0.0;
  R mu_wall = mu_i;
  if (X && rans && I.wall_fn && lab == 0 && nw > 0) {
    R rmin = (R)0, ns[3] = {0, 0, 0};
    uint32_t wmin = 0;
    for (int kk = nr; kk < nr + nw; ++kk) {
      const uint32_t w = list_at(Lst, kk);
      const V4<R> Wp = pk.WP[w];
      R d[3];
      const R rr = pair_vec<R, D, PER>(g, A0, Wp, d);
      R r;
      Ex<R>::len(rr, r);
      if (kk == nr || r < rmin) {
        rmin = r;
        wmin = w;
      }
      const R FV = kernel_F(g, r) * Wp.w;
#pragma unroll
      for (int c = 0; c < D; ++c) ns[c] -= FV * d[c];
    }
    const double y = from_R<R>(rmin) - 0.5 * I.dp;
    double nn = 0.0;
#pragma unroll
    for (int c = 0; c < D; ++c) nn += from_R<R>(ns[c]) * from_R<R>(ns[c]);
    nn = sqrt(nn);
    if (y > 0.0 && y < I.dp && nn > 0.0) {
      const V4<R> Wv = pk.WV[wmin];
      const double wv[3] = {from_R<R>(Wv.x), from_R<R>(Wv.y), from_R<R>(Wv.z)};
      double vr[3] = {0.0, 0.0, 0.0}, vn = 0.0, ut2 = 0.0;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        vr[c] = from_R<R>(vi[c]) - wv[c];
        vn += vr[c] * (from_R<R>(ns[c]) / nn);
      }
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const double t = vr[c] - vn * (from_R<R>(ns[c]) / nn);
        ut2 += t * t;
      }
      const double ut = sqrt(ut2);
      wf = true;
      wf_y = y;
      wf_utau = wall_utau(ut, y, I.nu_l, wf_log);
      if (ut > 0.0) mu_wall = to_R<R>(I.rho0 * (wf_utau * wf_utau * y / ut));
    }
  }

  // real neighbours
  for (int k0 = 0; k0 < nr; k0 += 4) {
    // four list entries per load, their four records gathered together
    const uint4 q4 = list_chunk(Lst, k0 >> 2);
    const uint32_t j4[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (k0 + c >= nr) break;
      const uint32_t j = j4[c];
      V4<R> B0, B1;
      ld_rec2<R>(pk.adv + RA * (size_t)j, B0, B1);
      V4<R> B2 = B1;
      if (D == 3 && rans) B2 = pk.adv_b[j];
      R d[3];
      const R rr = pair_vec<R, D, PER>(g, A0, B0, d);
      R r;
      Ex<R>::len(rr, r);
      const R F = kernel_F(g, r);  // dW/dr / r
      const R V = vol<R, D>(B0);
      if (!mirror || !(local0<R, D>(mo, mn, rec_abs<R>(I, B0.x, 0), rec_abs<R>(I, B0.y, 1), rec_abs<R>(I, B0.z, 2)) < (R)0))
        sym_add_outer<R, D>(A, d, -F * V);
      if (tvf) {
        const R FV = F * V;
#pragma unroll
        for (int c = 0; c < D; ++c) gsum[c] += FV * d[c];
      }
      if (dsum) sig += kernel_u(g, r);
      const R vj[3] = {D == 2 ? B0.w : B1.x, D == 2 ? B1.x : B1.y, D == 2 ? (R)0 : B1.z};
      const R vij[3] = {vi[0] - vj[0], vi[1] - vj[1], vi[2] - vj[2]};
      const R f = Ex<R>::div(F * r, r + g.reg) * V;  // dW/dr / (r + 0.01h) V
      R mu_ad = mu_i;                                // laminar: harmonic mean of equal values
      if (rans) {
        const R k_j = D == 2 ? B1.y : B1.w, e_j = D == 2 ? B1.z : B2.x, nut_j = D == 2 ? B1.w : B2.y;
        const R nu_j = nu_l + nut_j;
        const R mut = Ex<R>::div(mu2_i * nu_j, nu_i + nu_j);
        R muR = -(vij[0] * d[0] + vij[1] * d[1] + vij[2] * d[2]) * Ex<R>::inv_len(rr, r) * muR_eta;
        muR = muR > (R)0 ? muR : (R)0;
        muR = muR < muR_c0 ? muR : muR_c0;
        mu_ad = mut > muR ? mut : muR;
        const R FV = F * V;
  #pragma unroll
        for (int p = 0; p < D; ++p)
  #pragma unroll
          for (int q = 0; q < D; ++q) G[p][q] += vij[p] * d[q] * FV;
        const R Dk_j = nu_l + nut_j * (R)(1.0 / kSigK), De_j = nu_l + nut_j * (R)(1.0 / kSigE);
        dk += Ex<R>::div(Dk_j, Dk_i + Dk_j) * (k_i - k_j) * f;
        de += Ex<R>::div(De_j, De_i + De_j) * (e_i - e_j) * f;
      }
  #pragma unroll
      for (int c = 0; c < D; ++c) sv[c] += mu_ad * f * vij[c];
    }
  }

  // wall dummies
  for (int kk = nr; kk < nr + nw; ++kk) {
    const uint32_t w = list_at(Lst, kk);
    const V4<R> Wp = pk.WP[w];
    R d[3];
    const R rr = pair_vec<R, D, PER>(g, A0, Wp, d);
    R r;
    Ex<R>::len(rr, r);
    const R F = kernel_F(g, r);
    const R V = Wp.w;
    if (!mirror || !(local0<R, D>(mo, mn, rec_abs<R>(I, Wp.x, 0), rec_abs<R>(I, Wp.y, 1), rec_abs<R>(I, Wp.z, 2)) < (R)0))
      sym_add_outer<R, D>(A, d, -F * V);
    if (tvf) {
      const R FV = F * V;
#pragma unroll
      for (int c = 0; c < D; ++c) gsum[c] += FV * d[c];
    }
    if (dsum) sig += kernel_u(g, r);
    const V4<R> Wv = pk.WV[w];
    // no-slip: the dummy carries 2 v_wall - v_i
    const R vij[3] = {(R)2 * (vi[0] - Wv.x), (R)2 * (vi[1] - Wv.y), (R)2 * (vi[2] - Wv.z)};
    R mu_ad = mu_wall;
    if (rans) {
      R muR = -(vij[0] * d[0] + vij[1] * d[1] + vij[2] * d[2]) * Ex<R>::inv_len(rr, r) * muR_eta;
      muR = muR > (R)0 ? muR : (R)0;
      muR = muR < muR_c0 ? muR : muR_c0;
      mu_ad = mu_wall > muR ? mu_wall : muR;
      const R FV = F * V;
#pragma unroll
      for (int p = 0; p < D; ++p)
#pragma unroll
        for (int q = 0; q < D; ++q) G[p][q] += vij[p] * d[q] * FV;
    }
    const R f = Ex<R>::div(F * r, r + g.reg) * V;
#pragma unroll
    for (int c = 0; c < D; ++c) sv[c] += mu_ad * f * vij[c];
  }

  if (mirror) {
    // images m_j = x_j - 2 x'_0(x_j) n_b of every particle on the fluid side
    // of the open face, searched around the image of x_i (two-cell margin)
    // absolute positions (the FP32 form decodes its fixed-point records)
    const R ax = rec_abs<R>(I, A0.x, 0), ay = rec_abs<R>(I, A0.y, 1), az = D == 3 ? rec_abs<R>(I, A0.z, 2) : (R)0;
    const R si = local0<R, D>(mo, mn, ax, ay, az);
    const double q0 = (double)ax - 2.0 * (double)si * mb->frame[0];
    const double q1 = (double)ay - 2.0 * (double)si * mb->frame[1];
    const double q2 = D == 3 ? (double)az - 2.0 * (double)si * mb->frame[2] : 0.0;
    const int qx = cell_coord(I, q0, 0), qy = cell_coord(I, q1, 1), qz = D == 3 ? cell_coord(I, q2, 2) : 0;
    auto mirror_one = [&](const V4<R> &Pj, R Vj) {
      const R jx = rec_abs<R>(I, Pj.x, 0), jy = rec_abs<R>(I, Pj.y, 1), jz = D == 3 ? rec_abs<R>(I, Pj.z, 2) : (R)0;
      const R sj = local0<R, D>(mo, mn, jx, jy, jz);
      if (sj < (R)0) return;
      const R two_s = Ex<R>::mul((R)2, sj);
      R xj[3] = {jx, jy, jz}, xi[3] = {ax, ay, az};
      R d[3] = {0, 0, 0};
      R dd = 0;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        R img = Ex<R>::sub(xj[c], Ex<R>::mul(two_s, mn[c]));
        d[c] = Ex<R>::sub(xi[c], img);
        dd = (c == 0) ? Ex<R>::mul(d[c], d[c]) : Ex<R>::add(dd, Ex<R>::mul(d[c], d[c]));
      }
      if (!(dd > (R)0 && dd < g.cut2)) return;
      R r;
      Ex<R>::len(dd, r);
      sym_add_outer<R, D>(A, d, -kernel_F(g, r) * Vj);
    };
    for (int set = 0; set < 2; ++set) {
      const uint32_t *offs = set == 0 ? a.off : a.woff;
      const V4<R> *recs = set == 0 ? pk.adv : pk.WP;
      const int stride = set == 0 ? RA : 1;
      visit_cells<D, PER>(I, qx, qy, qz, 2, offs, [&](uint32_t jb, uint32_t je) {
        for (uint32_t j = jb; j < je; ++j) {
          const V4<R> Pj = recs[(size_t)j * stride];
          mirror_one(Pj, set == 0 ? vol<R, D>(Pj) : Pj.w);
        }
      });
    }
  }

  // ---------------- epilogue ----------------
  // B = A^-1.  FP64 where the support is cut (wall dummies in the list,
  // particles in a buffer): there A can be ill-conditioned.  Interior
  // particles of the FP32 form, whose A is close to the full-support
  // lattice value (about 0.97 I), invert in the sweep precision.
  R BR[6] = {(R)0, (R)0, (R)0, (R)0, (R)0, (R)0};
  if (I.obc == SPH_OBC_VIPO) {
    // case 1 of the ablation: no kernel correction
    BR[0] = BR[1] = (R)1;
    if (D == 3) BR[2] = (R)1;
    a.der.B[0][i] = 1.0;
    a.der.B[1][i] = 1.0;
    a.der.B[3][i] = 0.0;
    if (D == 3) {
      a.der.B[2][i] = 1.0;
      a.der.B[4][i] = 0.0;
      a.der.B[5][i] = 0.0;
    }
  } else if (sizeof(R) == 4 && nw == 0 && lab == 0) {
    invert_guarded_fast<R, D>(A, BR);
  } else {
    double Ad[6] = {(double)A[0], (double)A[1], 0.0, (double)A[3], 0.0, 0.0};
    if (D == 3) {
      Ad[2] = (double)A[2];
      Ad[4] = (double)A[4];
      Ad[5] = (double)A[5];
    }
    double Bd[6];
    invert_guarded<D>(Ad, Bd);  // FP64 inversion (one reciprocal)
    for (int c = 0; c < 6; ++c) BR[c] = to_R<R>(Bd[c]);
    if (sizeof(R) == 8) {  // FP64 form: keep every bit of the FP64 inverse
      a.der.B[0][i] = Bd[0];
      a.der.B[1][i] = Bd[1];
      a.der.B[3][i] = Bd[3];
      if (D == 3) {
        a.der.B[2][i] = Bd[2];
        a.der.B[4][i] = Bd[4];
        a.der.B[5][i] = Bd[5];
      }
    }
  }
  if (sizeof(R) == 4 && I.obc != SPH_OBC_VIPO) {
    a.der.B[0][i] = from_R<R>(BR[0]);
    a.der.B[1][i] = from_R<R>(BR[1]);
    a.der.B[3][i] = from_R<R>(BR[3]);
    if (D == 3) {
      a.der.B[2][i] = from_R<R>(BR[2]);
      a.der.B[4][i] = from_R<R>(BR[4]);
      a.der.B[5][i] = from_R<R>(BR[5]);
    }
  }
  const double rho_i = m.rho[i];
  const R inv_rho = Ex<R>::div((R)1, to_R<R>(rho_i));
  R an[3] = {0, 0, 0};
#pragma unroll
  for (int c = 0; c < D; ++c) {
    an[c] = (R)2 * sv[c] * inv_rho;
    a.der.an[c][i] = from_R<R>(an[c]);
  }
  pk.Ap[i] = V4<R>{an[0] + kc.g[0], an[1] + kc.g[1], D == 3 ? an[2] + kc.g[2] : (R)0, (R)0};

  R kw = (R)0;
  if (rans && !I.freeze_turb) {
    // grad v = -(sum v_ij (x) grad W V) B^T, (p, q) = dv_p / dx_q
    const R Bf[3][3] = {{BR[0], BR[3], BR[4]}, {BR[3], BR[1], BR[5]}, {BR[4], BR[5], BR[2]}};
    R tr = 0, prod = 0;
    R gv[3][3];
#pragma unroll
    for (int p = 0; p < D; ++p)
#pragma unroll
      for (int q = 0; q < D; ++q) {
        R s = 0;
#pragma unroll
        for (int c = 0; c < D; ++c) s += G[p][c] * Bf[q][c];
        gv[p][q] = -s;
      }
#pragma unroll
    for (int p = 0; p < D; ++p) {
      tr += gv[p][p];
#pragma unroll
      for (int q = 0; q < D; ++q) prod += (gv[p][q] + gv[q][p]) * gv[p][q];
    }
    const R inv_k = Ex<R>::div((R)1, k_i);
    R Gk = nut_i * prod - (R)(2.0 / 3.0) * k_i * tr;
    // wall function: the log-law production tau_w du/dy = u_tau^3 / (kappa y)
    // (none in the viscous sublayer)
    if (wf) Gk = wf_log ? to_R<R>(wf_utau * wf_utau * wf_utau / (kWfKappa * wf_y)) : (R)0;
    const R dk_all = (R)2 * rho0 * Dk_i * dk, de_all = (R)2 * rho0 * De_i * de;
    const R dkdt = Gk - e_i + (R)2 * dk_all * inv_rho;
    const R dedt = (R)kC1 * e_i * inv_k * Gk - (R)kC2 * e_i * e_i * inv_k + (R)2 * de_all * inv_rho;
    // explicit update over dt_ad in the sweep precision (k, eps are not
    // among the FP64-integrated fields; in the FP64 form this is FP64)
    const R dta = to_R<R>(I.dt_ad);
    R k1r = k_i + dta * dkdt, e1r = e_i + dta * dedt;
    k1r = k1r > (R)kFloor ? k1r : (R)kFloor;
    e1r = e1r > (R)kFloor ? e1r : (R)kFloor;
    if (wf) {
      // the wall value of eps from the updated k
      const double kk = from_R<R>(k1r);
      const double ew = wf_log ? I.wf_cmu34 * (kk * sqrt(kk)) / (kWfKappa * wf_y) : 2.0 * I.nu_l * kk / (wf_y * wf_y);
      e1r = to_R<R>(ew > kFloor ? ew : kFloor);
    }
    m.k[i] = from_R<R>(k1r);
    m.eps[i] = from_R<R>(e1r);
    m.nut[i] = from_R<R>(Ex<R>::div((R)kCmu * k1r * k1r, e1r));
    kw = (R)(2.0 / 3.0) * k1r;
  } else if (rans) {
    kw = (R)(2.0 / 3.0) * k_i;  // turbulence held over a differentiated window
  }
  // first half of sub-step 0 (a8): rho += dt/2 drho; p = c0^2 (rho - rho0);
  // x += dt/2 v.  The pressure master keeps the value of the step's last
  // first half, so only that one is stored.
  // The density reinitialisation and the transport-velocity shift of a fluid
  // particle come before it (the terms above used the volumes from before).
  const double hdt = 0.5 * I.dt;
  const double rho_s = dsum ? I.dsum_k * ((double)1 + from_R<R>(sig)) : rho_i;
  const double rho = rho_s + hdt * m.drho[i];
  const R p = to_R<R>(rho - I.rho0) * sweep_const<R>(I).c0sq;
  m.rho[i] = rho;
  if (I.n_ac == 1) m.p[i] = from_R<R>(p);
  // a pressure-buffer particle takes the shift across its buffer axis only:
  // its support is cut at the open face, so the sum points into the fluid
  double sh[3] = {0.0, 0.0, 0.0};
  if (tvf) {
#pragma unroll
    for (int c = 0; c < D; ++c) sh[c] = from_R<R>(gsum[c]);
    if (tvf_b) {
      double sn = 0.0;
#pragma unroll
      for (int c = 0; c < D; ++c) sn += sh[c] * mb->frame[c];
#pragma unroll
      for (int c = 0; c < D; ++c) sh[c] -= sn * mb->frame[c];
    }
  }
#pragma unroll
  for (int c = 0; c < D; ++c) {
    double xc = m.x[c][i];
    if (tvf) xc = xc + I.tvf_k * sh[c];
    m.x[c][i] = xc + hdt * m.v[c][i];
  }
  // momentum record; pressure-buffer particles are marked so that their
  // neighbours use their own B (the condition B_k = B_i, Sec. 3.3)
  const R V = Ex<R>::div(to_R<R>(m.mass[i]), to_R<R>(rho));
  const R bxx = own_B ? (R)-1 : BR[0];
  if (D == 2) {
    pk.mom[2 * (size_t)i] = V4<R>{A0.x, A0.y, V, p};
    pk.mom[2 * (size_t)i + 1] = V4<R>{bxx, BR[3], BR[1], kw};
  } else {
    pk.mom[2 * (size_t)i] = V4<R>{A0.x, A0.y, A0.z, V};
    pk.mom[2 * (size_t)i + 1] = V4<R>{p, kw, bxx, BR[1]};
    pk.mom_b[i] = V4<R>{BR[2], BR[3], BR[4], BR[5]};
  }
}

// =========================================================================
// momentum sweep (a9)
// =========================================================================
template <typename R, int D, bool PER>
__device__ __forceinline__ void mom_one(const SweepArgs &a, const Packs<R> &pk, const int i) {
  constexpr int RM = RecLayout<D>::mom;
  const Masters &m = a.m;
  const int ii = m.inst[i];
  const InstDev &I = a.inst[ii];
  if (a.sub >= I.n_ac) return;
  const Geo<R> g = make_geo<R, D>(I);
  const uint32_t *__restrict__ Lst = list_of(a.nl, i);
  const int nr = a.nl.n_real[i], nw = a.nl.n_wall[i];
  const bool rans = I.rans != 0;
  const R rho0 = sweep_const<R>(I).rho0, inv_c0sq = sweep_const<R>(I).inv_c0sq;
  const V4<R> M0 = pk.mom[RM * (size_t)i], M1 = pk.mom[RM * (size_t)i + 1];
  V4<R> M2 = M1;
  if (D == 3) M2 = pk.mom_b[i];
  R Bi[6], kw_i, p_i = M0.w;
  if (!mom_B<R, D>(M1, M2, Bi, kw_i, p_i)) {  // pressure-buffer particle: FP64 master B
    for (int c = 0; c < 6; ++c) Bi[c] = (R)a.der.B[c][i];
    if (D == 2) Bi[2] = Bi[4] = Bi[5] = (R)0;
  }
  const R pe_i = rans ? p_eff(p_i, kw_i, rho0, inv_c0sq) : p_i;

  R S1[3] = {0, 0, 0}, Cb[3] = {0, 0, 0}, S2[3] = {0, 0, 0}, Ct[3] = {0, 0, 0};
  // four list entries per load, their four records gathered together; the
  // next chunk is requested before this one is processed
  uint4 nxt = nr > 0 ? list_chunk(Lst, 0) : make_uint4(0u, 0u, 0u, 0u);
  for (int k0 = 0; k0 < nr; k0 += 4) {
    const uint4 q4 = nxt;
    if (k0 + 4 < nr) nxt = list_chunk(Lst, (k0 >> 2) + 1);
    const uint32_t j4[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (k0 + c >= nr) break;
      const uint32_t j = j4[c];
      V4<R> N0, N1, N2;
      ld_rec2<R>(pk.mom + RM * (size_t)j, N0, N1);
      N2 = D == 3 ? pk.mom_b[j] : N1;
      R d[3];
      const R rr = pair_vec<R, D, PER>(g, M0, N0, d);
      R r;
      Ex<R>::len(rr, r);
      const R FV = kernel_F(g, r) * vol<R, D>(N0);       // V_j dW/dr / r
      const R gw[3] = {FV * d[0], FV * d[1], FV * d[2]};  // V_j grad_i W_ij
      R Bj[6], kw_j, p_j = N0.w;
      const bool own = mom_B<R, D>(N1, N2, Bj, kw_j, p_j);
      const R pe_j = rans ? p_eff(p_j, kw_j, rho0, inv_c0sq) : p_j;
      if (own) {
        R bg[3];
        sym_matvec<R, D>(Bj, gw, bg);
  #pragma unroll
        for (int c = 0; c < D; ++c) S1[c] += bg[c];
      } else {
  #pragma unroll
        for (int c = 0; c < D; ++c) Cb[c] += gw[c];  // pressure-buffer neighbour: B^_j = B_i
      }
  #pragma unroll
      for (int c = 0; c < D; ++c) {
        S2[c] += pe_j * gw[c];
        Ct[c] += gw[c];
      }
    }
  }
  for (int kk = nr; kk < nr + nw; ++kk) {
    const uint32_t w = list_at(Lst, kk);
    const V4<R> Wp = pk.WP[w];
    R d[3];
    const R rr = pair_vec<R, D, PER>(g, M0, Wp, d);
    R r;
    Ex<R>::len(rr, r);
    const R FV = kernel_F(g, r) * Wp.w;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const R gv = FV * d[c];
      Cb[c] += gv;         // wall dummy: B^_j = B_i
      S2[c] += pe_i * gv;  // wall dummy: p_j = p_i
      Ct[c] += gv;
    }
  }
  // a = -(1/rho_i) (p_i (S1 + B_i Cb) + B_i S2) [+ (2 p_ob / rho_i) B_i Ct]
  const double rho_i = m.rho[i];
  const R inv_rho = Ex<R>::div((R)1, to_R<R>(rho_i));
  R bcb[3], bs2[3];
  sym_matvec<R, D>(Bi, Cb, bcb);
  sym_matvec<R, D>(Bi, S2, bs2);
  R acc[3] = {0, 0, 0};
#pragma unroll
  for (int c = 0; c < D; ++c) acc[c] = -(pe_i * (S1[c] + bcb[c]) + bs2[c]) * inv_rho;
  const int lab = m.label[i];
  if (lab > 0 && lab <= I.nbuf) {
    const BufDev &b = a.buf[I.buf0 + lab - 1];
    if (b.type == SPH_BUF_PRESSURE) {
      R pob = (R)b.p_ob;
      if (rans) pob += (R)(2.0 / 3.0) * (R)rho_i * (R)m.k[i];
      // compensation with B_i (final Eq. of Sec. 3.3), or without it as in
      // the original VIPO (ablation cases 1-3)
      R bct[3] = {Ct[0], Ct[1], Ct[2]};
      if (I.obc == SPH_OBC_IMPROVED || I.obc == SPH_OBC_MINIMAL_MIRROR) sym_matvec<R, D>(Bi, Ct, bct);
#pragma unroll
      for (int c = 0; c < D; ++c) acc[c] += (R)2 * pob * inv_rho * bct[c];
    }
  }
  if (a.tape_S) {
    // the four sums for the reverse pass of a differentiated window
    double *t = a.tape_S + (size_t)a.sub * 12 * a.nl.stride;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      t[(size_t)(0 + c) * a.nl.stride + i] = (double)S1[c];
      t[(size_t)(3 + c) * a.nl.stride + i] = (double)Cb[c];
      t[(size_t)(6 + c) * a.nl.stride + i] = (double)S2[c];
      t[(size_t)(9 + c) * a.nl.stride + i] = (double)Ct[c];
    }
  }
  // FP64 kick and half drift
  const V4<R> ap = pk.Ap[i];
  const R apr[3] = {ap.x, ap.y, ap.z};
  const double dt = I.dt, hdt = 0.5 * I.dt;
  R vo[3] = {(R)0, (R)0, (R)0};
#pragma unroll
  for (int c = 0; c < D; ++c) {
    const double v = m.v[c][i] + dt * from_R<R>(acc[c] + apr[c]);
    m.v[c][i] = v;
    m.x[c][i] = m.x[c][i] + hdt * v;
    vo[c] = to_R<R>(v);
  }
  // continuity record: 2D (x y V p)(vx vy - -), 3D (x y z V)(p vx vy vz)
  pk.cont[2 * (size_t)i] = M0;
  if (D == 2)
    pk.cont[2 * (size_t)i + 1] = V4<R>{vo[0], vo[1], (R)0, (R)0};
  else
    pk.cont[2 * (size_t)i + 1] = V4<R>{p_i, vo[0], vo[1], vo[2]};
}

// =========================================================================
// continuity sweep (a10) + density update + boundary values (a11) + next
// half step (a8)
// =========================================================================
template <typename R, int D, bool PER>
__device__ __forceinline__ void cont_one(const SweepArgs &a, const Packs<R> &pk, const int i) {
  constexpr int RM = RecLayout<D>::mom;
  const Masters &m = a.m;
  const int ii = m.inst[i];
  const InstDev &I = a.inst[ii];
  if (a.sub >= I.n_ac) return;
  const Geo<R> g = make_geo<R, D>(I);
  const uint32_t *__restrict__ Lst = list_of(a.nl, i);
  const int nr = a.nl.n_real[i], nw = a.nl.n_wall[i];
  const V4<R> C0 = pk.cont[2 * (size_t)i], C1 = pk.cont[2 * (size_t)i + 1];
  const R vi[3] = {D == 2 ? C1.x : C1.y, D == 2 ? C1.y : C1.z, D == 2 ? (R)0 : C1.w};
  const R p_i = D == 2 ? C0.w : C1.x;
  const R inv_rc = sweep_const<R>(I).inv_rc0;
  // drho_i / rho_i = sum_j [v_ij . r_ij / r + (p_i - p_j) / (rho0 c0)] dW/dr V_j
  R sum = 0;
  // four list entries per load, their four records gathered together; the
  // next chunk is requested before this one is processed
  uint4 nxt = nr > 0 ? list_chunk(Lst, 0) : make_uint4(0u, 0u, 0u, 0u);
  for (int k0 = 0; k0 < nr; k0 += 4) {
    const uint4 q4 = nxt;
    if (k0 + 4 < nr) nxt = list_chunk(Lst, (k0 >> 2) + 1);
    const uint32_t j4[4] = {q4.x, q4.y, q4.z, q4.w};
    // all four gathers issued before any is used; entries past the list's
    // end re-read entry 0 and add nothing
    V4<R> N0[4], N1[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) ld_rec2<R>(pk.cont + 2 * (size_t)(k0 + c < nr ? j4[c] : j4[0]), N0[c], N1[c]);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      R d[3];
      const R rr = pair_vec<R, D, PER>(g, C0, N0[c], d);
      R r;
      Ex<R>::len(rr, r);
      const R FV = kernel_F(g, r) * vol<R, D>(N0[c]);
      const R vj[3] = {D == 2 ? N1[c].x : N1[c].y, D == 2 ? N1[c].y : N1[c].z, D == 2 ? (R)0 : N1[c].w};
      const R p_j = D == 2 ? N0[c].w : N1[c].x;
      const R vd = (vi[0] - vj[0]) * d[0] + (vi[1] - vj[1]) * d[1] + (vi[2] - vj[2]) * d[2];
      if (k0 + c < nr) sum += (vd + (p_i - p_j) * inv_rc * r) * FV;
    }
  }
  for (int kk = nr; kk < nr + nw; ++kk) {
    const uint32_t w = list_at(Lst, kk);
    const V4<R> Wp = pk.WP[w];
    R d[3];
    const R rr = pair_vec<R, D, PER>(g, C0, Wp, d);
    R r;
    Ex<R>::len(rr, r);
    const V4<R> Wv = pk.WV[w];
    // dummy velocity 2 v_wall - v_i, dummy pressure p_i
    const R vd = (R)2 * ((vi[0] - Wv.x) * d[0] + (vi[1] - Wv.y) * d[1] + (vi[2] - Wv.z) * d[2]);
    sum += vd * kernel_F(g, r) * Wp.w;
  }
  const double hdt = 0.5 * I.dt;
  const double rho_i = m.rho[i];
  const double drho = rho_i * from_R<R>(sum);
  m.drho[i] = drho;
  double rho = rho_i + hdt * drho;
  m.rho[i] = rho;
  const int lab = m.label[i];
  if (a.flag && a.sub + 1 == I.n_ac) {
    // the step's last sub-step of this instance: positions are final, so
    // the buffer-update flag is taken here (as the flags kernel would)
    uint8_t f = kKeep;
    if (lab > 0 && lab <= I.nbuf) {
      f = buffer_flag(a.buf[I.buf0 + lab - 1], I.dim, m.x[0][i], m.x[1][i], m.x[2][i]);
      if (f == kInject) {
        atomicAdd(&a.inst_spawn[ii], 1);
        atomicAdd(&a.block_cnt[i / kBlock], 1);
      }
    }
    a.flag[i] = f;
  }
  bool kw_reset = false;
  R kw_bc = (R)0;
  if (lab > 0 && lab <= I.nbuf) {
    const BufDev &b = a.buf[I.buf0 + lab - 1];
    apply_bc(I, b, m, i, a.cnt->step, (uint32_t)a.sub);
    rho = m.rho[i];
    if (I.rans && !I.freeze_turb && b.turb == SPH_TURB_FREESTREAM) {
      kw_reset = true;
      kw_bc = (R)((2.0 / 3.0) * b.k_in);
    }
  }
  double v[3] = {m.v[0][i], m.v[1][i], D == 3 ? m.v[2][i] : 0.0};
  // non-finite test on the exponent bits (integer pipe)
  auto nonfinite = [](double x) { return (__double2hiint(x) & 0x7ff00000) == 0x7ff00000; };
  bool bad = nonfinite(rho);
#pragma unroll
  for (int c = 0; c < D; ++c) bad |= nonfinite(v[c]);
  if (bad) set_status(a.status, SPH_ERR_NONFINITE);
  if (a.sub + 1 < I.n_ac) {
    // first half of the next sub-step and the momentum record it reads
    // (B and kw stay from the advection sweep unless a free-stream buffer
    // reset k)
    rho = rho + hdt * drho;
    const R p = to_R<R>(rho - I.rho0) * sweep_const<R>(I).c0sq;
    m.rho[i] = rho;
    if (a.sub + 2 == I.n_ac) m.p[i] = from_R<R>(p);  // the step's last first half
#pragma unroll
    for (int c = 0; c < D; ++c) m.x[c][i] = m.x[c][i] + hdt * v[c];
    const R Vn = Ex<R>::div(to_R<R>(m.mass[i]), to_R<R>(rho));
    if (D == 2) {
      pk.mom[2 * (size_t)i] = V4<R>{C0.x, C0.y, Vn, p};
      if (kw_reset) {
        V4<R> r1 = pk.mom[2 * (size_t)i + 1];
        r1.w = kw_bc;
        pk.mom[2 * (size_t)i + 1] = r1;
      }
    } else {
      pk.mom[RM * (size_t)i] = V4<R>{C0.x, C0.y, C0.z, Vn};
      V4<R> r1 = pk.mom[RM * (size_t)i + 1];
      r1.x = p;
      if (kw_reset) r1.y = kw_bc;
      pk.mom[RM * (size_t)i + 1] = r1;
    }
  }
}

// ------------------------------------------------------------------------
// kernels: grid-stride over the live particles
// ------------------------------------------------------------------------
// resident 256-thread blocks per SM asked of the sweeps (registers =
// 65536 / (256 x blocks)) where that buys warps for their latency-bound
// gathers at few spills (measured): the fused later sub-steps of 2D at 48
// (3D takes them as separate launches).  The FP32 momentum and continuity
// sweeps take register counts of their own (__maxnreg__, below); the FP64
// forms keep the compiler's count.
template <typename R, int D>
constexpr int kContMinBlocks = sizeof(R) == 4 ? 5 : 1;
template <typename R, int D>
constexpr int kSubMinBlocks = sizeof(R) == 4 ? (D == 2 ? 5 : 4) : 1;
// the FP32 list builder at 48 registers as well (few spills)
template <typename R, int D>
constexpr int kListMinBlocks = sizeof(R) == 4 ? 5 : 0;
// the FP32 advection sweep at 64 registers, 8 resident 128-thread blocks:
// in 2D instead of 76 (87.4 against 90.7 us on the 2D channel), in 3D
// instead of 80 (1.71 against 1.77 ms on the 3D mixer, some spills
// included; 97 registers took 2.27 ms)
template <typename R, int D>
constexpr int kAdvMinBlocks = sizeof(R) == 4 ? 4 : 0;

template <typename R, int D, bool PER>
__global__ void __launch_bounds__(kMaxBlock, kListMinBlocks<R, D>) k_list(SweepArgs a, Packs<R> pk) {
  // after a device error (non-finite state, capacity) the state is not
  // advanced further: non-finite positions would all fall into one edge
  // cell and make the candidate scan quadratic
  if (a.cnt->status) return;
  // the time step of every instance (needs the permute's maxima, which are
  // complete when this launch starts; read first by the advection sweep)
  if (a.with_time_step && blockIdx.x == 0)
    for (int ii = threadIdx.x; ii < a.ts.ninst; ii += blockDim.x) time_step_instance(a.ts, ii);
  const int n = a.cnt->n_live;
  // whole blocks iterate together so that every lane of a warp takes part
  // in the reduction of the tile's longest list
  for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const int i = base + threadIdx.x;
    const int cnt = i < n ? list_one<R, D, PER>(a, pk, i) : 0;
    const int rows = __reduce_max_sync(0xffffffffu, cnt);
    if ((threadIdx.x & 31) == 0 && i < n) a.nl.rows[i / kListTile] = (uint16_t)rows;
  }
}

template <typename R, int D, bool PER, bool X>
__global__ void __launch_bounds__(kMaxBlock, kAdvMinBlocks<R, D>) k_adv(SweepArgs a, Packs<R> pk) {
  if (a.cnt->status) return;
  const int n = a.cnt->n_live;
  const int step = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += step) {
    // the next tile's neighbour list on its way to L2 while this one runs
    if ((threadIdx.x & 31) == 0 && i + step < n) prefetch_list_tile(a.nl, i + step);
    adv_one<R, D, PER, X>(a, pk, i);
  }
}

template <typename R, int D, bool PER>
// (the 2D FP32 momentum sweep at 56 registers: 48.7 -> 47.1 us on the 2D
// channel against 48; the other forms keep the compiler's count)
__global__ void __maxnreg__((sizeof(R) == 4 && D == 2) ? 56 : 255) k_mom(SweepArgs a, Packs<R> pk) {
  if (a.sub >= a.cnt->n_ac_all || a.cnt->status) return;  // no instance takes this sub-step
  const int n = a.cnt->n_live;
  const int step = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += step) {
    // the next tile's neighbour list on its way to L2 while this one runs
    if ((threadIdx.x & 31) == 0 && i + step < n) prefetch_list_tile(a.nl, i + step);
    mom_one<R, D, PER>(a, pk, i);
  }
}

template <typename R, int D, bool PER>
__device__ __forceinline__ void cont_sweep(const SweepArgs &a, const Packs<R> &pk) {
  if (a.sub >= a.cnt->n_ac_all || a.cnt->status) return;
  const int n = a.cnt->n_live;
  const int step = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += step) {
    // the next tile's neighbour list on its way to L2 while this one runs
    if ((threadIdx.x & 31) == 0 && i + step < n) prefetch_list_tile(a.nl, i + step);
    cont_one<R, D, PER>(a, pk, i);
  }
}

template <typename R, int D, bool PER>
__global__ void __launch_bounds__(kMaxBlock, kContMinBlocks<R, D>) k_cont(SweepArgs a, Packs<R> pk) {
  cont_sweep<R, D, PER>(a, pk);
}

// the 3D FP32 continuity sweep at 56 registers: no spills (at 48 it spilled)
// and 9 resident 128-thread blocks; 1.08 -> 0.96 ms per sweep on the 3D
// mixer, whose five sub-steps take one each
template <bool PER>
__global__ void __maxnreg__(56) k_cont3f(SweepArgs a, Packs<float> pk) {
  cont_sweep<float, 3, PER>(a, pk);
}
// and the 2D FP32 continuity sweep likewise (no spills; 38.9 -> 37.7 us on
// the 2D channel against 48 registers)
template <bool PER>
__global__ void __maxnreg__(56) k_cont2f(SweepArgs a, Packs<float> pk) {
  cont_sweep<float, 2, PER>(a, pk);
}

// Sub-steps 1 .. n_ac_all - 1 in one cooperative launch (2D; 3D contexts
// launch the momentum and continuity sweeps per sub-step): momentum over all
// particles, grid barrier, continuity, grid barrier, and so on.  When no
// instance takes a second acoustic sub-step -- the usual case -- every block
// ends at once, so the bound on sub-steps costs one empty launch instead of
// two per surplus sub-step.  Every block reads the same n_ac_all (written by
// the time step before this launch), so all of them take the same barriers.
// There is no early exit on the status word here: a block could see a word
// that another block set during the launch and leave the barriers unmatched;
// the work after an error is bounded (fixed lists) and its result unused.
template <typename R, int D, bool PER>
__global__ void __launch_bounds__(kMaxBlock, kSubMinBlocks<R, D>) k_substeps(SweepArgs a, Packs<R> pk, GridBarrier *gb) {
  __shared__ int s_ok;
  const int nac = a.cnt->n_ac_all;
  if (nac <= 1) return;
  const int n = a.cnt->n_live;
  const int step = gridDim.x * blockDim.x;
  uint32_t k = 0;
  for (int s = 1; s < nac; ++s) {
    a.sub = s;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += step) {
      if ((threadIdx.x & 31) == 0 && i + step < n) prefetch_list_tile(a.nl, i + step);
      mom_one<R, D, PER>(a, pk, i);
    }
    if (!grid_sync(gb, ++k, a.status, &s_ok)) break;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += step) {
      if ((threadIdx.x & 31) == 0 && i + step < n) prefetch_list_tile(a.nl, i + step);
      cont_one<R, D, PER>(a, pk, i);
    }
    if (s + 1 < nac && !grid_sync(gb, ++k, a.status, &s_ok)) break;
  }
  grid_leave(gb);
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
  for (int set = 0; set < 2; ++set) {
    auto body = [&](uint32_t jb, uint32_t je) {
      for (uint32_t j = jb; j < je; ++j) {
        if (set == 0) {
          if ((int)j == i) continue;
          const double xj[3] = {m.x[0][j], m.x[1][j], m.x[2][j]};
          if (test(xj)) emit(m.uid[j], 0);
        } else {
          const double xj[3] = {wx[j], wy[j], wz[j]};
          if (test(xj)) emit(wall_index[j], 1);
        }
      }
    };
    if (I.dim == 2)
      visit_cells<2, true>(I, cx, cy, cz, 1, set == 0 ? a.off : a.woff, body);
    else
      visit_cells<3, true>(I, cx, cy, cz, 1, set == 0 ? a.off : a.woff, body);
  }
}

// =========================================================================
// the neighbour list the sweeps walk, as rows (uid_i, uid_j or wall index,
// is_wall, instance), test aid
// =========================================================================
__global__ void __launch_bounds__(kBlock) k_list_rows(SweepArgs a, const uint32_t *__restrict__ wall_index,
                                                      int64_t *out, int64_t max, unsigned long long *counter) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.cnt->n_live) return;
  const uint32_t *L = list_of(a.nl, i);
  const int nr = a.nl.n_real[i], nw = a.nl.n_wall[i];
  for (int k = 0; k < nr + nw; ++k) {
    const uint32_t j = list_at(L, k);
    const bool wall = k >= nr;
    const unsigned long long t = atomicAdd(counter, 1ull);
    if ((int64_t)t < max) {
      out[4 * t + 0] = a.m.uid[i];
      out[4 * t + 1] = wall ? wall_index[j] : a.m.uid[j];
      out[4 * t + 2] = wall ? 1 : 0;
      out[4 * t + 3] = a.m.inst[i];
    }
  }
}

// ------------------------------------------------------------------------
// launch wrappers
// ------------------------------------------------------------------------
// blocks to launch: all resident blocks of the GPU at the chosen block size,
// or fewer when the particles need fewer.  The occupancy query runs once per
// device, kernel and block size (64, 128 or 256 threads).
static int resident_blocks(const void *kernel, int block) {
  static std::mutex mu;
  static std::map<std::tuple<int, const void *, int>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_tuple(dev, kernel, block);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int sms = 1, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0);
  const int r = sms * (per_sm > 0 ? per_sm : 1);
  cache[key] = r;
  return r;
}

template <typename K>
static int resident_grid(K kernel, int block, int max_n) {
  const int per_gpu = resident_blocks((const void *)kernel, block);
  int need = (max_n + block - 1) / block;
  if (need < 1) need = 1;
  return need < per_gpu ? need : per_gpu;
}

// which: 0 advection, 1 momentum, 2 continuity, 3 neighbour list,
// 4 sub-steps after the first (cooperative)
template <typename R, int D, bool PER>
static void launch_sweeps_impl(int which, const SweepArgs &a, Packs<R> &pk, int max_n, cudaStream_t st) {
  const int b = (a.block == 64 || a.block == 256) ? a.block : 128;
  if (which == 4) {
    auto k = k_substeps<R, D, PER>;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)resident_grid(k, b, max_n));
    cfg.blockDim = dim3((unsigned)b);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k, a, pk, a.gbar);
  } else if (which == 3) {
    auto k = k_list<R, D, PER>;
    k<<<resident_grid(k, b, max_n), b, 0, st>>>(a, pk);
  } else if (which == 0) {
    auto k = a.any_extra ? k_adv<R, D, PER, true> : k_adv<R, D, PER, false>;
    k<<<resident_grid(k, b, max_n), b, 0, st>>>(a, pk);
  } else if (which == 1) {
    auto k = k_mom<R, D, PER>;
    k<<<resident_grid(k, b, max_n), b, 0, st>>>(a, pk);
  } else {
    if constexpr (sizeof(R) == 4 && D == 2) {
      auto k = k_cont2f<PER>;
      k<<<resident_grid(k, b, max_n), b, 0, st>>>(a, pk);
    } else if constexpr (sizeof(R) == 4 && D == 3) {
      auto k = k_cont3f<PER>;
      k<<<resident_grid(k, b, max_n), b, 0, st>>>(a, pk);
    } else {
      auto k = k_cont<R, D, PER>;
      k<<<resident_grid(k, b, max_n), b, 0, st>>>(a, pk);
    }
  }
}

template <typename R>
static void launch_sweeps(int which, const SweepArgs &a, void *packs, int dim, int max_n, cudaStream_t st) {
  Packs<R> &pk = *(Packs<R> *)packs;
  if (dim == 2) {
    if (a.any_periodic)
      launch_sweeps_impl<R, 2, true>(which, a, pk, max_n, st);
    else
      launch_sweeps_impl<R, 2, false>(which, a, pk, max_n, st);
  } else {
    if (a.any_periodic)
      launch_sweeps_impl<R, 3, true>(which, a, pk, max_n, st);
    else
      launch_sweeps_impl<R, 3, false>(which, a, pk, max_n, st);
  }
}

void launch_neighbour_list(const SweepArgs &a, void *packs, int prec, int dim, int max_n, cudaStream_t st) {
  if (prec == SPH_PREC_FP32)
    launch_sweeps<float>(3, a, packs, dim, max_n, st);
  else
    launch_sweeps<double>(3, a, packs, dim, max_n, st);
}

void launch_advection_sweep(const SweepArgs &a, void *packs, int prec, int dim, int max_n, cudaStream_t st) {
  if (prec == SPH_PREC_FP32)
    launch_sweeps<float>(0, a, packs, dim, max_n, st);
  else
    launch_sweeps<double>(0, a, packs, dim, max_n, st);
}

// the sub-step index travels in SweepArgs::sub
void launch_momentum_sweep(const SweepArgs &a, void *packs, int prec, int dim, int max_n, int,
                           cudaStream_t st) {
  if (prec == SPH_PREC_FP32)
    launch_sweeps<float>(1, a, packs, dim, max_n, st);
  else
    launch_sweeps<double>(1, a, packs, dim, max_n, st);
}

void launch_continuity_sweep(const SweepArgs &a, void *packs, int prec, int dim, int max_n, int,
                             cudaStream_t st) {
  if (prec == SPH_PREC_FP32)
    launch_sweeps<float>(2, a, packs, dim, max_n, st);
  else
    launch_sweeps<double>(2, a, packs, dim, max_n, st);
}

// sub-steps 1 .. n_ac_all - 1 (momentum and continuity) in one launch (2D)
void launch_substeps(const SweepArgs &a, void *packs, int prec, int dim, int max_n, cudaStream_t st) {
  if (prec == SPH_PREC_FP32)
    launch_sweeps<float>(4, a, packs, dim, max_n, st);
  else
    launch_sweeps<double>(4, a, packs, dim, max_n, st);
}

void launch_debug_list(const SweepArgs &a, const uint32_t *wall_index, int64_t *out, int64_t max,
                       unsigned long long *counter, int max_n, cudaStream_t st) {
  int g = (max_n + kBlock - 1) / kBlock;
  k_list_rows<<<g < 1 ? 1 : g, kBlock, 0, st>>>(a, wall_index, out, max, counter);
}

void launch_debug_pairs(const SweepArgs &a, const double *wx, const double *wy, const double *wz,
                        const uint32_t *wall_index, int64_t *out, int64_t max, unsigned long long *counter,
                        int max_n, cudaStream_t st) {
  int g = (max_n + kBlock - 1) / kBlock;
  k_pairs<<<g < 1 ? 1 : g, kBlock, 0, st>>>(a, wx, wy, wz, wall_index, out, max, counter);
}

}  // namespace sphk
