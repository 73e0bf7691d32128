/*
 * sph_oracle.h -- plain, slow FP64 CPU oracle of one WCSPH(-RANS) advection
 * step with the improved bidirectional buffer (Wang & Hu, arXiv 2510.25702).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA path; it is
 * imported by tests/, by __graft_entry__.smoke() and by bench.py's CPU
 * baseline leg, and by nothing else.  It shares no code, header, helper or
 * constant table with the CUDA library.
 *
 * Everything is FP64, compiled with -ffp-contract=off, sums taken left to
 * right in ascending neighbour order (real particles first, then wall dummies).
 * Neighbours are found by brute force O(N^2) or by a plain cell grid whose
 * per-particle lists are re-sorted into the brute-force order, so both modes
 * give bit-identical results.
 *
 * Vectors are stored with 3 components per particle ([n][3], z = 0 in 2D);
 * matrices as [n][3][3] row-major.
 */
#ifndef SPH_ORACLE_H
#define SPH_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_BUFFERS 16
#define ORC_MAX_THETA 64

/* Buffer types (Table "buffer BC" of Sec. 4.3; Sec. 2.4.2) */
#define ORC_BUF_VELOCITY 0 /* prescribed velocity profile, pressure extrapolated */
#define ORC_BUF_PRESSURE 1 /* prescribed pressure p_ob, velocity extrapolated */
/* turbulence BC on a buffer */
#define ORC_TURB_ZERO_GRADIENT 0
#define ORC_TURB_FREESTREAM 1
/* time-step modes (Sec. 2.3, dual-criteria) */
#define ORC_DT_DUAL 0   /* advection dt + n acoustic sub-steps */
#define ORC_DT_SINGLE 1 /* one sub-step of min(dt_ad, dt_ac) */
#define ORC_DT_FIXED 2  /* dt_ad and n_ac given */

/* return codes */
#define ORC_OK 0
#define ORC_ERR_ARG -1
#define ORC_ERR_CAPACITY -3
#define ORC_ERR_NOMEM -8

typedef struct orc_config {
  int dim;        /* 2 or 3 */
  int rans;       /* 0 laminar, 1 k-epsilon RANS (Sec. 2.1) */
  int dt_mode;    /* ORC_DT_* */
  int n_ac_fixed; /* sub-steps per advection step in ORC_DT_FIXED */
  double dp;      /* particle spacing */
  double h;       /* smoothing length (1.3 dp, Sec. 2.2) */
  double rho0, c0, nu_l;
  double eta;     /* ARD limiter parameter (3, Sec. 2.2) */
  double U_ref;   /* reference speed of the advection criterion */
  double dt_ad_fixed;
  double g[3];
  double lo[3], hi[3]; /* cell-grid box; periodic length = hi - lo */
  int periodic[3];
  uint32_t seed;       /* Philox key word 0 for inlet noise */
  /* switches (1 = the paper's improved scheme) used by ablation pins */
  double gen_offset; /* generation line offset in dp (0.5, Sec. 3.1) */
  int id_check;      /* delete only if particle ID == buffer ID (Sec. 3.2) */
  int contain_check; /* region-constrained labelling (Sec. 3.2) */
  int mirror_B;      /* mirror support for B at pressure buffers (Sec. 3.3) */
  int compensation;  /* compensated pressure term (Sec. 3.3, final Eq.) */
  int neighbor_mode; /* 0 brute force, 1 cell grid */
  int rkgc;          /* 1: kernel correction B (Sec. 2.2); 0: B = I (Case 1) */
  int freeze_turb;   /* 1: k, eps, nu_t held (frozen-turbulence gradient windows) */
  int comp_B;        /* compensation multiplied by B_i (final Eq. of Sec. 3.3); */
                     /* 0: the uncorrected form of the original VIPO (Cases 1-3) */
  int bhat_buffer;   /* B^_j = B_i for pressure-buffer neighbours (B_k = B_i,   */
                     /* Sec. 3.3); 0: their own B_j (Case 2)                     */
  int density_sum;   /* 1: fluid density reinitialised by kernel summation   */
                     /* once per advection step (dual-criteria scheme, Sec. 2.3) */
  int wall_fn;       /* 1: step-wise wall function at the walls (RANS, Sec. 2.3) */
  int tvf_pbuf;      /* 1: the transport-velocity shift also moves pressure-buffer
                        particles, across the buffer axis only */
  double tvf_alpha;  /* transport-velocity correction (Sec. 2.3): fluid       */
                     /* particles move by -2 alpha h^2 sum_j V_j grad_i W_ij    */
                     /* once per advection step; 0 = off                       */
} orc_config;

typedef struct orc_buffer {
  int type;    /* ORC_BUF_* */
  int turb_bc; /* ORC_TURB_* */
  int n_theta; /* samples of the velocity profile across [-half0, half0] */
  int pad0;
  double origin[3];
  double frame[9]; /* rows: n_b (into the domain), t1, t2; orthonormal */
  double length;   /* L_b along n_b */
  double half[2];  /* half widths along t1, t2 */
  double p_ob;     /* prescribed pressure (pressure buffers) */
  double noise;    /* relative amplitude of the inlet fluctuation */
  double k_in, eps_in;
  double theta[ORC_MAX_THETA];
} orc_buffer;

typedef struct orc_state {
  int64_t n;   /* entries in the arrays (live + pending-deleted) */
  int64_t cap; /* capacity of every per-particle array */
  int64_t nw;  /* wall dummies */
  /* per-particle master state (capacity cap) */
  double *pos, *vel;        /* [cap][3] */
  double *pos0;             /* [cap][3] positions of the frozen configuration
                               (start of the advection step); pair geometry
                               of every sweep in the step uses these */
  double *rho, *mass, *drho;
  double *k, *eps, *nut;    /* RANS; zero when laminar */
  int32_t *label;           /* 0 fluid, b+1 in buffer b */
  uint32_t *uid;
  uint8_t *dead;            /* deleted at the end of the last step */
  /* per-step outputs kept for inspection */
  double *p;                /* pressure (EOS) at the last sub-step */
  double *B;                /* [cap][9] correction matrix */
  double *acc_nu;           /* [cap][3] viscous acceleration */
  double *acc_p;            /* [cap][3] pressure acceleration, last sub-step */
  double *gradv;            /* [cap][9] velocity gradient (RANS) */
  /* wall dummies (fixed) */
  double *wpos, *wvel;      /* [nw][3] */
  /* counters */
  uint32_t next_uid;
  int32_t nbuf;
  int64_t step;
  double t;
  double dt_ad, dt_ac, dt; /* last step */
  int32_t n_ac;
  int32_t pad0;
  int64_t n_spawned, n_deleted; /* cumulative */
  orc_buffer buf[ORC_MAX_BUFFERS];
} orc_state;

/* kernel, Sec. 2.2 */
double orc_W(int dim, double h, double r);
double orc_dW(int dim, double h, double r);

/* Philox4x32-10 (Salmon et al., SC'11), one block */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* 53-bit uniform in [-1, 1) from two 32-bit words */
double orc_uniform_pm1(uint32_t a, uint32_t b);

/* cell index of a point (cell size 2h), -1 never; and grid dims */
int64_t orc_cell_key(const orc_config *c, const double *x);
void orc_grid_dims(const orc_config *c, int64_t nc[3]);

/* neighbour pairs of the frozen configuration: for real i, all real j != i
   and wall w with 0 < |r_ij|^2 < (2h)^2.  Writes up to max pairs as
   (i, j, is_wall) triples; returns the total count (may exceed max). */
int64_t orc_pairs(const orc_config *c, const orc_state *s, int64_t *out, int64_t max);

/* stages of one advection step, in the order orc_step runs them */
int orc_compact_sort(const orc_config *c, orc_state *s);        /* a14 commit + a1/a2 */
int orc_configure(const orc_config *c, orc_state *s);           /* pos0 = pos */
int orc_label(const orc_config *c, orc_state *s);               /* a3 */
int orc_time_step(const orc_config *c, orc_state *s);           /* a4 */
int orc_bmatrix(const orc_config *c, orc_state *s, double *A);  /* a5, A optional [cap][9] */
int orc_viscous(const orc_config *c, orc_state *s);             /* a6 */
int orc_transport(const orc_config *c, orc_state *s);           /* transport-velocity shift */
int orc_density_sum(const orc_config *c, orc_state *s);         /* density reinitialisation */
/* reference number density: sum of W over the lattice of spacing dp around
   a site, the site included (the value a perfect lattice sums to) */
double orc_lattice_kernel_sum(const orc_config *c);
/* threads the per-particle loops use (1 without OpenMP; OMP_NUM_THREADS) */
int orc_num_threads(void);
void orc_set_threads(int n);
/* friction velocity of the step-wise wall law for the tangential speed ut
   at wall distance y: viscous sublayer ut = utau^2 y / nu when
   y+ = utau y / nu <= 11.225, else ut = (utau / 0.4187) ln(9.793 y utau / nu);
   *log_layer (may be NULL) tells which */
double orc_wall_utau(double ut, double y, double nu, int *log_layer);
int orc_rans(const orc_config *c, orc_state *s, double dt);     /* a7 */
int orc_half1(const orc_config *c, orc_state *s, double dt);    /* a8 */
int orc_momentum(const orc_config *c, orc_state *s);            /* a9 force only -> acc_p */
int orc_kick(const orc_config *c, orc_state *s, double dt);     /* a9 update v, x */
int orc_continuity(const orc_config *c, orc_state *s);          /* a10 -> drho */
int orc_density(const orc_config *c, orc_state *s, double dt);  /* a10 update rho */
int orc_apply_bc(const orc_config *c, orc_state *s, int64_t step, uint32_t sub); /* a11 */
int orc_buffer_update(const orc_config *c, orc_state *s, int64_t step); /* a12 + a13 */

/* the whole step, nsteps times */
int orc_step(const orc_config *c, orc_state *s, int nsteps);

/* a one-off FP64 sum over the pair list: out[i][3] = sum_j V_j grad_i W_ij
   (used by the first-order consistency pin) */
int orc_kernel_gradient_sum(const orc_config *c, const orc_state *s, double *out);
/* sum_j W_ij V_j including the self term (partition-of-unity pin) */
int orc_kernel_sum(const orc_config *c, const orc_state *s, double *out);

#ifdef __cplusplus
}
#endif
#endif
