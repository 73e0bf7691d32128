/*
 * sph_oracle.c -- plain FP64 CPU oracle of one WCSPH(-RANS) advection step
 * with the improved bidirectional buffer (Wang & Hu, arXiv 2510.25702).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and
 * bench.py's CPU baseline; never by the product path.  Shares no code with
 * the CUDA library.  Compile with -O2 -ffp-contract=off.
 *
 * Paper sections cited: 2.1 governing equations, 2.2 discretisation,
 * 2.3 wall treatment and time stepping, 2.4 open boundary (2.4.1 buffer
 * region, 2.4.2 inflow, 2.4.3 outflow), 3.1 consistency (generation line),
 * 3.2 independence (IDs, contain check), 3.3 accuracy (mirror B and the
 * compensated pressure term), App. A (k-epsilon constants).
 *
 * Where the paper is silent or garbled, the reading taken is stated beside
 * the function.  Frozen configuration: every pair sum of an advection step
 * uses the positions pos0 taken at the start of that step (the dual-criteria
 * scheme updates the configuration once per advection step); the positions
 * pos are integrated through the sub-steps and used by the buffer update.
 */
#include "sph_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PI_D 3.14159265358979323846

/* k-epsilon constants, App. A table */
#define KE_C1 1.44
#define KE_C2 1.92
#define KE_CMU 0.09
#define KE_SIGMA_K 1.0
#define KE_SIGMA_E 1.3
#define KE_FLOOR 1e-12

/* sub-step index used for the noise of a recycled buffer particle */
#define SUB_RECYCLE 0xFFFFFFFFu

/* ------------------------------------------------------------------ */
/* Kernel: Wendland C2 with support 2h, h = 1.3 dp (Sec. 2.2).         */
/* W(q) = a_d (1 - q/2)^4 (1 + 2q), a_2 = 7/(4 pi h^2),                */
/* a_3 = 21/(16 pi h^3);  dW/dr = (a_d/h)(-5q)(1 - q/2)^3.             */
/* ------------------------------------------------------------------ */
static double wendland_alpha(int dim, double h) {
  if (dim == 2) return 7.0 / (4.0 * PI_D * h * h);
  return 21.0 / (16.0 * PI_D * h * h * h);
}

double orc_W(int dim, double h, double r) {
  double q = r / h;
  if (!(q < 2.0)) return 0.0;
  double a = 1.0 - 0.5 * q;
  return wendland_alpha(dim, h) * a * a * a * a * (1.0 + 2.0 * q);
}

double orc_dW(int dim, double h, double r) {
  double q = r / h;
  if (!(q < 2.0)) return 0.0;
  double a = 1.0 - 0.5 * q;
  return wendland_alpha(dim, h) / h * (-5.0 * q) * a * a * a;
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10, written from Salmon, Moraes, Dror, Shaw, "Parallel   */
/* random numbers: as easy as 1, 2, 3", SC'11: per round two 32x32->64  */
/* products, outputs mixed with the key; Weyl key schedule; 10 rounds. */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* 53-bit uniform u in [0,1) from the top 27 bits of a and 26 bits of b,
   mapped to [-1, 1) by 2u - 1 (both steps exact in FP64). */
double orc_uniform_pm1(uint32_t a, uint32_t b) {
  double m = (double)(a >> 5) * 67108864.0 + (double)(b >> 6);
  double u = m * (1.0 / 9007199254740992.0);
  return 2.0 * u - 1.0;
}

/* ------------------------------------------------------------------ */
/* small helpers (left-to-right sums, no contraction)                  */
/* ------------------------------------------------------------------ */
static double dotd(int dim, const double *a, const double *b) {
  double s = 0.0;
  for (int k = 0; k < dim; ++k) s += a[k] * b[k];
  return s;
}

/* r_ij = x_i - x_j with the minimum image on periodic axes */
static void pair_vector(const orc_config *c, const double *xi, const double *xj, double *r) {
  for (int a = 0; a < 3; ++a) r[a] = 0.0;
  for (int a = 0; a < c->dim; ++a) {
    double d = xi[a] - xj[a];
    if (c->periodic[a]) {
      double L = c->hi[a] - c->lo[a];
      if (d > 0.5 * L)
        d -= L;
      else if (d < -0.5 * L)
        d += L;
    }
    r[a] = d;
  }
}

static double cutoff2(const orc_config *c) {
  double s = 2.0 * c->h;
  return s * s;
}

static double wall_volume(const orc_config *c) {
  double v = c->dp * c->dp;
  if (c->dim == 3) v *= c->dp;
  return v;
}

/* buffer-local coordinate k of x: (x - o) . frame_row_k (the coordinate
   transform of the aligned box, Sec. 3.2) */
static double local_coord(const orc_config *c, const orc_buffer *b, const double *x, int k) {
  double d[3];
  for (int a = 0; a < 3; ++a) d[a] = x[a] - b->origin[a];
  return dotd(c->dim, d, &b->frame[3 * k]);
}

static double vol_of(const orc_state *s, int64_t j) { return s->mass[j] / s->rho[j]; }

static int is_pressure_buffer(const orc_state *s, int32_t label) {
  return label > 0 && label <= s->nbuf && s->buf[label - 1].type == ORC_BUF_PRESSURE;
}

/* y = M x for a row-major 3x3 M restricted to dim */
static void matvec(int dim, const double *M, const double *x, double *y) {
  for (int a = 0; a < 3; ++a) y[a] = 0.0;
  for (int a = 0; a < dim; ++a) y[a] = dotd(dim, &M[3 * a], x);
}

static double eos(const orc_config *c, double rho) {
  return c->rho0 * c->c0 * c->c0 * (rho / c->rho0 - 1.0);
}

/* ------------------------------------------------------------------ */
/* a1: cell binning with cell size 2h (>= cut-off; Sec. 2.4.1).        */
/* cell = floor((x - lo) / 2h) clamped to [0, n-1], n = floor(L / 2h).  */
/* ------------------------------------------------------------------ */
void orc_grid_dims(const orc_config *c, int64_t nc[3]) {
  double cs = 2.0 * c->h;
  for (int a = 0; a < 3; ++a) {
    nc[a] = 1;
    if (a < c->dim) {
      double f = floor((c->hi[a] - c->lo[a]) / cs);
      nc[a] = (f >= 1.0) ? (int64_t)f : 1;
    }
  }
}

static int64_t cell_coord(const orc_config *c, const double *x, int a, const int64_t *nc) {
  double cs = 2.0 * c->h;
  double f = floor((x[a] - c->lo[a]) / cs);
  if (!(f >= 0.0)) return 0;
  if (f >= (double)nc[a]) return nc[a] - 1;
  return (int64_t)f;
}

int64_t orc_cell_key(const orc_config *c, const double *x) {
  int64_t nc[3];
  orc_grid_dims(c, nc);
  int64_t cx = cell_coord(c, x, 0, nc);
  int64_t cy = cell_coord(c, x, 1, nc);
  int64_t cz = (c->dim == 3) ? cell_coord(c, x, 2, nc) : 0;
  return (cz * nc[1] + cy) * nc[0] + cx;
}

/* ------------------------------------------------------------------ */
/* Neighbour lists of the frozen configuration                          */
/* ------------------------------------------------------------------ */
typedef struct {
  int64_t j;
  int32_t wall;
} nb_t;

typedef struct {
  int64_t *start; /* n+1 */
  nb_t *nb;
  int64_t count, cap;
} nblist;

static void nblist_free(nblist *L) {
  free(L->start);
  free(L->nb);
  L->start = NULL;
  L->nb = NULL;
}

static int nblist_push(nblist *L, int64_t j, int wall) {
  if (L->count == L->cap) {
    int64_t nc = L->cap ? 2 * L->cap : 1024;
    nb_t *p = (nb_t *)realloc(L->nb, (size_t)nc * sizeof(nb_t));
    if (!p) return ORC_ERR_NOMEM;
    L->nb = p;
    L->cap = nc;
  }
  L->nb[L->count].j = j;
  L->nb[L->count].wall = wall;
  L->count++;
  return ORC_OK;
}

static int nb_cmp(const void *a, const void *b) {
  const nb_t *x = (const nb_t *)a, *y = (const nb_t *)b;
  if (x->wall != y->wall) return x->wall < y->wall ? -1 : 1;
  if (x->j != y->j) return x->j < y->j ? -1 : 1;
  return 0;
}

/* plain cell grid (CSR by cell) over the real particles (pos0) and walls */
typedef struct {
  int64_t nc[3];
  int64_t ncell;
  int64_t *rstart, *ridx;
  int64_t *wstart, *widx;
} grid_t;

static void grid_free(grid_t *g) {
  free(g->rstart);
  free(g->ridx);
  free(g->wstart);
  free(g->widx);
  memset(g, 0, sizeof(*g));
}

static int grid_build_set(const orc_config *c, const double *pos, int64_t n, const uint8_t *skip,
                          int64_t ncell, int64_t **start_out, int64_t **idx_out) {
  int64_t *start = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
  int64_t *idx = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  int64_t *fill = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
  if (!start || !idx || !fill) {
    free(start);
    free(idx);
    free(fill);
    return ORC_ERR_NOMEM;
  }
  for (int64_t i = 0; i < n; ++i) {
    if (skip && skip[i]) continue;
    start[orc_cell_key(c, &pos[3 * i]) + 1]++;
  }
  for (int64_t k = 0; k < ncell; ++k) start[k + 1] += start[k];
  for (int64_t i = 0; i < n; ++i) {
    if (skip && skip[i]) continue;
    int64_t key = orc_cell_key(c, &pos[3 * i]);
    idx[start[key] + fill[key]++] = i;
  }
  free(fill);
  *start_out = start;
  *idx_out = idx;
  return ORC_OK;
}

static int grid_build(const orc_config *c, const orc_state *s, grid_t *g) {
  memset(g, 0, sizeof(*g));
  orc_grid_dims(c, g->nc);
  g->ncell = g->nc[0] * g->nc[1] * g->nc[2];
  int rc = grid_build_set(c, s->pos0, s->n, s->dead, g->ncell, &g->rstart, &g->ridx);
  if (rc) return rc;
  return grid_build_set(c, s->wpos, s->nw, NULL, g->ncell, &g->wstart, &g->widx);
}

/* every real / wall index in the cells within +-span of q's cell (periodic
   wrap where set, each distinct cell visited once), appended to L */
static int grid_candidates(const orc_config *c, const grid_t *g, const double *q, int span,
                           nblist *L) {
  int64_t cc[3] = {0, 0, 0};
  for (int a = 0; a < c->dim; ++a) cc[a] = cell_coord(c, q, a, g->nc);
  int64_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int a = 0; a < c->dim; ++a) {
    lo[a] = cc[a] - span;
    hi[a] = cc[a] + span;
  }
  int64_t seen[125];
  int64_t nseen = 0;
  for (int64_t z = lo[2]; z <= hi[2]; ++z)
    for (int64_t y = lo[1]; y <= hi[1]; ++y)
      for (int64_t x = lo[0]; x <= hi[0]; ++x) {
        int64_t v[3] = {x, y, z};
        int ok = 1;
        for (int a = 0; a < c->dim; ++a) {
          if (v[a] < 0 || v[a] >= g->nc[a]) {
            if (c->periodic[a])
              v[a] = ((v[a] % g->nc[a]) + g->nc[a]) % g->nc[a];
            else
              ok = 0;
          }
        }
        if (!ok) continue;
        int64_t key = (v[2] * g->nc[1] + v[1]) * g->nc[0] + v[0];
        int dup = 0;
        for (int64_t t = 0; t < nseen; ++t)
          if (seen[t] == key) dup = 1;
        if (dup) continue;
        if (nseen < 125) seen[nseen++] = key;
        for (int64_t t = g->rstart[key]; t < g->rstart[key + 1]; ++t)
          if (nblist_push(L, g->ridx[t], 0)) return ORC_ERR_NOMEM;
        for (int64_t t = g->wstart[key]; t < g->wstart[key + 1]; ++t)
          if (nblist_push(L, g->widx[t], 1)) return ORC_ERR_NOMEM;
      }
  return ORC_OK;
}

static int all_candidates(const orc_state *s, nblist *cand) {
  for (int64_t j = 0; j < s->n; ++j)
    if (!s->dead[j] && nblist_push(cand, j, 0)) return ORC_ERR_NOMEM;
  for (int64_t w = 0; w < s->nw; ++w)
    if (nblist_push(cand, w, 1)) return ORC_ERR_NOMEM;
  return ORC_OK;
}

/* Neighbours of the frozen configuration: real j != i and wall w with
   0 < |r_ij|^2 < (2h)^2 (the tie at the cut-off is out, coincident pairs
   are skipped), in ascending (wall, j) order whichever mode finds them. */
static int build_pairs(const orc_config *c, const orc_state *s, nblist *L) {
  memset(L, 0, sizeof(*L));
  L->start = (int64_t *)calloc((size_t)s->n + 1, sizeof(int64_t));
  if (!L->start) return ORC_ERR_NOMEM;
  double cut2 = cutoff2(c);
  grid_t g;
  int use_grid = (c->neighbor_mode == 1);
  if (use_grid && grid_build(c, s, &g)) return ORC_ERR_NOMEM;
  int rc = ORC_OK;
  /* two passes over the particles (threads take particles independently):
     count each list, place the lists by a prefix sum, then fill them */
  for (int pass = 0; pass < 2 && rc == ORC_OK; ++pass) {
    if (pass == 1) {
      int64_t tot = 0;
      for (int64_t i = 0; i < s->n; ++i) {
        int64_t k = L->start[i];
        L->start[i] = tot;
        tot += k;
      }
      L->start[s->n] = tot;
      L->count = L->cap = tot;
      L->nb = (nb_t *)malloc((size_t)(tot > 0 ? tot : 1) * sizeof(nb_t));
      if (!L->nb) {
        rc = ORC_ERR_NOMEM;
        break;
      }
    }
#pragma omp parallel
    {
      nblist cand;
      memset(&cand, 0, sizeof(cand));
#pragma omp for schedule(dynamic, 256)
      for (int64_t i = 0; i < s->n; ++i) {
        int64_t k = 0;
        if (!s->dead[i]) {
          const double *xi = &s->pos0[3 * i];
          cand.count = 0;
          int r;
          if (use_grid) {
            r = grid_candidates(c, &g, xi, 1, &cand);
            if (!r) qsort(cand.nb, (size_t)cand.count, sizeof(nb_t), nb_cmp);
          } else {
            r = all_candidates(s, &cand);
          }
          if (r) {
#pragma omp atomic write
            rc = r;
          } else {
            for (int64_t t = 0; t < cand.count; ++t) {
              int64_t j = cand.nb[t].j;
              int wall = cand.nb[t].wall;
              if (!wall && j == i) continue;
              const double *xj = wall ? &s->wpos[3 * j] : &s->pos0[3 * j];
              double rv[3];
              pair_vector(c, xi, xj, rv);
              double rr = dotd(c->dim, rv, rv);
              if (rr > 0.0 && rr < cut2) {
                if (pass == 1) {
                  L->nb[L->start[i] + k].j = j;
                  L->nb[L->start[i] + k].wall = wall;
                }
                ++k;
              }
            }
          }
        }
        if (pass == 0) L->start[i] = k;
      }
      free(cand.nb);
    }
  }
  if (use_grid) grid_free(&g);
  return rc;
}

int64_t orc_pairs(const orc_config *c, const orc_state *s, int64_t *out, int64_t max) {
  nblist L;
  if (build_pairs(c, s, &L)) return ORC_ERR_NOMEM;
  int64_t m = 0;
  for (int64_t i = 0; i < s->n; ++i)
    for (int64_t t = L.start[i]; t < L.start[i + 1]; ++t) {
      if (m < max) {
        out[3 * m + 0] = i;
        out[3 * m + 1] = L.nb[t].j;
        out[3 * m + 2] = L.nb[t].wall;
      }
      ++m;
    }
  nblist_free(&L);
  return m;
}

/* geometry of a listed pair from pos0: r_ij, |r_ij|, dW/dr, grad_i W */
typedef struct {
  double r[3];
  double rl;
  double dw;
  double gw[3];
} geom_t;

static void pair_geom(const orc_config *c, const double *xi, const double *xj, geom_t *G) {
  pair_vector(c, xi, xj, G->r);
  G->rl = sqrt(dotd(c->dim, G->r, G->r));
  G->dw = orc_dW(c->dim, c->h, G->rl);
  for (int a = 0; a < 3; ++a) G->gw[a] = G->dw * (G->r[a] / G->rl);
}

static const double *xj_of(const orc_state *s, int64_t j, int wall) {
  return wall ? &s->wpos[3 * j] : &s->pos0[3 * j];
}

/* ------------------------------------------------------------------ */
/* a14 commit + a1/a2.  Particles marked deleted by the last buffer     */
/* update are dropped; survivors keep index order and the copies        */
/* appended at the end of the array (Sec. 2.4.2) follow.  Periodic axes */
/* are wrapped, then the array is stable-sorted by cell key: the cell-   */
/* linked list is rebuilt after deletion each advection step            */
/* (Sec. 2.4.3).  The paper's overwrite-with-last deletion is replaced   */
/* by this stable compaction, so indices differ from SPHinXsys.          */
/* ------------------------------------------------------------------ */
typedef struct {
  int64_t key, idx;
} keyidx_t;

static int keyidx_cmp(const void *a, const void *b) {
  const keyidx_t *x = (const keyidx_t *)a, *y = (const keyidx_t *)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
  return 0;
}

static int permute(void *arr, size_t elem, const keyidx_t *ord, int64_t m) {
  char *src = (char *)arr;
  char *tmp = (char *)malloc((size_t)(m > 0 ? m : 1) * elem);
  if (!tmp) return ORC_ERR_NOMEM;
  for (int64_t t = 0; t < m; ++t) memcpy(tmp + (size_t)t * elem, src + (size_t)ord[t].idx * elem, elem);
  memcpy(src, tmp, (size_t)m * elem);
  free(tmp);
  return ORC_OK;
}

int orc_compact_sort(const orc_config *c, orc_state *s) {
  keyidx_t *ord = (keyidx_t *)malloc((size_t)(s->n > 0 ? s->n : 1) * sizeof(keyidx_t));
  if (!ord) return ORC_ERR_NOMEM;
  int64_t m = 0;
  for (int64_t i = 0; i < s->n; ++i) {
    if (s->dead[i]) continue;
    double *x = &s->pos[3 * i];
    for (int a = 0; a < c->dim; ++a)
      if (c->periodic[a]) {
        double L = c->hi[a] - c->lo[a];
        if (x[a] >= c->hi[a])
          x[a] -= L;
        else if (x[a] < c->lo[a])
          x[a] += L;
      }
    ord[m].key = orc_cell_key(c, x);
    ord[m].idx = i;
    ++m;
  }
  qsort(ord, (size_t)m, sizeof(keyidx_t), keyidx_cmp);
  int rc = 0;
  rc |= permute(s->pos, 3 * sizeof(double), ord, m);
  rc |= permute(s->vel, 3 * sizeof(double), ord, m);
  rc |= permute(s->rho, sizeof(double), ord, m);
  rc |= permute(s->mass, sizeof(double), ord, m);
  rc |= permute(s->drho, sizeof(double), ord, m);
  rc |= permute(s->k, sizeof(double), ord, m);
  rc |= permute(s->eps, sizeof(double), ord, m);
  rc |= permute(s->nut, sizeof(double), ord, m);
  rc |= permute(s->label, sizeof(int32_t), ord, m);
  rc |= permute(s->uid, sizeof(uint32_t), ord, m);
  free(ord);
  if (rc) return ORC_ERR_NOMEM;
  s->n = m;
  memset(s->dead, 0, (size_t)s->cap);
  return ORC_OK;
}

int orc_configure(const orc_config *c, orc_state *s) {
  (void)c;
  memcpy(s->pos0, s->pos, (size_t)s->n * 3 * sizeof(double));
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* a3: region-constrained, independent labelling (Sec. 3.2).           */
/* In the buffer frame x' = F_b (x - o_b), the particle is in buffer b  */
/* iff 0 <= x'_0 < L_b and |x'_k| <= half_k; it then gets label b+1     */
/* (its buffer ID).  Outside every box the label is unchanged:          */
/* relabelling happens only inside the buffer region (Sec. 3.1).        */
/* contain_check = 0 (ablation of Sec. 3.2): the lateral test becomes   */
/* membership of the particle's cell in the buffer's local cell list    */
/* (the box's cells dilated by one cell ring).                          */
/* ------------------------------------------------------------------ */
static int in_local_cells(const orc_config *c, const orc_buffer *b, const double *x) {
  double cs = 2.0 * c->h;
  double lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    lo[a] = 1e300;
    hi[a] = -1e300;
  }
  int nz = (c->dim == 3) ? 2 : 1;
  for (int i0 = 0; i0 < 2; ++i0)
    for (int i1 = 0; i1 < 2; ++i1)
      for (int i2 = 0; i2 < nz; ++i2) {
        double u0 = i0 ? b->length : 0.0;
        double u1 = i1 ? b->half[0] : -b->half[0];
        double u2 = (c->dim == 3) ? (i2 ? b->half[1] : -b->half[1]) : 0.0;
        for (int a = 0; a < 3; ++a) {
          double p = b->origin[a] + u0 * b->frame[a] + u1 * b->frame[3 + a] + u2 * b->frame[6 + a];
          if (p < lo[a]) lo[a] = p;
          if (p > hi[a]) hi[a] = p;
        }
      }
  int64_t nc[3];
  orc_grid_dims(c, nc);
  for (int a = 0; a < c->dim; ++a) {
    double ql[3] = {lo[a] - cs, lo[a] - cs, lo[a] - cs};
    double qu[3] = {hi[a] + cs, hi[a] + cs, hi[a] + cs};
    int64_t ca = cell_coord(c, x, a, nc);
    if (ca < cell_coord(c, ql, a, nc) || ca > cell_coord(c, qu, a, nc)) return 0;
  }
  return 1;
}

static int box_contains(const orc_config *c, const orc_buffer *b, const double *x) {
  double s0 = local_coord(c, b, x, 0);
  if (!(s0 >= 0.0 && s0 < b->length)) return 0;
  if (!c->contain_check) return in_local_cells(c, b, x);
  double s1 = local_coord(c, b, x, 1);
  if (!(fabs(s1) <= b->half[0])) return 0;
  if (c->dim == 3) {
    double s2 = local_coord(c, b, x, 2);
    if (!(fabs(s2) <= b->half[1])) return 0;
  }
  return 1;
}

int orc_label(const orc_config *c, orc_state *s) {
  #pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < s->n; ++i) {
    if (s->dead[i]) continue;
    for (int b = 0; b < s->nbuf; ++b)
      if (box_contains(c, &s->buf[b], &s->pos[3 * i])) s->label[i] = b + 1;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* a4: dual-criteria time step (Sec. 2.3 names the two criteria; the   */
/* constants are the usual ones of the dual-criteria scheme):           */
/*   dt_ad = min(0.25 h / max(|v|max, U_ref), 0.125 h^2 / nu_eff,max)   */
/*   dt_ac = 0.6 h / (c0 + |v|max)                                      */
/* DUAL: n = ceil(dt_ad / dt_ac) equal sub-steps dt_ad / n, so the      */
/* sub-steps add up to dt_ad.  SINGLE: one sub-step of min(dt_ad,dt_ac). */
/* ------------------------------------------------------------------ */
int orc_time_step(const orc_config *c, orc_state *s) {
  double v2max = 0.0, nutmax = 0.0;
  for (int64_t i = 0; i < s->n; ++i) {
    if (s->dead[i]) continue;
    double v2 = dotd(c->dim, &s->vel[3 * i], &s->vel[3 * i]);
    if (v2 > v2max) v2max = v2;
    if (c->rans && s->nut[i] > nutmax) nutmax = s->nut[i];
  }
  double vmax = sqrt(v2max);
  double u = (vmax > c->U_ref) ? vmax : c->U_ref;
  double dt_adv = 0.25 * c->h / u;
  double nu_eff = c->nu_l + nutmax;
  double dt_visc = 0.125 * c->h * c->h / nu_eff;
  double dt_ad = (dt_adv < dt_visc) ? dt_adv : dt_visc;
  double dt_ac = 0.6 * c->h / (c->c0 + vmax);
  int n;
  if (c->dt_mode == ORC_DT_FIXED) {
    dt_ad = c->dt_ad_fixed;
    n = c->n_ac_fixed;
  } else if (c->dt_mode == ORC_DT_SINGLE) {
    if (dt_ac < dt_ad) dt_ad = dt_ac;
    n = 1;
  } else {
    double f = ceil(dt_ad / dt_ac);
    n = (f >= 1.0) ? (int)f : 1;
  }
  if (n < 1) return ORC_ERR_ARG;
  s->dt_ad = dt_ad;
  s->dt_ac = dt_ac;
  s->n_ac = n;
  s->dt = dt_ad / (double)n;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* a5: correction matrix B_i = (-sum_j r_ij (x) grad_i W_ij V_j)^-1     */
/* (Sec. 2.2) over real neighbours and wall dummies.                   */
/* Mirror condition (Sec. 3.3): for a particle                          */
/* labelled in a pressure buffer, neighbours beyond the open face       */
/* (x'_0 < 0 in that buffer's frame) are left out and the mirror        */
/* images across the face x'_0 = 0 of every particle with x'_0 >= 0     */
/* are summed instead, so the truncated support is completed.           */
/* Guard (the paper is silent): det A <= 1e-3 (tr A / d)^d             */
/* gives B = I.                                                         */
/* ------------------------------------------------------------------ */
static void accum_A(int dim, double *A, const double *r, const double *gw, double V) {
  for (int a = 0; a < dim; ++a)
    for (int b = 0; b < dim; ++b) A[3 * a + b] += (-r[a]) * gw[b] * V;
}

static void invert_guarded(int dim, const double *A, double *B) {
  for (int k = 0; k < 9; ++k) B[k] = 0.0;
  double tr = 0.0;
  for (int a = 0; a < dim; ++a) tr += A[4 * a];
  double t = tr / (double)dim;
  double thr = (dim == 2) ? 1e-3 * t * t : 1e-3 * t * t * t;
  if (dim == 2) {
    double det = A[0] * A[4] - A[1] * A[3];
    if (!(det > thr)) {
      B[0] = 1.0;
      B[4] = 1.0;
      return;
    }
    B[0] = A[4] / det;
    B[1] = -A[1] / det;
    B[3] = -A[3] / det;
    B[4] = A[0] / det;
  } else {
    double c00 = A[4] * A[8] - A[5] * A[7];
    double c01 = A[5] * A[6] - A[3] * A[8];
    double c02 = A[3] * A[7] - A[4] * A[6];
    double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    if (!(det > thr)) {
      B[0] = 1.0;
      B[4] = 1.0;
      B[8] = 1.0;
      return;
    }
    B[0] = c00 / det;
    B[1] = (A[2] * A[7] - A[1] * A[8]) / det;
    B[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    B[3] = c01 / det;
    B[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    B[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    B[6] = c02 / det;
    B[7] = (A[1] * A[6] - A[0] * A[7]) / det;
    B[8] = (A[0] * A[4] - A[1] * A[3]) / det;
  }
}

static int orc_bmatrix_impl(const orc_config *c, orc_state *s, double *Aout, const nblist *Lp) {
  const nblist L = *Lp;
  grid_t g;
  int use_grid = (c->neighbor_mode == 1);
  if (use_grid && grid_build(c, s, &g)) return ORC_ERR_NOMEM;
  double cut2 = cutoff2(c);
  double Vw = wall_volume(c);
  int rc = ORC_OK;
#pragma omp parallel
  {
  nblist cand;
  memset(&cand, 0, sizeof(cand));
#pragma omp for schedule(dynamic, 256)
  for (int64_t i = 0; i < s->n; ++i) {
    if (s->dead[i]) continue;
    const double *xi = &s->pos0[3 * i];
    double A[9] = {0};
    int mirror = c->mirror_B && is_pressure_buffer(s, s->label[i]);
    const orc_buffer *b = mirror ? &s->buf[s->label[i] - 1] : NULL;
    for (int64_t t = L.start[i]; t < L.start[i + 1]; ++t) {
      int64_t j = L.nb[t].j;
      int wall = L.nb[t].wall;
      const double *xj = xj_of(s, j, wall);
      if (mirror && local_coord(c, b, xj, 0) < 0.0) continue;
      geom_t G;
      pair_geom(c, xi, xj, &G);
      accum_A(c->dim, A, G.r, G.gw, wall ? Vw : vol_of(s, j));
    }
    if (mirror) {
      /* image of j: m_j = x_j - 2 x'_0(x_j) n_b; pair vector d = x_i - m_j */
      cand.count = 0;
      if (use_grid) {
        /* |x_i - M x_j| = |M x_i - x_j|: search around the image of x_i with a
           two-cell margin so that rounding never drops a candidate */
        double si = local_coord(c, b, xi, 0);
        double q[3];
        for (int a = 0; a < 3; ++a) q[a] = xi[a] - 2.0 * si * b->frame[a];
        int r = grid_candidates(c, &g, q, 2, &cand);
        if (r) {
#pragma omp atomic write
          rc = r;
          continue;
        }
        qsort(cand.nb, (size_t)cand.count, sizeof(nb_t), nb_cmp);
      } else {
        int r = all_candidates(s, &cand);
        if (r) {
#pragma omp atomic write
          rc = r;
          continue;
        }
      }
      for (int64_t t = 0; t < cand.count; ++t) {
        int64_t j = cand.nb[t].j;
        int wall = cand.nb[t].wall;
        const double *xj = xj_of(s, j, wall);
        double sj = local_coord(c, b, xj, 0);
        if (sj < 0.0) continue;
        double d[3] = {0, 0, 0};
        for (int a = 0; a < c->dim; ++a) d[a] = xi[a] - (xj[a] - 2.0 * sj * b->frame[a]);
        double dd = dotd(c->dim, d, d);
        if (!(dd > 0.0 && dd < cut2)) continue;
        double dl = sqrt(dd);
        double dw = orc_dW(c->dim, c->h, dl);
        double gw[3] = {0, 0, 0};
        for (int a = 0; a < c->dim; ++a) gw[a] = dw * (d[a] / dl);
        accum_A(c->dim, A, d, gw, wall ? Vw : vol_of(s, j));
      }
    }
    if (Aout) memcpy(&Aout[9 * i], A, sizeof(A));
    if (c->rkgc) {
      invert_guarded(c->dim, A, &s->B[9 * i]);
    } else {
      for (int q = 0; q < 9; ++q) s->B[9 * i + q] = (q % 4 == 0 && q / 4 < c->dim) ? 1.0 : 0.0;
    }
  }
  free(cand.nb);
  }
  if (use_grid) grid_free(&g);
  return rc;
}

int orc_bmatrix(const orc_config *c, orc_state *s, double *Aout) {
  nblist L;
  if (build_pairs(c, s, &L)) return ORC_ERR_NOMEM;
  int rc = orc_bmatrix_impl(c, s, Aout, &L);
  nblist_free(&L);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Step-wise wall function (Sec. 2.3 uses the one of its reference for   */
/* turbulent walls and gives no formula; this is the standard two-layer  */
/* wall law).  A near-wall particle is a fluid particle (label 0) of a   */
/* RANS run with the wall function on that has wall neighbours and lies  */
/* less than dp from the wall surface: y_i = min_w |r_iw| - dp/2 (the    */
/* first dummy layer sits dp/2 inside the wall).  Its wall normal is     */
/* n = -sum_w V_w grad_i W_iw normalised (pointing away from the wall),  */
/* its tangential speed u_t = |v_r - (v_r . n) n| with v_r = v_i - v_w of */
/* the nearest dummy.  The friction velocity u_tau solves the viscous    */
/* sublayer law u_t = u_tau^2 y / nu_l while y+ = u_tau y / nu_l <=      */
/* 11.225 (where the two laws meet), else the log law                    */
/* u_t = (u_tau / kappa) ln(E y u_tau / nu_l), kappa = 0.4187, E = 9.793 */
/* (the two laws meet at y+ = 11.225), by 8 Newton steps from the        */
/* sublayer value (the log-law residual is                               */
/* convex and increasing in u_tau and that value lies below the root).   */
/* Effects: the viscous term of its wall pairs uses nu_w = u_tau^2 y /   */
/* u_t, so that the wall shear stress is rho0 u_tau^2; in the k-eps      */
/* sweep its production is the log-law value G_k = u_tau^3 / (kappa y)    */
/* (0 in the sublayer) and after the update eps is set to the wall value */
/* C_mu^(3/4) k^(3/2) / (kappa y) (2 nu_l k / y^2 in the sublayer).      */
/* ------------------------------------------------------------------ */
#define WF_KAPPA 0.4187
#define WF_E 9.793
#define WF_YPLUS 11.225

double orc_wall_utau(double ut, double y, double nu, int *log_layer) {
  if (!(ut > 0.0) || !(y > 0.0)) {
    if (log_layer) *log_layer = 0;
    return 0.0;
  }
  double u = sqrt(nu * ut / y);
  if (u * y / nu <= WF_YPLUS) {
    if (log_layer) *log_layer = 0;
    return u;
  }
  for (int it = 0; it < 8; ++it) {
    double L = log(WF_E * y * u / nu);
    double f = u * L / WF_KAPPA - ut;
    double fp = (L + 1.0) / WF_KAPPA;
    u = u - f / fp;
  }
  if (log_layer) *log_layer = 1;
  return u;
}

typedef struct {
  int on;        /* near-wall particle */
  int log_layer; /* u_tau from the log law */
  double y, ut, utau;
} nearwall_t;

static void near_wall(const orc_config *c, const orc_state *s, const nblist *L, int64_t i, nearwall_t *w) {
  memset(w, 0, sizeof(*w));
  if (!c->rans || !c->wall_fn || s->label[i] != 0) return;
  double Vw = wall_volume(c);
  double rmin = 0.0, nsum[3] = {0, 0, 0};
  int64_t wmin = -1;
  for (int64_t t = L->start[i]; t < L->start[i + 1]; ++t) {
    if (!L->nb[t].wall) continue;
    int64_t j = L->nb[t].j;
    geom_t G;
    pair_geom(c, &s->pos0[3 * i], &s->wpos[3 * j], &G);
    if (wmin < 0 || G.rl < rmin) {
      rmin = G.rl;
      wmin = j;
    }
    for (int a = 0; a < 3; ++a) nsum[a] -= Vw * G.gw[a];
  }
  if (wmin < 0) return;
  double y = rmin - 0.5 * c->dp;
  if (!(y > 0.0 && y < c->dp)) return;
  double nn = sqrt(dotd(c->dim, nsum, nsum));
  if (!(nn > 0.0)) return;
  double vr[3] = {0, 0, 0}, vn = 0.0;
  for (int a = 0; a < c->dim; ++a) {
    vr[a] = s->vel[3 * i + a] - s->wvel[3 * wmin + a];
    vn += vr[a] * (nsum[a] / nn);
  }
  double ut2 = 0.0;
  for (int a = 0; a < c->dim; ++a) {
    double t = vr[a] - vn * (nsum[a] / nn);
    ut2 += t * t;
  }
  w->on = 1;
  w->y = y;
  w->ut = sqrt(ut2);
  w->utau = orc_wall_utau(w->ut, y, c->nu_l, &w->log_layer);
}

/* ------------------------------------------------------------------ */
/* a6: ARD viscous acceleration (Sec. 2.2), once per advection step:    */
/*   a_i = (2/rho_i) sum_j mu_ad v_ij dW/(r_ij + 0.01h) V_j,            */
/*   mu_ad = max(harmonic(mu_i, mu_j), mu_R), mu = rho0 nu_eff,         */
/*   mu_R = 0.5 rho0 h min(eta max(v_ij . e_ij, 0), c0), e_ij the unit  */
/*   vector from i to j; mu_R = 0 when laminar.                         */
/* Wall dummy (no-slip, Sec. 2.3): the dummy carries v_j = 2 v_wall - v_i */
/* so that the no-slip plane lies on the wall surface, and the harmonic  */
/* mean is replaced by mu_i.  (Taking v_j = v_wall instead puts the    */
/* no-slip plane inside the wall and fails the Poiseuille pin.)         */
/* ------------------------------------------------------------------ */
static double mu_of(const orc_config *c, const orc_state *s, int64_t i) {
  double nu = c->nu_l + (c->rans ? s->nut[i] : 0.0);
  return c->rho0 * nu;
}

static int orc_viscous_impl(const orc_config *c, orc_state *s, const nblist *Lp) {
  const nblist L = *Lp;
  double Vw = wall_volume(c);
  #pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < s->n; ++i) {
    if (s->dead[i]) continue;
    const double *xi = &s->pos0[3 * i];
    const double *vi = &s->vel[3 * i];
    double mui = mu_of(c, s, i);
    /* wall pairs of a near-wall particle: the wall-function viscosity */
    double muw = mui;
    nearwall_t nw;
    near_wall(c, s, &L, i, &nw);
    if (nw.on && nw.ut > 0.0) muw = c->rho0 * (nw.utau * nw.utau * nw.y / nw.ut);
    double S[3] = {0, 0, 0};
    for (int64_t t = L.start[i]; t < L.start[i + 1]; ++t) {
      int64_t j = L.nb[t].j;
      int wall = L.nb[t].wall;
      geom_t G;
      pair_geom(c, xi, xj_of(s, j, wall), &G);
      double vij[3] = {0, 0, 0};
      for (int a = 0; a < c->dim; ++a) {
        double vj = wall ? 2.0 * s->wvel[3 * j + a] - vi[a] : s->vel[3 * j + a];
        vij[a] = vi[a] - vj;
      }
      double mut;
      if (wall) {
        mut = muw;
      } else {
        double muj = mu_of(c, s, j);
        mut = 2.0 * mui * muj / (mui + muj);
      }
      double muR = 0.0;
      if (c->rans) {
        double ve = -dotd(c->dim, vij, G.r) / G.rl;
        double lim = c->eta * (ve > 0.0 ? ve : 0.0);
        double beta = lim < c->c0 ? lim : c->c0;
        muR = 0.5 * c->rho0 * c->h * beta;
      }
      double mu_ad = mut > muR ? mut : muR;
      double V = wall ? Vw : vol_of(s, j);
      double f = mu_ad * (G.dw / (G.rl + 0.01 * c->h)) * V;
      for (int a = 0; a < c->dim; ++a) S[a] += f * vij[a];
    }
    for (int a = 0; a < 3; ++a) s->acc_nu[3 * i + a] = (a < c->dim) ? 2.0 * S[a] / s->rho[i] : 0.0;
  }
  return ORC_OK;
}

int orc_viscous(const orc_config *c, orc_state *s) {
  nblist L;
  if (build_pairs(c, s, &L)) return ORC_ERR_NOMEM;
  int rc = orc_viscous_impl(c, s, &L);
  nblist_free(&L);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Transport-velocity formulation (Sec. 2.3 names it and cites the       */
/* generalized TVF of Zhang, Hu & Adams (2017) without a formula).       */
/* Reading: particles are carried by the transport velocity v + dv,      */
/* dv = -(2 p_b / rho) dt sum_j V_j grad_i W_ij (the background-pressure */
/* term of the transport-velocity SPH of Adami, Hu & Adams 2013), and    */
/* with the background pressure tied to the step so that p_b dt^2 / rho  */
/* = alpha h^2, the displacement it adds over one advection step is      */
/*   dr_i = -2 alpha h^2 sum_j V_j grad_i W_ij                          */
/* over all real and wall neighbours of the frozen configuration, taken  */
/* once per advection step (before the sub-steps), for fluid particles   */
/* (label 0), and with tvf_pbuf for particles labelled in a pressure     */
/* buffer too.  A pressure buffer fixes the pressure, not the motion:    */
/* its particles move under the momentum equation like fluid particles   */
/* and can crowd like them, but their support is cut at the open face,   */
/* so the sum points into the fluid; only its part across the buffer     */
/* axis n_b is taken (dr - (dr . n_b) n_b), which leaves the flux        */
/* through the face to the momentum equation.  Velocity-buffer particles */
/* keep the motion their prescribed velocity gives them.  grad_i W       */
/* points from i towards j, so a particle is moved away from where its   */
/* neighbours crowd.  The pair geometry of the step stays that of the    */
/* frozen configuration; the shift takes effect at the next rebuild and  */
/* in the buffer update.                                                 */
/* ------------------------------------------------------------------ */
static int orc_transport_impl(const orc_config *c, orc_state *s, const nblist *Lp) {
  const nblist L = *Lp;
  if (!(c->tvf_alpha > 0.0)) return ORC_OK;
  double Vw = wall_volume(c);
  double f = -2.0 * c->tvf_alpha * c->h * c->h;
  #pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < s->n; ++i) {
    int pb = c->tvf_pbuf && is_pressure_buffer(s, s->label[i]);
    if (s->dead[i] || (s->label[i] != 0 && !pb)) continue;
    double S[3] = {0, 0, 0};
    for (int64_t t = L.start[i]; t < L.start[i + 1]; ++t) {
      int64_t j = L.nb[t].j;
      int wall = L.nb[t].wall;
      geom_t G;
      pair_geom(c, &s->pos0[3 * i], xj_of(s, j, wall), &G);
      double V = wall ? Vw : vol_of(s, j);
      for (int a = 0; a < 3; ++a) S[a] += V * G.gw[a];
    }
    if (pb) {
      const double *nb = s->buf[s->label[i] - 1].frame;
      double sn = dotd(c->dim, S, nb);
      for (int a = 0; a < c->dim; ++a) S[a] -= sn * nb[a];
    }
    for (int a = 0; a < c->dim; ++a) s->pos[3 * i + a] += f * S[a];
  }
  return ORC_OK;
}

int orc_transport(const orc_config *c, orc_state *s) {
  nblist L;
  if (build_pairs(c, s, &L)) return ORC_ERR_NOMEM;
  int rc = orc_transport_impl(c, s, &L);
  nblist_free(&L);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Density reinitialisation (dual-criteria time stepping, Sec. 2.3: the  */
/* scheme it cites re-evaluates the density from the particle            */
/* configuration once per advection step; the acoustic sub-steps then    */
/* integrate the Riemann continuity equation of Sec. 2.2).  Reading: for  */
/* fluid particles (label 0) the density becomes                        */
/*   rho_i = rho0 sigma_i / sigma_0,  sigma_i = W(0) + sum_j W_ij        */
/* over all real and wall neighbours of the frozen configuration, with   */
/* sigma_0 the same sum on the perfect lattice of spacing dp, so that an */
/* undisturbed lattice has rho0 exactly.  Buffer particles keep their   */
/* values (their boundary condition sets or extrapolates them).  It is  */
/* taken after the correction matrix, viscous, k-epsilon and transport   */
/* terms of the step, which use the volumes m / rho from before it.      */
/* ------------------------------------------------------------------ */
int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

double orc_lattice_kernel_sum(const orc_config *c) {
  int R = (int)ceil(2.0 * c->h / c->dp) + 1;
  int Rz = c->dim == 3 ? R : 0;
  double S = 0.0;
  for (int a = -R; a <= R; ++a)
    for (int b = -R; b <= R; ++b)
      for (int k = -Rz; k <= Rz; ++k) {
        double r = c->dp * sqrt((double)(a * a + b * b + k * k));
        S += orc_W(c->dim, c->h, r);
      }
  return S;
}

static int orc_density_sum_impl(const orc_config *c, orc_state *s, const nblist *Lp) {
  const nblist L = *Lp;
  if (!c->density_sum) return ORC_OK;
  double sigma0 = orc_lattice_kernel_sum(c);
  double *rs = (double *)malloc((size_t)(s->n > 0 ? s->n : 1) * sizeof(double));
  if (!rs) return ORC_ERR_NOMEM;
  #pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < s->n; ++i) {
    rs[i] = s->rho[i];
    if (s->dead[i] || s->label[i] != 0) continue;
    double sigma = orc_W(c->dim, c->h, 0.0);
    for (int64_t t = L.start[i]; t < L.start[i + 1]; ++t) {
      geom_t G;
      pair_geom(c, &s->pos0[3 * i], xj_of(s, L.nb[t].j, L.nb[t].wall), &G);
      sigma += orc_W(c->dim, c->h, G.rl);
    }
    rs[i] = c->rho0 * sigma / sigma0;
  }
  for (int64_t i = 0; i < s->n; ++i) s->rho[i] = rs[i];
  free(rs);
  return ORC_OK;
}

int orc_density_sum(const orc_config *c, orc_state *s) {
  nblist L;
  if (build_pairs(c, s, &L)) return ORC_ERR_NOMEM;
  int rc = orc_density_sum_impl(c, s, &L);
  nblist_free(&L);
  return rc;
}

/* ------------------------------------------------------------------ */
/* a7: k-epsilon sweep (Sec. 2.1, 2.2; App. A), explicit Euler over the */
/* advection step with floors 1e-12, then nu_t = C_mu k^2 / eps.        */
/*   grad v_i = -sum_j v_ij (x) (B_i grad_i W_ij) V_j, (a,b) = dv_a/dx_b */
/*     (sign fixed so that a linear field is reproduced)                */
/*   G_k = tau_t : grad v, tau_t = nu_t (grad v + grad v^T) - 2k I / 3   */
/*   dk/dt = G_k - eps + (2/rho_i) sum_j rho0 harm(D_k) k_ij f_ij V_j    */
/*   deps/dt = C1 eps/k G_k - C2 eps^2/k + same with D_eps              */
/*   f_ij = dW/(r + 0.01h); D_k = nu_l + nu_t/sigma_k, D_eps likewise.   */
/* Walls: v_j = 2 v_wall - v_i in grad v (no-slip on the wall surface,  */
/* as in the viscous term); no diffusion across walls (zero              */
/* gradient); with wall_fn the step-wise wall function (near_wall)       */
/* replaces the production and eps of the first fluid layer.             */
/* Pinned: homogeneous decay against its closed form; one step under     */
/* linear velocity fields (shear, rotation, strain, dilatation) against  */
/* the textbook production in both equations; diffusion conserves        */
/* sum m k, dissipates sum m k^2 and damps a sine mode at its rate.      */
/* Parity unpinned: the zero-gradient wall treatment of k and eps        */
/* without the wall function (checked by conservation only).             */
/* ------------------------------------------------------------------ */
static int orc_rans_impl(const orc_config *c, orc_state *s, double dt, const nblist *Lp) {
  const nblist L = *Lp;
  double Vw = wall_volume(c);
  int64_t n = s->n;
  double *kn = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  double *en = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  if (!kn || !en) {
    free(kn);
    free(en);
    return ORC_ERR_NOMEM;
  }
  int dim = c->dim;
  #pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    kn[i] = s->k[i];
    en[i] = s->eps[i];
    if (s->dead[i]) continue;
    const double *xi = &s->pos0[3 * i];
    const double *vi = &s->vel[3 * i];
    const double *Bi = &s->B[9 * i];
    double Dk_i = c->nu_l + s->nut[i] / KE_SIGMA_K;
    double De_i = c->nu_l + s->nut[i] / KE_SIGMA_E;
    double S[9] = {0};
    double dk = 0.0, de = 0.0;
    for (int64_t t = L.start[i]; t < L.start[i + 1]; ++t) {
      int64_t j = L.nb[t].j;
      int wall = L.nb[t].wall;
      geom_t G;
      pair_geom(c, xi, xj_of(s, j, wall), &G);
      double V = wall ? Vw : vol_of(s, j);
      double bg[3], vij[3] = {0, 0, 0};
      matvec(dim, Bi, G.gw, bg);
      for (int a = 0; a < dim; ++a) {
        double vj = wall ? 2.0 * s->wvel[3 * j + a] - vi[a] : s->vel[3 * j + a];
        vij[a] = vi[a] - vj;
      }
      for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b) S[3 * a + b] += vij[a] * bg[b] * V;
      if (!wall) {
        double Dk_j = c->nu_l + s->nut[j] / KE_SIGMA_K;
        double De_j = c->nu_l + s->nut[j] / KE_SIGMA_E;
        double Dk = 2.0 * Dk_i * Dk_j / (Dk_i + Dk_j);
        double De = 2.0 * De_i * De_j / (De_i + De_j);
        double f = (G.dw / (G.rl + 0.01 * c->h)) * V;
        dk += c->rho0 * Dk * (s->k[i] - s->k[j]) * f;
        de += c->rho0 * De * (s->eps[i] - s->eps[j]) * f;
      }
    }
    double *gv = &s->gradv[9 * i];
    for (int k = 0; k < 9; ++k) gv[k] = -S[k];
    double ki = s->k[i], ei = s->eps[i];
    double prod = 0.0, tr = 0.0;
    for (int a = 0; a < dim; ++a) {
      tr += gv[4 * a];
      for (int b = 0; b < dim; ++b) prod += (gv[3 * a + b] + gv[3 * b + a]) * gv[3 * a + b];
    }
    double Gk = s->nut[i] * prod - (2.0 / 3.0) * ki * tr;
    nearwall_t nw;
    near_wall(c, s, &L, i, &nw);
    if (nw.on) Gk = nw.log_layer ? nw.utau * nw.utau * nw.utau / (WF_KAPPA * nw.y) : 0.0;
    double dkdt = Gk - ei + 2.0 * dk / s->rho[i];
    double dedt = KE_C1 * (ei / ki) * Gk - KE_C2 * ei * ei / ki + 2.0 * de / s->rho[i];
    double k1 = ki + dt * dkdt;
    double e1 = ei + dt * dedt;
    kn[i] = k1 > KE_FLOOR ? k1 : KE_FLOOR;
    en[i] = e1 > KE_FLOOR ? e1 : KE_FLOOR;
    if (nw.on) {
      /* the wall value of eps from the updated k */
      double kk = kn[i];
      double ew = nw.log_layer ? pow(KE_CMU, 0.75) * (kk * sqrt(kk)) / (WF_KAPPA * nw.y)
                               : 2.0 * c->nu_l * kk / (nw.y * nw.y);
      en[i] = ew > KE_FLOOR ? ew : KE_FLOOR;
    }
  }
  #pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    if (s->dead[i]) continue;
    s->k[i] = kn[i];
    s->eps[i] = en[i];
    s->nut[i] = KE_CMU * kn[i] * kn[i] / en[i];
  }
  free(kn);
  free(en);
  return ORC_OK;
}

int orc_rans(const orc_config *c, orc_state *s, double dt) {
  if (!c->rans) return ORC_OK;
  nblist L;
  if (build_pairs(c, s, &L)) return ORC_ERR_NOMEM;
  int rc = orc_rans_impl(c, s, dt, &L);
  nblist_free(&L);
  return rc;
}

/* ------------------------------------------------------------------ */
/* a8: first half of an acoustic sub-step (Sec. 2.3): rho += dt/2 drho,  */
/* p from the stiff EOS p = rho0 c0^2 (rho/rho0 - 1) (Sec. 2.1),         */
/* x += dt/2 v.                                                         */
/* ------------------------------------------------------------------ */
int orc_half1(const orc_config *c, orc_state *s, double dt) {
  #pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < s->n; ++i) {
    if (s->dead[i]) continue;
    s->rho[i] += 0.5 * dt * s->drho[i];
    s->p[i] = eos(c, s->rho[i]);
    for (int a = 0; a < c->dim; ++a) s->pos[3 * i + a] += 0.5 * dt * s->vel[3 * i + a];
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* a9: pressure acceleration, reverse kernel gradient correction        */
/* (Sec. 2.2):  a_i = -(1/rho_i) sum_j V_j (p_i B^_j + p_j B_i) grad_i W */
/* with p the effective pressure p + 2/3 rho k in RANS (Table 1).        */
/* B^_j = B_i for wall dummies and pressure-buffer particles (the       */
/* condition B_k = B_i of Sec. 3.3), else B_j.                         */
/* Wall dummy: p_j = p_i (Riemann wall condition without gravity,       */
/* Sec. 2.3).                                                           */
/* Pressure-buffer particle (compensated term, final Eq. of Sec. 3.3):  */
/*   a_i += (2 p_ob / rho_i) B_i sum_j V_j grad_i W_ij                  */
/* over all real and wall neighbours, with p_ob + 2/3 rho_i k_i in RANS. */
/* The ablation cases of Sec. 4.1 drop B_i there (comp_B = 0) or take   */
/* B^_j = B_j at buffer neighbours (bhat_buffer = 0).                   */
/* ------------------------------------------------------------------ */
static double p_eff(const orc_config *c, const orc_state *s, int64_t i) {
  return c->rans ? s->p[i] + (2.0 / 3.0) * s->rho[i] * s->k[i] : s->p[i];
}

static int orc_momentum_impl(const orc_config *c, orc_state *s, const nblist *Lp) {
  const nblist L = *Lp;
  double Vw = wall_volume(c);
  int dim = c->dim;
  #pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < s->n; ++i) {
    if (s->dead[i]) continue;
    const double *xi = &s->pos0[3 * i];
    const double *Bi = &s->B[9 * i];
    double pi = p_eff(c, s, i);
    double S[3] = {0, 0, 0};
    double C[3] = {0, 0, 0};
    for (int64_t t = L.start[i]; t < L.start[i + 1]; ++t) {
      int64_t j = L.nb[t].j;
      int wall = L.nb[t].wall;
      geom_t G;
      pair_geom(c, xi, xj_of(s, j, wall), &G);
      double V, pj;
      const double *Bj;
      if (wall) {
        V = Vw;
        pj = pi;
        Bj = Bi;
      } else {
        V = vol_of(s, j);
        pj = p_eff(c, s, j);
        Bj = (c->bhat_buffer && is_pressure_buffer(s, s->label[j])) ? Bi : &s->B[9 * j];
      }
      double bj[3], bi[3];
      matvec(dim, Bj, G.gw, bj);
      matvec(dim, Bi, G.gw, bi);
      for (int a = 0; a < dim; ++a) S[a] += V * (pi * bj[a] + pj * bi[a]);
      for (int a = 0; a < dim; ++a) C[a] += V * G.gw[a];
    }
    double *acc = &s->acc_p[3 * i];
    for (int a = 0; a < 3; ++a) acc[a] = (a < dim) ? -S[a] / s->rho[i] : 0.0;
    if (c->compensation && is_pressure_buffer(s, s->label[i])) {
      double pob = s->buf[s->label[i] - 1].p_ob;
      if (c->rans) pob += (2.0 / 3.0) * s->rho[i] * s->k[i];
      double bc[3] = {C[0], C[1], C[2]};
      if (c->comp_B) matvec(dim, Bi, C, bc);
      for (int a = 0; a < dim; ++a) acc[a] += 2.0 * pob / s->rho[i] * bc[a];
    }
  }
  return ORC_OK;
}

int orc_momentum(const orc_config *c, orc_state *s) {
  nblist L;
  if (build_pairs(c, s, &L)) return ORC_ERR_NOMEM;
  int rc = orc_momentum_impl(c, s, &L);
  nblist_free(&L);
  return rc;
}

/* v += dt (a_p + a_nu + g); x += dt/2 v  (Eq. of the general momentum
   discretisation, Sec. 2.2; Verlet half, Sec. 2.3) */
int orc_kick(const orc_config *c, orc_state *s, double dt) {
  #pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < s->n; ++i) {
    if (s->dead[i]) continue;
    for (int a = 0; a < c->dim; ++a) {
      s->vel[3 * i + a] += dt * (s->acc_p[3 * i + a] + s->acc_nu[3 * i + a] + c->g[a]);
      s->pos[3 * i + a] += 0.5 * dt * s->vel[3 * i + a];
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* a10: Riemann-based continuity (Sec. 2.2):                            */
/*   drho_i/dt = 2 rho_i sum_j (v_i - v*) . grad_i W_ij V_j,             */
/*   v* = U* e_ij + (vbar_ij - Ubar_ij e_ij), Ubar = vbar . e_ij,        */
/*   U* = Ubar + (p_i - p_j) / (2 rho0 c0),                             */
/* e_ij the unit vector from i to j, p the EOS                          */
/* pressure.  Wall dummy: v_j = 2 v_wall - v_i (so vbar = v_wall) and    */
/* p_j = p_i.                                                           */
/* ------------------------------------------------------------------ */
static int orc_continuity_impl(const orc_config *c, orc_state *s, const nblist *Lp) {
  const nblist L = *Lp;
  double Vw = wall_volume(c);
  int dim = c->dim;
  #pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < s->n; ++i) {
    if (s->dead[i]) continue;
    const double *xi = &s->pos0[3 * i];
    const double *vi = &s->vel[3 * i];
    double pi = s->p[i];
    double sum = 0.0;
    for (int64_t t = L.start[i]; t < L.start[i + 1]; ++t) {
      int64_t j = L.nb[t].j;
      int wall = L.nb[t].wall;
      geom_t G;
      pair_geom(c, xi, xj_of(s, j, wall), &G);
      double vj[3] = {0, 0, 0}, pj, V;
      if (wall) {
        for (int a = 0; a < dim; ++a) vj[a] = 2.0 * s->wvel[3 * j + a] - vi[a];
        pj = pi;
        V = Vw;
      } else {
        for (int a = 0; a < dim; ++a) vj[a] = s->vel[3 * j + a];
        pj = s->p[j];
        V = vol_of(s, j);
      }
      double e[3] = {0, 0, 0}, vbar[3] = {0, 0, 0};
      for (int a = 0; a < dim; ++a) {
        e[a] = -G.r[a] / G.rl;
        vbar[a] = 0.5 * (vi[a] + vj[a]);
      }
      double Ubar = dotd(dim, vbar, e);
      double Ustar = Ubar + (pi - pj) / (2.0 * c->rho0 * c->c0);
      double w[3] = {0, 0, 0};
      for (int a = 0; a < dim; ++a) {
        double vstar = Ustar * e[a] + (vbar[a] - Ubar * e[a]);
        w[a] = vi[a] - vstar;
      }
      sum += dotd(dim, w, G.gw) * V;
    }
    s->drho[i] = 2.0 * s->rho[i] * sum;
  }
  return ORC_OK;
}

int orc_continuity(const orc_config *c, orc_state *s) {
  nblist L;
  if (build_pairs(c, s, &L)) return ORC_ERR_NOMEM;
  int rc = orc_continuity_impl(c, s, &L);
  nblist_free(&L);
  return rc;
}

int orc_density(const orc_config *c, orc_state *s, double dt) {
  (void)c;
  #pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < s->n; ++i) {
    if (s->dead[i]) continue;
    s->rho[i] += 0.5 * dt * s->drho[i];
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* a11: boundary values on buffer particles (Sec. 2.4.2; buffer BC      */
/* table of Sec. 4.3).                                                  */
/* Velocity buffer: v = U(s) n_b + a U(s) xi, s = x'_1, U interpolated  */
/* linearly in theta over [-half0, half0], a the noise amplitude and xi */
/* in [-1,1)^d from Philox4x32-10 keyed by (seed, uid) with counter      */
/* (step, sub, 0|1, 0).  Pressure and density are extrapolated (kept). */
/* Pressure buffer: p = p_ob, rho = rho0 (1 + p_ob / (rho0 c0^2));       */
/* velocity extrapolated (kept).                                         */
/* Turbulence: freestream sets (k_in, eps_in) and nu_t; zero gradient    */
/* keeps the particle's own values.                                      */
/* ------------------------------------------------------------------ */
static double profile_U(const orc_buffer *b, double s1) {
  if (b->n_theta <= 1) return b->theta[0];
  double w = b->half[0];
  double u = (s1 + w) / (2.0 * w) * (double)(b->n_theta - 1);
  if (!(u > 0.0)) return b->theta[0];
  if (u >= (double)(b->n_theta - 1)) return b->theta[b->n_theta - 1];
  int k = (int)floor(u);
  double f = u - (double)k;
  return b->theta[k] + f * (b->theta[k + 1] - b->theta[k]);
}

static void apply_bc_one(const orc_config *c, orc_state *s, int64_t i, int64_t step, uint32_t sub) {
  const orc_buffer *b = &s->buf[s->label[i] - 1];
  if (b->type == ORC_BUF_VELOCITY) {
    double s1 = local_coord(c, b, &s->pos[3 * i], 1);
    double U = profile_U(b, s1);
    double xi[3] = {0, 0, 0};
    if (b->noise != 0.0) {
      uint32_t key[2] = {c->seed, s->uid[i]};
      uint32_t ctr[4] = {(uint32_t)step, sub, 0u, 0u};
      uint32_t o[4];
      orc_philox4x32_10(ctr, key, o);
      xi[0] = orc_uniform_pm1(o[0], o[1]);
      xi[1] = orc_uniform_pm1(o[2], o[3]);
      if (c->dim == 3) {
        ctr[2] = 1u;
        orc_philox4x32_10(ctr, key, o);
        xi[2] = orc_uniform_pm1(o[0], o[1]);
      }
    }
    for (int a = 0; a < c->dim; ++a) s->vel[3 * i + a] = U * b->frame[a] + b->noise * U * xi[a];
  } else {
    s->p[i] = b->p_ob;
    s->rho[i] = c->rho0 * (1.0 + b->p_ob / (c->rho0 * c->c0 * c->c0));
  }
  if (c->rans && !c->freeze_turb && b->turb_bc == ORC_TURB_FREESTREAM) {
    s->k[i] = b->k_in;
    s->eps[i] = b->eps_in;
    s->nut[i] = KE_CMU * b->k_in * b->k_in / b->eps_in;
  }
}

int orc_apply_bc(const orc_config *c, orc_state *s, int64_t step, uint32_t sub) {
  #pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < s->n; ++i) {
    if (s->dead[i]) continue;
    if (s->label[i] > 0 && s->label[i] <= s->nbuf) apply_bc_one(c, s, i, step, sub);
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* a12 + a13: buffer update at the end of the advection step.          */
/* Injection (Sec. 2.4.2 with the generation line of Sec. 3.1): a       */
/* particle labelled b+1 whose x'_0 >= L_b + 0.5 dp (it has crossed the */
/* generation line and its identity is 'buffer') spawns a fluid copy at */
/* its position that inherits every field (label 0, new uid), and is    */
/* recycled to r - L_b n_b with the buffer's boundary values.  Copies   */
/* are appended at the end of the array in index order.                 */
/* Deletion (Sec. 2.4.3 with the ID check of Sec. 3.2): a particle      */
/* labelled b+1 with x'_0 < 0 is deleted; only the buffer whose ID the   */
/* particle carries can delete it.  id_check = 0 (ablation): any buffer  */
/* particle in buffer c's local cells with x'_0(c) < 0 is deleted.       */
/* Capacity overflow returns ORC_ERR_CAPACITY and changes nothing.       */
/* ------------------------------------------------------------------ */
static void copy_particle(orc_state *s, int64_t dst, int64_t src) {
  memcpy(&s->pos[3 * dst], &s->pos[3 * src], 3 * sizeof(double));
  memcpy(&s->vel[3 * dst], &s->vel[3 * src], 3 * sizeof(double));
  s->rho[dst] = s->rho[src];
  s->mass[dst] = s->mass[src];
  s->drho[dst] = s->drho[src];
  s->k[dst] = s->k[src];
  s->eps[dst] = s->eps[src];
  s->nut[dst] = s->nut[src];
  s->p[dst] = s->p[src];
  s->label[dst] = s->label[src];
  s->uid[dst] = s->uid[src];
  s->dead[dst] = 0;
}

int orc_buffer_update(const orc_config *c, orc_state *s, int64_t step) {
  int64_t n_old = s->n;
  int64_t nspawn = 0;
  /* first pass: count spawns for the capacity check */
  for (int64_t i = 0; i < n_old; ++i) {
    int32_t l = s->label[i];
    if (s->dead[i] || l <= 0 || l > s->nbuf) continue;
    const orc_buffer *b = &s->buf[l - 1];
    if (local_coord(c, b, &s->pos[3 * i], 0) >= b->length + c->gen_offset * c->dp) ++nspawn;
  }
  if (n_old + nspawn > s->cap) return ORC_ERR_CAPACITY;
  int64_t rank = 0, ndel = 0;
  for (int64_t i = 0; i < n_old; ++i) {
    int32_t l = s->label[i];
    if (s->dead[i] || l <= 0 || l > s->nbuf) continue;
    const orc_buffer *b = &s->buf[l - 1];
    double s0 = local_coord(c, b, &s->pos[3 * i], 0);
    if (s0 >= b->length + c->gen_offset * c->dp) {
      int64_t d = n_old + rank;
      copy_particle(s, d, i);
      s->label[d] = 0;
      s->uid[d] = s->next_uid + (uint32_t)rank;
      for (int a = 0; a < c->dim; ++a) s->pos[3 * i + a] -= b->length * b->frame[a];
      apply_bc_one(c, s, i, step, SUB_RECYCLE);
      ++rank;
    } else if (c->id_check && s0 < 0.0) {
      s->dead[i] = 1;
      ++ndel;
    }
  }
  if (!c->id_check) {
    for (int64_t i = 0; i < n_old; ++i) {
      if (s->dead[i] || s->label[i] <= 0) continue;
      for (int b = 0; b < s->nbuf; ++b) {
        const orc_buffer *B = &s->buf[b];
        if (in_local_cells(c, B, &s->pos[3 * i]) && local_coord(c, B, &s->pos[3 * i], 0) < 0.0) {
          s->dead[i] = 1;
          ++ndel;
          break;
        }
      }
    }
  }
  s->n = n_old + rank;
  s->next_uid += (uint32_t)rank;
  s->n_spawned += rank;
  s->n_deleted += ndel;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* One advection step, in this order:                                   */
/* commit + sort, label, dt, frozen configuration, B, viscous, RANS,     */
/* acoustic sub-steps (half1, momentum, kick, continuity, density, BC),  */
/* buffer update.                                                       */
/* ------------------------------------------------------------------ */
int orc_step(const orc_config *c, orc_state *s, int nsteps) {
  for (int st = 0; st < nsteps; ++st) {
    int rc;
    if ((rc = orc_compact_sort(c, s))) return rc;
    if ((rc = orc_label(c, s))) return rc;
    if ((rc = orc_configure(c, s))) return rc;
    if ((rc = orc_time_step(c, s))) return rc;
    nblist L;
    if (build_pairs(c, s, &L)) return ORC_ERR_NOMEM;
    rc = orc_bmatrix_impl(c, s, NULL, &L);
    if (!rc) rc = orc_viscous_impl(c, s, &L);
    if (!rc && c->rans && !c->freeze_turb) rc = orc_rans_impl(c, s, s->dt_ad, &L);
    if (!rc) rc = orc_transport_impl(c, s, &L);
    if (!rc) rc = orc_density_sum_impl(c, s, &L);
    for (int sub = 0; sub < s->n_ac && !rc; ++sub) {
      double dt = s->dt;
      rc = orc_half1(c, s, dt);
      if (!rc) rc = orc_momentum_impl(c, s, &L);
      if (!rc) rc = orc_kick(c, s, dt);
      if (!rc) rc = orc_continuity_impl(c, s, &L);
      if (!rc) rc = orc_density(c, s, dt);
      if (!rc) rc = orc_apply_bc(c, s, s->step, (uint32_t)sub);
    }
    nblist_free(&L);
    if (rc) return rc;
    if ((rc = orc_buffer_update(c, s, s->step))) return rc;
    s->step += 1;
    s->t += s->dt_ad;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* pins                                                                 */
/* ------------------------------------------------------------------ */
int orc_kernel_gradient_sum(const orc_config *c, const orc_state *s, double *out) {
  nblist L;
  if (build_pairs(c, s, &L)) return ORC_ERR_NOMEM;
  double Vw = wall_volume(c);
  for (int64_t i = 0; i < s->n; ++i) {
    double S[3] = {0, 0, 0};
    for (int64_t t = L.start[i]; t < L.start[i + 1]; ++t) {
      int64_t j = L.nb[t].j;
      int wall = L.nb[t].wall;
      geom_t G;
      pair_geom(c, &s->pos0[3 * i], xj_of(s, j, wall), &G);
      double V = wall ? Vw : vol_of(s, j);
      for (int a = 0; a < 3; ++a) S[a] += V * G.gw[a];
    }
    memcpy(&out[3 * i], S, sizeof(S));
  }
  nblist_free(&L);
  return ORC_OK;
}

int orc_kernel_sum(const orc_config *c, const orc_state *s, double *out) {
  nblist L;
  if (build_pairs(c, s, &L)) return ORC_ERR_NOMEM;
  double Vw = wall_volume(c);
  for (int64_t i = 0; i < s->n; ++i) {
    double S = orc_W(c->dim, c->h, 0.0) * vol_of(s, i);
    for (int64_t t = L.start[i]; t < L.start[i + 1]; ++t) {
      int64_t j = L.nb[t].j;
      int wall = L.nb[t].wall;
      geom_t G;
      pair_geom(c, &s->pos0[3 * i], xj_of(s, j, wall), &G);
      S += orc_W(c->dim, c->h, G.rl) * (wall ? Vw : vol_of(s, j));
    }
    out[i] = S;
  }
  nblist_free(&L);
  return ORC_OK;
}
