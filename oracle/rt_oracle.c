/*
 * rt_oracle.c -- FP64 CPU oracle (test infrastructure only; see rt_oracle.h).
 *
 * A plain restatement of the Monte Carlo formal solution on a hierarchical
 * grid (Lunttila & Juvela, Sect. 2) in double precision, global (root-cell)
 * coordinates and one packet at a time:
 *   - the tree is a pointer octree built from the level-ordered description
 *     (Sect. 2.1: a grid hierarchy whose refined cells are replaced by 2x2x2
 *     subcells; every crossing looks up the leaf by descending from the
 *     root, the role of the subgrid identification array of Sect. 2.1);
 *   - packages carry a photon weight that decays by continuous absorption
 *     (Sect. 2.3, Lucy 1999) and are removed only at the outer boundary of
 *     the root grid or by Russian roulette (Sect. 2.3);
 *   - scattered light is peeled off towards observers after every scattering
 *     (Sect. 2.4, Yusef-Zadeh et al. 1984); optionally with Sect. 2.4's
 *     accelerated variant: the optical depth is followed exactly only to the
 *     boundary of the scattering point's block of root cells, and the rest
 *     is a column density tabulated from the centre of the face tile the ray
 *     leaves through to the model border;
 *   - dust temperatures follow from the equilibrium between absorbed and
 *     emitted energy (Sects. 3.2 and 4: a single dust component in
 *     equilibrium with the local radiation field).
 * Random numbers come from Philox4x32-10 (Salmon et al. 2011), implemented
 * here from the published definition; the stream layout is:
 *   key     = (seed_lo ^ job, seed_hi ^ iter)
 *   counter = (pkt_lo, pkt_hi, draw >> 2, stream),  word = draw & 3
 *   stream  = (source << 16) | wavelength bin
 *   uniform = (u32 + 0.5) * 2^-32
 */
#include "rt_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
#define C_CGS 2.99792458e10
#define H_CGS 6.62607015e-27
#define K_CGS 1.380649e-16

/* ------------------------------------------------------------------------ */
/* Philox (Salmon, Moraes, Dror, Shaw 2011): an S-P network of 10 rounds.   */
/* Each round multiplies words 0 and 2 by fixed odd constants, and forms    */
/* the new block from the high/low halves xor'ed with the other words and   */
/* the round key; the key is bumped by the Weyl constants between rounds.   */
/* One macro text instantiates both word widths.                            */
/* ------------------------------------------------------------------------ */
static inline void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}
static inline void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}

#define ORC_PHILOX_DEF(NAME, T, MULHILO, M0, M1, W0, W1)                 \
  void NAME(const T ctr[4], const T key[2], T out[4]) {                 \
    T x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];               \
    T k0 = key[0], k1 = key[1];                                          \
    for (int r = 0; r < 10; ++r) {                                       \
      if (r > 0) { k0 += (T)(W0); k1 += (T)(W1); }                       \
      T hi0, lo0, hi1, lo1;                                              \
      MULHILO((T)(M0), x0, &hi0, &lo0);                                  \
      MULHILO((T)(M1), x2, &hi1, &lo1);                                  \
      T y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;      \
      x0 = y0; x1 = y1; x2 = y2; x3 = y3;                                \
    }                                                                    \
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;                  \
  }

ORC_PHILOX_DEF(orc_philox4x32, uint32_t, mulhilo32, 0xD2511F53u, 0xCD9E8D57u,
               0x9E3779B9u, 0xBB67AE85u)
ORC_PHILOX_DEF(orc_philox4x64, uint64_t, mulhilo64, 0xD2E7470EE14C6C93ull,
               0xCA5A826395121157ull, 0x9E3779B97F4A7C15ull, 0xBB67AE8584CAA73Bull)

uint32_t orc_draw_u32(uint64_t seed, uint32_t job, uint32_t iter, uint32_t stream,
                      uint64_t pkt, uint64_t j) {
  uint32_t key[2] = {(uint32_t)seed ^ job, (uint32_t)(seed >> 32) ^ iter};
  uint32_t ctr[4] = {(uint32_t)pkt, (uint32_t)(pkt >> 32), (uint32_t)(j >> 2), stream};
  uint32_t out[4];
  orc_philox4x32(ctr, key, out);
  return out[j & 3];
}

typedef struct {
  uint64_t seed, pkt, next;
  uint32_t job, iter, stream;
} rstream;

static double uni(rstream* s) {
  uint32_t x = orc_draw_u32(s->seed, s->job, s->iter, s->stream, s->pkt, s->next++);
  return ((double)x + 0.5) * (1.0 / 4294967296.0);
}

/* ------------------------------------------------------------------------ */
/* Tree                                                                       */
/* ------------------------------------------------------------------------ */
typedef struct orc_node {
  int64_t id;
  int level;
  double lo[3];    /* root-cell units */
  double size;     /* 2^-level */
  double rho;      /* g/cm^3 */
  struct orc_node* child;  /* first of 8 children (octant ox+2oy+4oz), NULL for a leaf */
} orc_node;

struct orc_tree {
  int root[3];
  double box[3];
  double h0;
  int n_levels;
  int64_t n_cells;
  orc_node* nodes;
};

orc_tree* orc_tree_build(const orc_tree_desc* d) {
  if (!d || d->root[0] <= 0 || d->root[1] <= 0 || d->root[2] <= 0 || d->n_levels <= 0) return NULL;
  double h0 = d->box[0] / d->root[0];
  for (int a = 1; a < 3; ++a)
    if (fabs(d->box[a] / d->root[a] - h0) > 1e-12 * h0) return NULL;
  int64_t n0 = (int64_t)d->root[0] * d->root[1] * d->root[2];
  int64_t total = n0, level_n = n0;
  for (int l = 0; l < d->n_levels; ++l) {
    if (d->n_refined[l] < 0 || d->n_refined[l] > level_n) return NULL;
    if (l == d->n_levels - 1 && d->n_refined[l] != 0) return NULL;
    level_n = 8 * d->n_refined[l];
    total += level_n;
  }
  total -= level_n;  /* last level has no children */
  orc_tree* t = (orc_tree*)calloc(1, sizeof(orc_tree));
  t->nodes = (orc_node*)calloc((size_t)total, sizeof(orc_node));
  memcpy(t->root, d->root, sizeof t->root);
  memcpy(t->box, d->box, sizeof t->box);
  t->h0 = h0;
  t->n_levels = d->n_levels;
  t->n_cells = total;
  /* root grid, x fastest */
  for (int iz = 0; iz < d->root[2]; ++iz)
    for (int iy = 0; iy < d->root[1]; ++iy)
      for (int ix = 0; ix < d->root[0]; ++ix) {
        int64_t id = ix + (int64_t)d->root[0] * (iy + (int64_t)d->root[1] * iz);
        orc_node* n = &t->nodes[id];
        n->id = id; n->level = 0; n->size = 1.0;
        n->lo[0] = ix; n->lo[1] = iy; n->lo[2] = iz;
      }
  /* breadth-first: the k-th refined cell (in level order) owns cells n0+8k..n0+8k+7 */
  int64_t next_child = n0, refined_seen = 0;
  int64_t lvl_begin = 0, lvl_end = n0;
  for (int l = 0; l < d->n_levels; ++l) {
    int64_t cnt = 0;
    for (int64_t id = lvl_begin; id < lvl_end; ++id) {
      orc_node* n = &t->nodes[id];
      n->rho = d->density[id];
      if (d->refine_flags[id]) {
        if (next_child + 8 > total) { orc_tree_free(t); return NULL; }
        n->child = &t->nodes[next_child];
        for (int o = 0; o < 8; ++o) {
          orc_node* c = &n->child[o];
          c->id = next_child + o;
          c->level = l + 1;
          c->size = 0.5 * n->size;
          c->lo[0] = n->lo[0] + ((o >> 0) & 1) * c->size;
          c->lo[1] = n->lo[1] + ((o >> 1) & 1) * c->size;
          c->lo[2] = n->lo[2] + ((o >> 2) & 1) * c->size;
        }
        next_child += 8;
        ++cnt;
        ++refined_seen;
      } else if (!(n->rho >= 0.0) || !isfinite(n->rho)) {
        orc_tree_free(t);
        return NULL;
      }
    }
    if (cnt != d->n_refined[l]) { orc_tree_free(t); return NULL; }
    lvl_begin = lvl_end;
    lvl_end = next_child;
  }
  (void)refined_seen;
  if (next_child != total) { orc_tree_free(t); return NULL; }
  return t;
}

void orc_tree_free(orc_tree* t) {
  if (!t) return;
  free(t->nodes);
  free(t);
}

int64_t orc_tree_ncells(const orc_tree* t) { return t->n_cells; }

void orc_tree_cells(const orc_tree* t, uint8_t* level, uint8_t* is_leaf) {
  for (int64_t i = 0; i < t->n_cells; ++i) {
    if (level) level[i] = (uint8_t)t->nodes[i].level;
    if (is_leaf) is_leaf[i] = t->nodes[i].child == NULL;
  }
}

/* Leaf containing x; a coordinate exactly on a face belongs to the cell the
 * direction points into (d >= 0: upper cell). NULL outside the root grid. */
static const orc_node* locate(const orc_tree* t, const double x[3], const double d[3]) {
  int64_t ic[3];
  for (int a = 0; a < 3; ++a) {
    double f = floor(x[a]);
    int64_t i = (int64_t)f;
    if (x[a] == f && d[a] < 0) i -= 1;
    if (i < 0 || i >= t->root[a]) return NULL;
    ic[a] = i;
  }
  const orc_node* n = &t->nodes[ic[0] + t->root[0] * (ic[1] + (int64_t)t->root[1] * ic[2])];
  while (n->child) {
    int oct = 0;
    for (int a = 0; a < 3; ++a) {
      double mid = n->lo[a] + 0.5 * n->size;
      int upper = (x[a] > mid) || (x[a] == mid && d[a] >= 0);
      oct |= upper << a;
    }
    n = &n->child[oct];
  }
  return n;
}

/* distance (root units) to the exit face of leaf n; lowest axis wins ties */
static double exit_dist(const orc_node* n, const double x[3], const double d[3], int* axis) {
  double best = INFINITY;
  int ab = -1;
  for (int a = 0; a < 3; ++a) {
    double t;
    if (d[a] > 0) t = (n->lo[a] + n->size - x[a]) / d[a];
    else if (d[a] < 0) t = (n->lo[a] - x[a]) / d[a];
    else continue;
    if (t < 0) t = 0;
    if (t < best) { best = t; ab = a; }
  }
  *axis = ab;
  return best;
}

static void move_to_face(const orc_node* n, double x[3], const double d[3], double t, int a) {
  for (int b = 0; b < 3; ++b)
    if (b != a) x[b] += t * d[b];
  x[a] = d[a] > 0 ? n->lo[a] + n->size : n->lo[a];
}

static double face_margin(const orc_node* n, const double x[3], int a) {
  double m = INFINITY;
  for (int b = 0; b < 3; ++b) {
    if (b == a) continue;
    double u = (x[b] - n->lo[b]) / n->size;
    double v = fmin(fabs(u), fabs(1.0 - u));
    if (v < m) m = v;
  }
  return m;
}

int64_t orc_walk(const orc_tree* t, const double origin[3], const double dir[3], int64_t max_seg,
                 int64_t* cells, double* lengths, double* margins) {
  double x[3], d[3];
  for (int a = 0; a < 3; ++a) { x[a] = origin[a] / t->h0; d[a] = dir[a]; }
  const orc_node* n = locate(t, x, d);
  if (!n) return -1;
  int64_t k = 0;
  while (n && k < max_seg) {
    int a;
    double s = exit_dist(n, x, d, &a);
    move_to_face(n, x, d, s, a);
    const orc_node* nn = locate(t, x, d);
    if (s > 0) {
      double m = face_margin(n, x, a);
      if (nn) {
        double m2 = face_margin(nn, x, a);
        if (m2 < m) m = m2;
      }
      cells[k] = n->id;
      lengths[k] = s * t->h0;
      margins[k] = m;
      ++k;
    }
    n = nn;
  }
  return k;
}

/* ------------------------------------------------------------------------ */
/* Scattering                                                                 */
/* ------------------------------------------------------------------------ */
/* Henyey-Greenstein: inverse of the cumulative distribution of mu. */
double orc_hg_mu(double g, double u) {
  double mu;
  if (g == 0.0) {
    mu = 2.0 * u - 1.0;
  } else {
    double s = (1.0 - g * g) / (1.0 - g + 2.0 * g * u);
    mu = (1.0 + g * g - s * s) / (2.0 * g);
  }
  if (mu > 1.0) mu = 1.0;
  if (mu < -1.0) mu = -1.0;
  return mu;
}

double orc_hg_phase(double g, double mu) {
  double den = 1.0 + g * g - 2.0 * g * mu;
  return (1.0 - g * g) / (4.0 * ORC_PI * den * sqrt(den));
}

/* New direction at polar cosine mu and azimuth phi about d (the usual
 * rotation formula of Monte Carlo photon transport). */
void orc_scatter_dir(const double d[3], double mu, double phi, double out[3]) {
  double st = sqrt(fmax(0.0, 1.0 - mu * mu));
  double cp = cos(phi), sp = sin(phi);
  if (fabs(d[2]) > 0.99999) {
    out[0] = st * cp;
    out[1] = st * sp;
    out[2] = d[2] > 0 ? mu : -mu;
  } else {
    double den = sqrt(1.0 - d[2] * d[2]);
    out[0] = st * (d[0] * d[2] * cp - d[1] * sp) / den + d[0] * mu;
    out[1] = st * (d[1] * d[2] * cp + d[0] * sp) / den + d[1] * mu;
    out[2] = -st * cp * den + d[2] * mu;
  }
  double nrm = sqrt(out[0] * out[0] + out[1] * out[1] + out[2] * out[2]);
  out[0] /= nrm; out[1] /= nrm; out[2] /= nrm;
}

static void iso_dir(double u1, double u2, double d[3]) {
  double mu = 2.0 * u1 - 1.0, phi = 2.0 * ORC_PI * u2;
  double st = sqrt(fmax(0.0, 1.0 - mu * mu));
  d[0] = st * cos(phi);
  d[1] = st * sin(phi);
  d[2] = mu;
}

/* ------------------------------------------------------------------------ */
/* Trace                                                                      */
/* ------------------------------------------------------------------------ */
typedef struct {
  const orc_tree* t;
  int n_src;
  const orc_source* src;
  const orc_optics* op;
  const orc_params* prm;
  const orc_observers* obs;
  int bins;
  int64_t n_packets;
  int64_t* seg_begin;      /* [n_src*n_lambda + 1] global packet offset of each (src,bin) */
  int64_t** first;         /* dust: [n_src][n_lambda] -> first package of each cell, [n_cells + 1] */
  double* w_dust;          /* dust: [n_src][n_lambda] energy of one package */
  double* rec;
  int shared_atomic;
  double* absorbed_shared;
  double* images_shared;
  double* peel_tab;        /* accelerated peel-off: orc_peel_table of the observers, or NULL */
} trace_job;

/* One photon-package path: the primary package, or a copy made where a
 * package entered a deeper grid (package splitting, Sect. 2.3). */
typedef struct {
  double x[3], d[3], W, W0, tau;
  rstream rs;
  const orc_node* prev;
  int mlev;  /* shallowest grid level visited (subiterations) */
  int plev;  /* resampling: grid level of the last cell, capped at split_max_level (-1: none yet) */
} orc_path;

typedef struct {
  trace_job* job;
  int64_t p0, p1;
  double* absorbed;
  double* images;
  double* sumsq;
  double* hits;
  double* pkt_acc;
  int64_t* stamp;
  int64_t* touched;
  int64_t n_touched, cap_touched;
  double* img_sumsq;             /* per-pixel sum of squared package contributions, or NULL */
  double* img_acc;               /* the current package's contribution per pixel */
  int64_t* img_stamp;
  int64_t* img_touched;
  int64_t n_img_touched, cap_img_touched;
  int64_t cur_pkt;               /* package being traced (for the per-package image tallies) */
  orc_path* stack;               /* copies waiting to be followed (package splitting) */
  int64_t n_stack, cap_stack;
  orc_ledger led;
} trace_worker;

static void atomic_add_double(double* p, double v) {
  uint64_t* q = (uint64_t*)p;
  uint64_t old = __atomic_load_n(q, __ATOMIC_RELAXED), nw;
  do {
    double cur;
    memcpy(&cur, &old, 8);
    cur += v;
    memcpy(&nw, &cur, 8);
  } while (!__atomic_compare_exchange_n(q, &old, nw, 0, __ATOMIC_RELAXED, __ATOMIC_RELAXED));
}

static void deposit(trace_worker* w, int64_t slot, int64_t pkt, double v) {
  if (v == 0.0) return;
  if (w->job->shared_atomic) atomic_add_double(&w->job->absorbed_shared[slot], v);
  else w->absorbed[slot] += v;
  if (w->pkt_acc) {
    if (w->stamp[slot] != pkt) {
      w->stamp[slot] = pkt;
      w->pkt_acc[slot] = 0.0;
      if (w->n_touched == w->cap_touched) {
        w->cap_touched = w->cap_touched ? 2 * w->cap_touched : 256;
        w->touched = (int64_t*)realloc(w->touched, (size_t)w->cap_touched * sizeof(int64_t));
      }
      w->touched[w->n_touched++] = slot;
    }
    w->pkt_acc[slot] += v;
  }
}

static void flush_packet(trace_worker* w) {
  for (int64_t i = 0; i < w->n_touched; ++i) {
    int64_t s = w->touched[i];
    w->sumsq[s] += w->pkt_acc[s] * w->pkt_acc[s];
    w->hits[s] += 1.0;
  }
  w->n_touched = 0;
  if (w->img_acc) {
    for (int64_t i = 0; i < w->n_img_touched; ++i) {
      int64_t s = w->img_touched[i];
      w->img_sumsq[s] += w->img_acc[s] * w->img_acc[s];
    }
    w->n_img_touched = 0;
  }
}

/* a peel-off contribution c to image pixel `slot` */
static void image_add(trace_worker* w, int64_t slot, double c) {
  if (w->job->shared_atomic) atomic_add_double(&w->job->images_shared[slot], c);
  else w->images[slot] += c;
  if (w->img_acc && c != 0.0) {
    if (w->img_stamp[slot] != w->cur_pkt) {
      w->img_stamp[slot] = w->cur_pkt;
      w->img_acc[slot] = 0.0;
      if (w->n_img_touched == w->cap_img_touched) {
        w->cap_img_touched = w->cap_img_touched ? 2 * w->cap_img_touched : 256;
        w->img_touched = (int64_t*)realloc(w->img_touched, (size_t)w->cap_img_touched * sizeof(int64_t));
      }
      w->img_touched[w->n_img_touched++] = slot;
    }
    w->img_acc[slot] += c;
  }
}

/* Optical depth along x + s k to the root boundary (Sect. 2.4 peel-off). */
static double peel_march(trace_worker* w, const double x0[3], const double k[3], int bin, double tau_max,
                         int* cut) {
  const orc_tree* t = w->job->t;
  double x[3] = {x0[0], x0[1], x0[2]};
  double kext = w->job->op->kappa_ext[bin] * t->h0;
  double tau = 0.0;
  *cut = 0;
  const orc_node* n = locate(t, x, k);
  while (n) {
    int a;
    double s = exit_dist(n, x, k, &a);
    tau += kext * n->rho * s;
    if (s > 0) w->led.n_peel_cross += 1;
    if (tau_max > 0 && tau > tau_max) { *cut = 1; return tau; }
    move_to_face(n, x, k, s, a);
    n = locate(t, x, k);
  }
  return tau;
}

/* ------------------------------------------------------------------------ */
/* Accelerated peel-off (Sect. 2.4): extinction tables on block faces          */
/* ------------------------------------------------------------------------ */
static int blocks_along(const orc_tree* t, int a, int block) { return (t->root[a] + block - 1) / block; }

static int n_axes(const double k[3]) { return (k[0] != 0.0) + (k[1] != 0.0) + (k[2] != 0.0); }

static int axis_slot(const double k[3], int a) {
  int s = 0;
  for (int b = 0; b < a; ++b) s += k[b] != 0.0;
  return s;
}

/* column density (g/cm^3 x root-cell units) from x along k to the border */
static double column_march(const orc_tree* t, const double x0[3], const double k[3]) {
  double x[3] = {x0[0], x0[1], x0[2]};
  double col = 0.0;
  const orc_node* n = locate(t, x, k);
  while (n) {
    int a;
    double s = exit_dist(n, x, k, &a);
    col += n->rho * s;
    move_to_face(n, x, k, s, a);
    n = locate(t, x, k);
  }
  return col;
}

int64_t orc_peel_table(const orc_tree* t, const orc_observers* obs, int block, int tiles, double* out) {
  if (!t || !obs || block < 1 || tiles < 1) return -1;
  const int nb[3] = {blocks_along(t, 0, block), blocks_along(t, 1, block), blocks_along(t, 2, block)};
  const int64_t n_blocks = (int64_t)nb[0] * nb[1] * nb[2];
  int64_t idx = 0;
  for (int o = 0; o < obs->n_obs; ++o) {
    const double* k = &obs->dir[3 * o];
    const int na = n_axes(k);
    for (int64_t blk = 0; blk < n_blocks; ++blk) {
      const int b[3] = {(int)(blk % nb[0]), (int)((blk / nb[0]) % nb[1]), (int)(blk / ((int64_t)nb[0] * nb[1]))};
      for (int a = 0; a < 3; ++a) {
        if (k[a] == 0.0) continue;
        const int a1 = (a + 1) % 3, a2 = (a + 2) % 3;
        for (int iv = 0; iv < tiles; ++iv)
          for (int iu = 0; iu < tiles; ++iu, ++idx) {
            if (!out) continue;
            double c[3];
            c[a] = k[a] > 0 ? fmin((double)(b[a] + 1) * block, (double)t->root[a]) : (double)b[a] * block;
            const double w = (double)block / tiles;
            const double u0 = (double)b[a1] * block + iu * w, v0 = (double)b[a2] * block + iv * w;
            if (u0 >= t->root[a1] || v0 >= t->root[a2]) {
              out[idx] = 0.0;
              continue;
            }
            c[a1] = 0.5 * (u0 + fmin(u0 + w, (double)t->root[a1]));
            c[a2] = 0.5 * (v0 + fmin(v0 + w, (double)t->root[a2]));
            out[idx] = column_march(t, c, k);
          }
      }
    }
    (void)na;
  }
  return idx;
}

/* offset of observer o's entries in the table */
static int64_t table_offset(const orc_tree* t, const orc_observers* obs, int block, int tiles, int o) {
  const int64_t n_blocks = (int64_t)blocks_along(t, 0, block) * blocks_along(t, 1, block) * blocks_along(t, 2, block);
  int64_t off = 0;
  for (int p = 0; p < o; ++p) off += n_blocks * n_axes(&obs->dir[3 * p]) * (int64_t)tiles * tiles;
  return off;
}

/* Peel-off march with the tables: exact optical depth until the ray leaves
 * the block of the scattering point, then the tabulated column of the tile
 * it leaves through. */
static double peel_march_tab(trace_worker* w, const double x0[3], int o, int bin, double tau_max, int* cut) {
  const orc_tree* t = w->job->t;
  const orc_observers* obs = w->job->obs;
  const int B = w->job->prm->peel_block, S = w->job->prm->peel_tiles;
  const double* k = &obs->dir[3 * o];
  double x[3] = {x0[0], x0[1], x0[2]};
  double kext = w->job->op->kappa_ext[bin] * t->h0;
  double tau = 0.0;
  *cut = 0;
  const orc_node* n = locate(t, x, k);
  if (!n) return 0.0;
  int b0[3];
  for (int a = 0; a < 3; ++a) b0[a] = (int)floor(n->lo[a]) / B;
  while (n) {
    int a;
    double s = exit_dist(n, x, k, &a);
    tau += kext * n->rho * s;
    if (s > 0) w->led.n_peel_cross += 1;
    if (tau_max > 0 && tau > tau_max) { *cut = 1; return tau; }
    move_to_face(n, x, k, s, a);
    n = locate(t, x, k);
    if (n && ((int)floor(n->lo[0]) / B != b0[0] || (int)floor(n->lo[1]) / B != b0[1] ||
              (int)floor(n->lo[2]) / B != b0[2])) {
      const int a1 = (a + 1) % 3, a2 = (a + 2) % 3;
      int iu = (int)floor((x[a1] - (double)b0[a1] * B) * S / B);
      int iv = (int)floor((x[a2] - (double)b0[a2] * B) * S / B);
      iu = iu < 0 ? 0 : (iu >= S ? S - 1 : iu);
      iv = iv < 0 ? 0 : (iv >= S ? S - 1 : iv);
      const int nb0 = blocks_along(t, 0, B), nb1 = blocks_along(t, 1, B);
      const int64_t blk = b0[0] + (int64_t)nb0 * (b0[1] + (int64_t)nb1 * b0[2]);
      const int64_t i = table_offset(t, obs, B, S, o) +
                        ((blk * n_axes(k) + axis_slot(k, a)) * S + iv) * (int64_t)S + iu;
      tau += kext * w->job->peel_tab[i];
      if (tau_max > 0 && tau > tau_max) *cut = 1;
      return tau;
    }
  }
  return tau;
}

static void peel(trace_worker* w, const double x[3], const double din[3], double W, int bin) {
  const orc_observers* obs = w->job->obs;
  const orc_tree* t = w->job->t;
  double g = w->job->op->g_hg[bin];
  int ob = w->job->bins > 1 ? bin : 0;
  for (int o = 0; o < obs->n_obs; ++o) {
    const double* k = &obs->dir[3 * o];
    double mu = din[0] * k[0] + din[1] * k[1] + din[2] * k[2];
    int cut;
    double tau = w->job->peel_tab ? peel_march_tab(w, x, o, bin, w->job->prm->peel_tau_max, &cut)
                                  : peel_march(w, x, k, bin, w->job->prm->peel_tau_max, &cut);
    if (cut) continue;
    double c = W * orc_hg_phase(g, mu) * exp(-tau);
    /* image basis: ex = normalise(up x k), ey = k x ex; centred on the box centre */
    const double* up = &obs->up[3 * o];
    double ex[3] = {up[1] * k[2] - up[2] * k[1], up[2] * k[0] - up[0] * k[2], up[0] * k[1] - up[1] * k[0]};
    double nn = sqrt(ex[0] * ex[0] + ex[1] * ex[1] + ex[2] * ex[2]);
    ex[0] /= nn; ex[1] /= nn; ex[2] /= nn;
    double ey[3] = {k[1] * ex[2] - k[2] * ex[1], k[2] * ex[0] - k[0] * ex[2], k[0] * ex[1] - k[1] * ex[0]};
    double r[3];
    for (int a = 0; a < 3; ++a) r[a] = x[a] * t->h0 - 0.5 * t->box[a];
    double u = r[0] * ex[0] + r[1] * ex[1] + r[2] * ex[2];
    double v = r[0] * ey[0] + r[1] * ey[1] + r[2] * ey[2];
    double fx = floor(u / (obs->fov[0] / obs->nx) + 0.5 * obs->nx);
    double fy = floor(v / (obs->fov[1] / obs->ny) + 0.5 * obs->ny);
    if (fx < 0 || fy < 0 || fx >= obs->nx || fy >= obs->ny) {
      w->led.n_peel_out += 1;
      continue;
    }
    int64_t slot = (((int64_t)o * w->job->bins + ob) * obs->ny + (int64_t)fy) * obs->nx + (int64_t)fx;
    image_add(w, slot, c);
    w->led.peeled += c;
  }
}

/* level of the shallowest grid between two cells: one below their deepest
 * common ancestor (0 if they lie in different root cells) */
static int visited_level(const orc_node* a, const orc_node* b) {
  const int top = a->level < b->level ? a->level : b->level;
  for (int l = top - 1; l >= 0; --l) {  /* ancestors at level l, deepest first */
    const double s = ldexp(1.0, l);
    int same = 1;
    for (int k = 0; k < 3; ++k) same &= floor(a->lo[k] * s) == floor(b->lo[k] * s);
    if (same) return l + 1;
  }
  return 0;
}

/* the cell whose packages include package k: the last c with first[c] <= k */
static int64_t search_first(const int64_t* first, int64_t n, int64_t k) {
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo + 1) / 2;
    if (first[mid] <= k) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

/* Dust packages of one (source, bin) per cell, in the form of the first
 * package index of each cell (first[n_cells] = their total); w_out: the
 * energy of one package.  Returns the total, -1 on a bad argument. */
static int64_t dust_first(const orc_tree* t, const orc_source* S, int src_index, int bin, const orc_params* prm,
                          int64_t* first, double* w_out) {
  const int64_t nc = t->n_cells;
  if (nc >= ((int64_t)1 << 30)) return -1;
  const double* em = S->emission + (int64_t)bin * nc;
  double E = 0.0;
  for (int64_t c = 0; c < nc; ++c) E += em[c];
  const int64_t N = S->packets[bin];
  double w = S->package_energy ? S->package_energy[bin] : (N > 0 ? E / (double)N : 0.0);
  if (w_out) *w_out = w;
  const uint32_t stream = ((uint32_t)src_index << 16) | (uint32_t)bin;
  int64_t tot = 0;
  for (int64_t c = 0; c < nc; ++c) {
    if (first) first[c] = tot;
    if (!(w > 0.0) || !(em[c] > 0.0)) continue;
    const uint64_t pk = ((uint64_t)0x80000000u << 32) | (uint64_t)c;
    const double u = ((double)orc_draw_u32(prm->seed, prm->job, prm->iter, stream, pk, 0) + 0.5) / 4294967296.0;
    tot += (int64_t)floor(em[c] / w + u);
  }
  if (first) first[nc] = tot;
  return tot;
}

int64_t orc_dust_packages(const orc_tree* t, const orc_source* src, int src_index, int n_lambda,
                          const orc_params* prm, int64_t* per_bin) {
  if (!t || !src || !prm || src->kind != ORC_SRC_DUST || !src->emission || !src->packets) return -1;
  int64_t tot = 0;
  for (int b = 0; b < n_lambda; ++b) {
    const int64_t n = src->packets[b] > 0 ? dust_first(t, src, src_index, b, prm, NULL, NULL) : 0;
    if (n < 0) return -1;
    if (per_bin) per_bin[b] = n;
    tot += n;
  }
  return tot;
}

static uint32_t raw_word(rstream* s) {
  return orc_draw_u32(s->seed, s->job, s->iter, s->stream, s->pkt, s->next++);
}

static int ipow(int b, int e) {
  int r = 1;
  while (e-- > 0) r *= b;
  return r;
}

/* Resampling at a change of grid level (Sect. 2.3): entering a grid dl
 * levels deeper, the package becomes M = N^dl packages of weight W/M at the
 * same point and direction, the copies with their own random streams (three
 * words drawn by the package name them) and free paths; leaving for a grid
 * dl levels shallower, it survives with probability 1/M (an integer test on
 * one drawn word) and then carries M W.  W0, the reference of the ordinary
 * roulette, follows the weight.  Returns 1 when the package is killed. */
static int resample(trace_worker* w, orc_path* P, const orc_node* n) {
  const orc_params* prm = w->job->prm;
  const int lv = n->level < prm->split_max_level ? n->level : prm->split_max_level;
  const int last = P->plev;
  P->plev = lv;
  if (last < 0 || lv == last) return 0;
  if (lv > last) {
    const int M = ipow(prm->split_factor, lv - last);
    const uint32_t w0 = raw_word(&P->rs), w1 = raw_word(&P->rs), w2 = raw_word(&P->rs);
    P->W /= M;
    P->W0 /= M;
    for (int k = 1; k < M; ++k) {
      if (w->n_stack == w->cap_stack) {
        w->cap_stack = w->cap_stack ? 2 * w->cap_stack : 64;
        w->stack = (orc_path*)realloc(w->stack, (size_t)w->cap_stack * sizeof(orc_path));
      }
      orc_path* c = &w->stack[w->n_stack++];
      *c = *P;
      c->rs.pkt = (uint64_t)w0 | ((uint64_t)w1 << 32);
      c->rs.next = 0;
      c->rs.stream = 0x80000000u | (w2 & 0x7FFFFF00u) | (uint32_t)k;
      c->tau = -log(uni(&c->rs));
    }
    w->led.n_split += M - 1;
    return 0;
  }
  const uint32_t M = (uint32_t)ipow(prm->split_factor, last - lv);
  const uint32_t u = raw_word(&P->rs);
  if ((uint64_t)u * M < ((uint64_t)1 << 32)) {
    const double Wn = P->W * M;
    w->led.rr_gain += Wn - P->W;
    P->W = Wn;
    P->W0 *= M;
    return 0;
  }
  w->led.rr_loss += P->W;
  P->W = 0;
  return 1;
}

/* Follows one path until it escapes, is killed or absorbed; returns its
 * fate (0 escaped, 1 roulette, 2 step limit, 3 analog absorption). */
static int follow(trace_worker* w, orc_path* P, int64_t p, int bin, double kext_b, int64_t origin,
                  double* nscat_out, double* ncross_out) {
  trace_job* J = w->job;
  const orc_tree* t = J->t;
  const orc_params* prm = J->prm;
  int64_t nc = t->n_cells;
  int ob = J->bins > 1 ? bin : 0;
  double alb = J->op->albedo[bin], g = J->op->g_hg[bin];
  int analog = prm->estimator == ORC_EST_ANALOG;
  double* x = P->x;
  double* d = P->d;
  double W = P->W, tau = P->tau;
  double nscat = 0, ncross = 0;
  int fate = 0;
  int64_t steps = 0;
  for (;;) {
    const orc_node* n = locate(t, x, d);
    if (!n) {  /* left through the outer boundary of the root grid */
      w->led.escaped += W;
      fate = 0;
      break;
    }
    if (n != P->prev) {
      const int v = P->prev ? visited_level(P->prev, n) : n->level;
      if (P->prev && prm->confine_level >= 0 && v <= prm->confine_level) {
        w->led.escaped += W;  /* left the subtree of the subiteration */
        fate = 0;
        break;
      }
      if (!P->prev || v < P->mlev) P->mlev = v;
      P->prev = n;
      if (prm->split_factor > 1) {
        P->W = W;
        P->tau = tau;
        if (resample(w, P, n)) { W = 0; fate = 1; break; }
        W = P->W;
      }
    }
    if (prm->per_level) ob = P->mlev;
    if (prm->step_limit > 0 && steps >= prm->step_limit) {
      w->led.killed += W;
      w->led.n_killed += 1;
      fate = 2;
      W = 0;
      break;
    }
    ++steps;
    int a;
    double s = exit_dist(n, x, d, &a);
    double kext = kext_b * n->rho;
    int64_t slot = (int64_t)ob * nc + n->id;
    if (!analog) {
      double ksca = alb * kext, kabs = (1.0 - alb) * kext;
      if (ksca > 0 && ksca * s >= tau) {
        /* scattering inside this cell */
        double ts = tau / ksca;
        double dep = -W * expm1(-kabs * ts);   /* W (1 - e^-dtau) without cancellation */
        deposit(w, slot, p, dep);
        if (prm->self_absorbed && n->id == origin)
          atomic_add_double(&prm->self_absorbed[(int64_t)bin * nc + n->id], dep);
        w->led.absorbed += dep;
        W *= exp(-kabs * ts);
        for (int b = 0; b < 3; ++b) x[b] += ts * d[b];
        if (ts > 0) { ncross += 1; w->led.n_cross += 1; }
        nscat += 1;
        w->led.n_scatter += 1;
        if (J->obs && J->obs->n_obs > 0) peel(w, x, d, W, bin);
        double mu = orc_hg_mu(g, uni(&P->rs));
        double phi = 2.0 * ORC_PI * uni(&P->rs);
        double nd[3];
        orc_scatter_dir(d, mu, phi, nd);
        d[0] = nd[0]; d[1] = nd[1]; d[2] = nd[2];
        if (prm->rr_wmin > 0 && W < prm->rr_wmin * P->W0) {
          double ur = uni(&P->rs);
          if (ur < prm->rr_p) {
            w->led.rr_loss += W;
            W = 0;
            fate = 1;
            break;
          }
          double Wn = W / (1.0 - prm->rr_p);
          w->led.rr_gain += Wn - W;
          W = Wn;
        }
        tau = -log(uni(&P->rs));
      } else {
        tau -= ksca * s;
        double dep = -W * expm1(-kabs * s);
        deposit(w, slot, p, dep);
        if (prm->self_absorbed && n->id == origin)
          atomic_add_double(&prm->self_absorbed[(int64_t)bin * nc + n->id], dep);
        w->led.absorbed += dep;
        W *= exp(-kabs * s);
        if (s > 0) { ncross += 1; w->led.n_cross += 1; }
        move_to_face(n, x, d, s, a);
      }
    } else {
      if (kext > 0 && kext * s >= tau) {
        double ts = tau / kext;
        for (int b = 0; b < 3; ++b) x[b] += ts * d[b];
        if (ts > 0) { ncross += 1; w->led.n_cross += 1; }
        double ua = uni(&P->rs);
        if (ua < alb) {
          nscat += 1;
          w->led.n_scatter += 1;
          if (J->obs && J->obs->n_obs > 0) peel(w, x, d, W, bin);
          double mu = orc_hg_mu(g, uni(&P->rs));
          double phi = 2.0 * ORC_PI * uni(&P->rs);
          double nd[3];
          orc_scatter_dir(d, mu, phi, nd);
          d[0] = nd[0]; d[1] = nd[1]; d[2] = nd[2];
        } else {
          deposit(w, slot, p, W);
          if (prm->self_absorbed && n->id == origin)
            atomic_add_double(&prm->self_absorbed[(int64_t)bin * nc + n->id], W);
          w->led.absorbed += W;
          W = 0;
          fate = 3;
          break;
        }
        tau = -log(uni(&P->rs));
      } else {
        tau -= kext * s;
        if (s > 0) { ncross += 1; w->led.n_cross += 1; }
        move_to_face(n, x, d, s, a);
      }
    }
  }
  P->W = W;
  P->tau = tau;
  *nscat_out = nscat;
  *ncross_out = ncross;
  return fate;
}

/* ------------------------------------------------------------------------ */
/* Polychromatic packages (Sect. 2.3, after Jonsson 2006)                     */
/* ------------------------------------------------------------------------ */
/* A package carries weights W_j for the bins j of its group; free paths and
 * scattering directions are drawn for the reference bin r.  Each W_j
 * carries the likelihood ratio of that path for its own bin: along a
 * segment of length s with no scattering the ratio of the no-scattering
 * probabilities, e^{-(ks_j - ks_r) rho s}; at a scattering the ratio of the
 * scattering coefficients ks_j / ks_r and of the phase functions
 * p_j(mu) / p_r(mu).  Absorption stays continuous: over a segment the bin-j
 * deposit is the integral of W_j(t) ka_j rho dt with
 * W_j(t) = W_j e^{-(ka_j + ks_j - ks_r) rho t}, i.e.
 *     W_j ta_j (1 - e^{-x_j}) / x_j,   x_j = (ka_j + ks_j - ks_r) rho s,
 * and W_j <- W_j e^{-x_j}.  For j = r this is the monochromatic package. */
static double phi1(double x) { return x != 0.0 ? -expm1(-x) / x : 1.0; }

#define ORC_POLY_MAX 8

static void peel_poly(trace_worker* w, const double x[3], const double din[3], const double* W, int first,
                      int size) {
  const orc_observers* obs = w->job->obs;
  const orc_tree* t = w->job->t;
  const orc_optics* op = w->job->op;
  for (int o = 0; o < obs->n_obs; ++o) {
    const double* k = &obs->dir[3 * o];
    double mu = din[0] * k[0] + din[1] * k[1] + din[2] * k[2];
    const double* up = &obs->up[3 * o];
    double ex[3] = {up[1] * k[2] - up[2] * k[1], up[2] * k[0] - up[0] * k[2], up[0] * k[1] - up[1] * k[0]};
    double nn = sqrt(ex[0] * ex[0] + ex[1] * ex[1] + ex[2] * ex[2]);
    ex[0] /= nn; ex[1] /= nn; ex[2] /= nn;
    double ey[3] = {k[1] * ex[2] - k[2] * ex[1], k[2] * ex[0] - k[0] * ex[2], k[0] * ex[1] - k[1] * ex[0]};
    double r[3];
    for (int a = 0; a < 3; ++a) r[a] = x[a] * t->h0 - 0.5 * t->box[a];
    double u = r[0] * ex[0] + r[1] * ex[1] + r[2] * ex[2];
    double v = r[0] * ey[0] + r[1] * ey[1] + r[2] * ey[2];
    double fx = floor(u / (obs->fov[0] / obs->nx) + 0.5 * obs->nx);
    double fy = floor(v / (obs->fov[1] / obs->ny) + 0.5 * obs->ny);
    if (fx < 0 || fy < 0 || fx >= obs->nx || fy >= obs->ny) {
      w->led.n_peel_out += 1;
      continue;
    }
    /* column density to the border (density x root-cell units): one march for all bins */
    double xx[3] = {x[0], x[1], x[2]};
    double col = 0.0;
    const orc_node* n = locate(t, xx, k);
    while (n) {
      int a;
      double s = exit_dist(n, xx, k, &a);
      col += n->rho * s;
      if (s > 0) w->led.n_peel_cross += 1;
      move_to_face(n, xx, k, s, a);
      n = locate(t, xx, k);
    }
    for (int j = 0; j < size; ++j) {
      const int b = first + j;
      double c = W[j] * orc_hg_phase(op->g_hg[b], mu) * exp(-op->kappa_ext[b] * t->h0 * col);
      int ob = w->job->bins > 1 ? b : 0;
      int64_t slot = (((int64_t)o * w->job->bins + ob) * obs->ny + (int64_t)fy) * obs->nx + (int64_t)fx;
      image_add(w, slot, c);
      w->led.peeled += c;
    }
  }
}

/* One polychromatic package of the group that starts at bin `first`. */
static void trace_poly(trace_worker* w, int64_t p, int si, int first, int64_t k, int64_t npk) {
  trace_job* J = w->job;
  const orc_tree* t = J->t;
  const orc_params* prm = J->prm;
  const orc_optics* op = J->op;
  const int nl = op->n_lambda;
  const int size = prm->poly_group < nl - first ? prm->poly_group : nl - first;
  const int rb = first + (size - 1) / 2;
  const orc_source* S = &J->src[si];
  rstream rs = {prm->seed, (uint64_t)(k + prm->packet_offset), 0, prm->job, prm->iter,
                ((uint32_t)si << 16) | (uint32_t)first};
  const int64_t nc = t->n_cells;
  double W[ORC_POLY_MAX], W0[ORC_POLY_MAX], ka[ORC_POLY_MAX], ks[ORC_POLY_MAX];
  double W0sum = 0.0;
  for (int j = 0; j < size; ++j) {
    const int b = first + j;
    W0[j] = S->bin_energy[b] / (double)npk;
    W[j] = W0[j];
    W0sum += W0[j];
    ka[j] = (1.0 - op->albedo[b]) * op->kappa_ext[b] * t->h0;
    ks[j] = op->albedo[b] * op->kappa_ext[b] * t->h0;
  }
  const double ksr = op->albedo[rb] * op->kappa_ext[rb] * t->h0, gr = op->g_hg[rb];
  double x[3], d[3];
  if (S->kind == ORC_SRC_POINT) {
    for (int a = 0; a < 3; ++a) x[a] = S->pos[a] / t->h0;
    double u1 = uni(&rs), u2 = uni(&rs);
    iso_dir(u1, u2, d);
  } else if (S->kind == ORC_SRC_BEAM) {
    double nn = sqrt(S->dir[0] * S->dir[0] + S->dir[1] * S->dir[1] + S->dir[2] * S->dir[2]);
    for (int a = 0; a < 3; ++a) { x[a] = S->pos[a] / t->h0; d[a] = S->dir[a] / nn; }
  } else {
    double area[3] = {t->box[1] * t->box[2], t->box[0] * t->box[2], t->box[0] * t->box[1]};
    double tot = 2.0 * (area[0] + area[1] + area[2]);
    double u0 = uni(&rs) * tot, cum = 0.0;
    int face = 5;
    for (int f = 0; f < 6; ++f) {
      cum += area[f / 2];
      if (u0 < cum) { face = f; break; }
    }
    int a = face / 2, a1 = (a + 1) % 3, a2 = (a + 2) % 3;
    if (a1 > a2) { int tmp = a1; a1 = a2; a2 = tmp; }
    double u1 = uni(&rs), u2 = uni(&rs), u3 = uni(&rs), u4 = uni(&rs);
    x[a] = (face & 1) ? (double)t->root[a] : 0.0;
    x[a1] = u1 * t->root[a1];
    x[a2] = u2 * t->root[a2];
    double mu = sqrt(u3), st = sqrt(fmax(0.0, 1.0 - mu * mu)), phi = 2.0 * ORC_PI * u4;
    d[a] = (face & 1) ? -mu : mu;
    d[a1] = st * cos(phi);
    d[a2] = st * sin(phi);
  }
  w->led.emitted += W0sum;
  w->led.n_packets += 1;
  double tau = -log(uni(&rs));
  double nscat = 0, ncross = 0;
  int fate = 0;
  int64_t steps = 0;
  for (;;) {
    const orc_node* n = locate(t, x, d);
    if (!n) {
      for (int j = 0; j < size; ++j) w->led.escaped += W[j];
      fate = 0;
      break;
    }
    if (prm->step_limit > 0 && steps >= prm->step_limit) {
      for (int j = 0; j < size; ++j) { w->led.killed += W[j]; W[j] = 0; }
      w->led.n_killed += 1;
      fate = 2;
      break;
    }
    ++steps;
    int a;
    double s = exit_dist(n, x, d, &a);
    const double ksr_c = ksr * n->rho;
    const int scat = ksr_c > 0 && ksr_c * s >= tau;
    const double seg = scat ? tau / ksr_c : s;
    for (int j = 0; j < size; ++j) {
      const double xj = (ka[j] + ks[j] - ksr) * n->rho * seg;
      const double dep = W[j] * ka[j] * n->rho * seg * phi1(xj);
      int ob = J->bins > 1 ? first + j : 0;
      deposit(w, (int64_t)ob * nc + n->id, p, dep);
      w->led.absorbed += dep;
      W[j] *= exp(-xj);
    }
    if (seg > 0) { ncross += 1; w->led.n_cross += 1; }
    if (scat) {
      for (int b = 0; b < 3; ++b) x[b] += seg * d[b];
      nscat += 1;
      w->led.n_scatter += 1;
      /* the event: each bin scatters here with ks_j / ks_r of the reference's rate */
      for (int j = 0; j < size; ++j) W[j] *= ks[j] / ksr;
      if (J->obs && J->obs->n_obs > 0) peel_poly(w, x, d, W, first, size);
      double mu = orc_hg_mu(gr, uni(&rs));
      double phi = 2.0 * ORC_PI * uni(&rs);
      double nd[3];
      orc_scatter_dir(d, mu, phi, nd);
      d[0] = nd[0]; d[1] = nd[1]; d[2] = nd[2];
      const double pr = orc_hg_phase(gr, mu);
      double rmax = 0.0;
      for (int j = 0; j < size; ++j) {
        W[j] *= orc_hg_phase(op->g_hg[first + j], mu) / pr;
        const double q = W[j] / W0[j];
        if (q > rmax) rmax = q;
      }
      if (prm->rr_wmin > 0 && rmax < prm->rr_wmin) {
        double ur = uni(&rs);
        if (ur < prm->rr_p) {
          for (int j = 0; j < size; ++j) { w->led.rr_loss += W[j]; W[j] = 0; }
          fate = 1;
          break;
        }
        for (int j = 0; j < size; ++j) {
          double Wn = W[j] / (1.0 - prm->rr_p);
          w->led.rr_gain += Wn - W[j];
          W[j] = Wn;
        }
      }
      tau = -log(uni(&rs));
    } else {
      tau -= ksr_c * s;
      move_to_face(n, x, d, s, a);
    }
  }
  if (w->pkt_acc) flush_packet(w);
  if (J->rec) {
    double* r = &J->rec[p * 10];
    double we = 0.0;
    for (int j = 0; j < size; ++j) we += W[j];
    r[0] = fate == 0 ? we : 0.0;
    r[1] = nscat;
    r[2] = ncross;
    r[3] = fate;
    for (int b = 0; b < 3; ++b) { r[4 + b] = x[b] * t->h0; r[7 + b] = d[b]; }
  }
}

static void trace_one(trace_worker* w, int64_t p) {
  trace_job* J = w->job;
  const orc_tree* t = J->t;
  const orc_params* prm = J->prm;
  int nl = J->op->n_lambda;
  /* which (source, bin) stream this packet belongs to */
  int64_t seg = 0;
  {
    int64_t lo = 0, hi = (int64_t)J->n_src * nl - 1;
    while (lo < hi) {
      int64_t mid = (lo + hi + 1) / 2;
      if (J->seg_begin[mid] <= p) lo = mid;
      else hi = mid - 1;
    }
    seg = lo;
  }
  int si = (int)(seg / nl), bin = (int)(seg % nl);
  int64_t k = p - J->seg_begin[seg];
  int64_t npk = J->seg_begin[seg + 1] - J->seg_begin[seg];
  if (prm->poly_group > 1) {
    trace_poly(w, p, si, bin, k, npk);
    return;
  }
  const orc_source* S = &J->src[si];
  rstream rs = {prm->seed, (uint64_t)(k + prm->packet_offset), 0, prm->job, prm->iter,
                ((uint32_t)si << 16) | (uint32_t)bin};
  int ob = J->bins > 1 ? bin : 0;
  int64_t nc = t->n_cells;

  double x[3], d[3], E;
  int64_t origin = -1;  /* emission cell of a dust package */
  double W0;
  if (S->kind == ORC_SRC_DUST) {
    W0 = J->w_dust[seg];
  } else {
    E = S->bin_energy[bin];
    W0 = E / (double)npk;
  }
  double W = W0;

  /* emission (Sect. 2.3: packages from internal sources; root inwards
   * array for the external field) */
  if (S->kind == ORC_SRC_POINT) {
    for (int a = 0; a < 3; ++a) x[a] = S->pos[a] / t->h0;
    double u1 = uni(&rs), u2 = uni(&rs);
    iso_dir(u1, u2, d);
  } else if (S->kind == ORC_SRC_BEAM) {
    double nn = sqrt(S->dir[0] * S->dir[0] + S->dir[1] * S->dir[1] + S->dir[2] * S->dir[2]);
    for (int a = 0; a < 3; ++a) { x[a] = S->pos[a] / t->h0; d[a] = S->dir[a] / nn; }
  } else if (S->kind == ORC_SRC_EXTERNAL) {
    double area[3] = {t->box[1] * t->box[2], t->box[0] * t->box[2], t->box[0] * t->box[1]};
    double tot = 2.0 * (area[0] + area[1] + area[2]);
    double u0 = uni(&rs) * tot, cum = 0.0;
    int face = 5;
    for (int f = 0; f < 6; ++f) {
      cum += area[f / 2];
      if (u0 < cum) { face = f; break; }
    }
    int a = face / 2, a1 = (a + 1) % 3, a2 = (a + 2) % 3;
    if (a1 > a2) { int tmp = a1; a1 = a2; a2 = tmp; }
    double u1 = uni(&rs), u2 = uni(&rs), u3 = uni(&rs), u4 = uni(&rs);
    x[a] = (face & 1) ? (double)t->root[a] : 0.0;
    x[a1] = u1 * t->root[a1];
    x[a2] = u2 * t->root[a2];
    double mu = sqrt(u3), st = sqrt(fmax(0.0, 1.0 - mu * mu)), phi = 2.0 * ORC_PI * u4;
    d[a] = (face & 1) ? -mu : mu;
    d[a1] = st * cos(phi);
    d[a2] = st * sin(phi);
  } else { /* dust emission: package j of its cell, with the cell's own stream */
    const int64_t c = search_first(J->first[seg], nc + 1, k);
    const int64_t j = k - J->first[seg][c];
    rs.pkt = ((uint64_t)(0x40000000u | (uint32_t)c) << 32) | (uint32_t)(j + prm->packet_offset);
    origin = c;
    if (prm->self_emitted) atomic_add_double(&prm->self_emitted[(int64_t)bin * nc + c], W0);
    if (prm->self_count) atomic_add_double(&prm->self_count[c], 1.0);
    const orc_node* n = &t->nodes[c];
    double u1 = uni(&rs), u2 = uni(&rs), u3 = uni(&rs);
    x[0] = n->lo[0] + u1 * n->size;
    x[1] = n->lo[1] + u2 * n->size;
    x[2] = n->lo[2] + u3 * n->size;
    double u4 = uni(&rs), u5 = uni(&rs);
    iso_dir(u4, u5, d);
  }
  w->led.emitted += W0;
  w->led.n_packets += 1;

  double kext_b = J->op->kappa_ext[bin] * t->h0;   /* per unit density, per root-cell unit */
  orc_path P;
  for (int k2 = 0; k2 < 3; ++k2) { P.x[k2] = x[k2]; P.d[k2] = d[k2]; }
  P.W = W;
  P.W0 = W0;
  P.rs = rs;
  P.tau = -log(uni(&P.rs));
  P.prev = NULL;
  P.mlev = 0;
  /* resampling (Sect. 2.3): the external field enters through the root grid */
  P.plev = S->kind == ORC_SRC_EXTERNAL ? 0 : -1;
  int primary = 1;
  for (;;) {
    double nscat = 0, ncross = 0;
    int fate = follow(w, &P, p, bin, kext_b, origin, &nscat, &ncross);
    if (primary && J->rec) {
      double* r = &J->rec[p * 10];
      r[0] = fate == 0 ? P.W : 0.0;
      r[1] = nscat;
      r[2] = ncross;
      r[3] = fate;
      for (int a = 0; a < 3; ++a) { r[4 + a] = P.x[a] * t->h0; r[7 + a] = P.d[a]; }
    }
    primary = 0;
    if (w->n_stack == 0) break;
    P = w->stack[--w->n_stack];
  }
  if (w->pkt_acc) flush_packet(w);
}

static void* trace_thread(void* arg) {
  trace_worker* w = (trace_worker*)arg;
  for (int64_t p = w->p0; p < w->p1; ++p) {
    w->cur_pkt = p;
    trace_one(w, p);
  }
  return NULL;
}

static void ledger_add(orc_ledger* a, const orc_ledger* b) {
  a->emitted += b->emitted; a->absorbed += b->absorbed; a->escaped += b->escaped;
  a->rr_gain += b->rr_gain; a->rr_loss += b->rr_loss; a->killed += b->killed; a->peeled += b->peeled;
  a->n_packets += b->n_packets; a->n_cross += b->n_cross; a->n_scatter += b->n_scatter;
  a->n_peel_cross += b->n_peel_cross; a->n_killed += b->n_killed; a->n_peel_out += b->n_peel_out;
  a->n_split += b->n_split;
}

int orc_trace(const orc_tree* t, int n_src, const orc_source* src, const orc_optics* op,
              const orc_params* prm, const orc_observers* obs, double* absorbed, double* images,
              double* sumsq, double* hits, double* rec, orc_ledger* ledger) {
  if (!t || n_src <= 0 || !src || !op || !prm || op->n_lambda <= 0) return -1;
  if (prm->per_level && obs && obs->n_obs > 0) return -1;  /* levels take the place of bins */
  if (prm->poly_group > 1) {  /* polychromatic: plain continuous estimator, no dust sources */
    if (prm->poly_group > ORC_POLY_MAX || prm->estimator != ORC_EST_CONTINUOUS || prm->split_factor > 1 ||
        prm->per_level || prm->self_absorbed || prm->peel_block > 0)
      return -1;
    for (int s = 0; s < n_src; ++s)
      if (src[s].kind == ORC_SRC_DUST) return -1;
    for (int f = 0; f < op->n_lambda; f += prm->poly_group) {  /* the reference bin must scatter */
      const int size = prm->poly_group < op->n_lambda - f ? prm->poly_group : op->n_lambda - f;
      const int r = f + (size - 1) / 2;
      int any = 0;
      for (int j = 0; j < size; ++j) any |= op->albedo[f + j] * op->kappa_ext[f + j] > 0;
      if (any && !(op->albedo[r] * op->kappa_ext[r] > 0)) return -1;
    }
  }
  if (prm->split_factor > 1) {  /* a split makes at most 256 packages */
    const int lm = prm->split_max_level < t->n_levels - 1 ? prm->split_max_level : t->n_levels - 1;
    if (lm < 0) return -1;
    int64_t m = 1;
    for (int l = 0; l < lm; ++l) m *= prm->split_factor;
    if (m > 256) return -1;
  }
  int nl = op->n_lambda;
  int bins = prm->per_level ? t->n_levels : (prm->per_lambda ? nl : 1);
  int64_t nc = t->n_cells;
  trace_job J;
  memset(&J, 0, sizeof J);
  J.t = t; J.n_src = n_src; J.src = src; J.op = op; J.prm = prm; J.obs = obs; J.bins = bins; J.rec = rec;
  J.seg_begin = (int64_t*)calloc((size_t)n_src * nl + 1, sizeof(int64_t));
  J.first = (int64_t**)calloc((size_t)n_src * nl, sizeof(int64_t*));
  J.w_dust = (double*)calloc((size_t)n_src * nl, sizeof(double));
  for (int s = 0; s < n_src; ++s)
    for (int b = 0; b < nl; ++b) {
      int64_t i = (int64_t)s * nl + b;
      int64_t n = src[s].packets[b];
      if (src[s].kind == ORC_SRC_DUST) {
        n = 0;
        if (src[s].packets[b] > 0) {
          J.first[i] = (int64_t*)malloc((size_t)(nc + 1) * sizeof(int64_t));
          n = dust_first(t, &src[s], s, b, prm, J.first[i], &J.w_dust[i]);
          if (n < 0) {
            for (int64_t j = 0; j <= i; ++j) free(J.first[j]);
            free(J.first); free(J.w_dust); free(J.seg_begin);
            return -1;
          }
        }
      }
      J.seg_begin[i + 1] = J.seg_begin[i] + n;
    }
  J.n_packets = J.seg_begin[(int64_t)n_src * nl];
  if (obs && obs->n_obs > 0 && prm->peel_block > 0) {
    const int64_t ne = orc_peel_table(t, obs, prm->peel_block, prm->peel_tiles, NULL);
    if (ne < 0) return -1;
    J.peel_tab = (double*)calloc((size_t)(ne > 0 ? ne : 1), sizeof(double));
    orc_peel_table(t, obs, prm->peel_block, prm->peel_tiles, J.peel_tab);
  }
  int T = prm->n_threads > 0 ? prm->n_threads : 1;
  if (J.n_packets < T) T = J.n_packets > 0 ? (int)J.n_packets : 1;
  int64_t n_img = obs && obs->n_obs > 0 ? (int64_t)obs->n_obs * bins * obs->ny * obs->nx : 0;
  double per_thread_bytes = 8.0 * ((double)bins * nc + (double)n_img);
  int validation = sumsq && hits;
  const int img_var = validation && n_img > 0 && prm->image_sumsq;
  J.shared_atomic = T > 1 && per_thread_bytes * T > 2.0e9;
  if (validation && J.shared_atomic) T = 1, J.shared_atomic = 0;
  J.absorbed_shared = absorbed;
  J.images_shared = images;

  trace_worker* ws = (trace_worker*)calloc((size_t)T, sizeof(trace_worker));
  pthread_t* th = (pthread_t*)calloc((size_t)T, sizeof(pthread_t));
  for (int i = 0; i < T; ++i) {
    trace_worker* w = &ws[i];
    w->job = &J;
    w->p0 = J.n_packets * i / T;
    w->p1 = J.n_packets * (i + 1) / T;
    if (T == 1 || J.shared_atomic) {
      w->absorbed = absorbed;
      w->images = images;
      w->sumsq = sumsq;
      w->hits = hits;
    } else {
      w->absorbed = (double*)calloc((size_t)bins * nc, sizeof(double));
      w->images = n_img ? (double*)calloc((size_t)n_img, sizeof(double)) : NULL;
      if (validation) {
        w->sumsq = (double*)calloc((size_t)bins * nc, sizeof(double));
        w->hits = (double*)calloc((size_t)bins * nc, sizeof(double));
      }
    }
    if (validation) {
      w->pkt_acc = (double*)calloc((size_t)bins * nc, sizeof(double));
      w->stamp = (int64_t*)malloc((size_t)bins * nc * sizeof(int64_t));
      for (int64_t k = 0; k < (int64_t)bins * nc; ++k) w->stamp[k] = -1;
    }
    if (img_var) {
      w->img_sumsq = T == 1 ? prm->image_sumsq : (double*)calloc((size_t)n_img, sizeof(double));
      w->img_acc = (double*)calloc((size_t)n_img, sizeof(double));
      w->img_stamp = (int64_t*)malloc((size_t)n_img * sizeof(int64_t));
      for (int64_t k = 0; k < n_img; ++k) w->img_stamp[k] = -1;
    }
  }
  if (T == 1) trace_thread(&ws[0]);
  else {
    for (int i = 0; i < T; ++i) pthread_create(&th[i], NULL, trace_thread, &ws[i]);
    for (int i = 0; i < T; ++i) pthread_join(th[i], NULL);
  }
  orc_ledger L;
  memset(&L, 0, sizeof L);
  for (int i = 0; i < T; ++i) {
    trace_worker* w = &ws[i];
    ledger_add(&L, &w->led);
    if (T > 1 && !J.shared_atomic) {
      for (int64_t k = 0; k < (int64_t)bins * nc; ++k) absorbed[k] += w->absorbed[k];
      for (int64_t k = 0; k < n_img; ++k) images[k] += w->images[k];
      if (validation)
        for (int64_t k = 0; k < (int64_t)bins * nc; ++k) { sumsq[k] += w->sumsq[k]; hits[k] += w->hits[k]; }
      free(w->absorbed); free(w->images); free(w->sumsq); free(w->hits);
    }
    if (img_var && T > 1) {
      for (int64_t k = 0; k < n_img; ++k) prm->image_sumsq[k] += w->img_sumsq[k];
      free(w->img_sumsq);
    }
    free(w->img_acc); free(w->img_stamp); free(w->img_touched);
    free(w->pkt_acc); free(w->stamp); free(w->touched); free(w->stack);
  }
  if (ledger) *ledger = L;
  for (int64_t i = 0; i < (int64_t)n_src * nl; ++i) free(J.first[i]);
  free(J.first); free(J.w_dust); free(J.seg_begin); free(ws); free(th); free(J.peel_tab);
  return 0;
}

/* One peel-off contribution from a given scattering point (cm) and incoming
 * direction, into images [n_obs][bins][ny][nx]. */
int orc_peel_point(const orc_tree* t, const orc_optics* op, const orc_observers* obs, int bin,
                   int per_lambda, const double x_cm[3], const double din[3], double W, double* images) {
  trace_job J;
  memset(&J, 0, sizeof J);
  orc_params prm;
  memset(&prm, 0, sizeof prm);
  J.t = t; J.op = op; J.obs = obs; J.prm = &prm; J.bins = per_lambda ? op->n_lambda : 1;
  trace_worker w;
  memset(&w, 0, sizeof w);
  w.job = &J;
  w.images = images;
  double x[3] = {x_cm[0] / t->h0, x_cm[1] / t->h0, x_cm[2] / t->h0};
  peel(&w, x, din, W, bin);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Dust temperature                                                           */
/* ------------------------------------------------------------------------ */
static double planck_nu(double nu, double T) {
  double x = H_CGS * nu / (K_CGS * T);
  return 2.0 * H_CGS * nu * nu * nu / (C_CGS * C_CGS) / expm1(x);
}

double orc_emission_per_mass(const orc_dust* d, double T) {
  double s = 0.0;
  for (int i = 0; i < d->n_lambda; ++i) {
    double nu = C_CGS / (d->lambda_um[i] * 1e-4);
    s += d->kappa_abs[i] * planck_nu(nu, T) * d->dnu[i];
  }
  return 4.0 * ORC_PI * s;
}

typedef struct {
  const orc_tree* t;
  const double* A;
  const orc_dust* d;
  double* T;
  int64_t c0, c1;
} temp_work;

static void* temp_thread(void* arg) {
  temp_work* w = (temp_work*)arg;
  const orc_tree* t = w->t;
  double Emin = orc_emission_per_mass(w->d, w->d->T_min);
  double Emax = orc_emission_per_mass(w->d, w->d->T_max);
  for (int64_t c = w->c0; c < w->c1; ++c) {
    const orc_node* n = &t->nodes[c];
    if (n->child) { w->T[c] = 0.0; continue; }
    double h = t->h0 * n->size;
    double mass = n->rho * h * h * h;
    if (!(mass > 0) || !(w->A[c] > 0)) { w->T[c] = w->d->T_min; continue; }
    double target = w->A[c] / mass;
    if (target <= Emin) { w->T[c] = w->d->T_min; continue; }
    if (target >= Emax) { w->T[c] = w->d->T_max; continue; }
    double lo = w->d->T_min, hi = w->d->T_max;
    while (hi - lo > 1e-13 * lo) {
      double mid = 0.5 * (lo + hi);
      if (orc_emission_per_mass(w->d, mid) < target) lo = mid;
      else hi = mid;
    }
    w->T[c] = 0.5 * (lo + hi);
  }
  return NULL;
}

int orc_dust_temperature(const orc_tree* t, const double* absorbed_total, const orc_dust* d,
                         int n_threads, double* T) {
  if (!t || !absorbed_total || !d || !T || d->n_lambda <= 0 || !(d->T_min > 0) || !(d->T_max > d->T_min))
    return -1;
  int NT = n_threads > 0 ? n_threads : 1;
  temp_work* ws = (temp_work*)calloc((size_t)NT, sizeof(temp_work));
  pthread_t* th = (pthread_t*)calloc((size_t)NT, sizeof(pthread_t));
  for (int i = 0; i < NT; ++i) {
    ws[i].t = t; ws[i].A = absorbed_total; ws[i].d = d; ws[i].T = T;
    ws[i].c0 = t->n_cells * i / NT;
    ws[i].c1 = t->n_cells * (i + 1) / NT;
  }
  if (NT == 1) temp_thread(&ws[0]);
  else {
    for (int i = 0; i < NT; ++i) pthread_create(&th[i], NULL, temp_thread, &ws[i]);
    for (int i = 0; i < NT; ++i) pthread_join(th[i], NULL);
  }
  free(ws); free(th);
  return 0;
}

/* The temperature of the ALI step with a diagonal operator per frequency
 * (Eq. 3; Sect. 3.1: the system decouples into one equation per cell):
 * sum_b w_b E_b(T) = rhs per leaf, with E_b(T) = 4 pi rho V kappa_b B_b(T)
 * dnu_b and weights w_b = 1 - Lambda_b ([n_lambda][n_cells]), by bisection
 * in T to 1e-13 relative, clamped to [T_min, T_max]. */
typedef struct {
  const orc_tree* t;
  const double* rhs;
  const double* w;
  const orc_dust* d;
  double* T;
  int64_t c0, c1;
} wtemp_work;

static double weighted_emission(const orc_dust* d, const double* w, int64_t nc, int64_t c, double T) {
  double s = 0.0;
  for (int b = 0; b < d->n_lambda; ++b) {
    double nu = C_CGS / (d->lambda_um[b] * 1e-4);
    s += w[(int64_t)b * nc + c] * d->kappa_abs[b] * planck_nu(nu, T) * d->dnu[b];
  }
  return 4.0 * ORC_PI * s;
}

static void* wtemp_thread(void* arg) {
  wtemp_work* w = (wtemp_work*)arg;
  const orc_tree* t = w->t;
  const int64_t nc = t->n_cells;
  for (int64_t c = w->c0; c < w->c1; ++c) {
    const orc_node* n = &t->nodes[c];
    if (n->child) { w->T[c] = 0.0; continue; }
    double h = t->h0 * n->size;
    double mass = n->rho * h * h * h;
    if (!(mass > 0) || !(w->rhs[c] > 0)) { w->T[c] = w->d->T_min; continue; }
    double target = w->rhs[c] / mass;
    if (target <= weighted_emission(w->d, w->w, nc, c, w->d->T_min)) { w->T[c] = w->d->T_min; continue; }
    if (target >= weighted_emission(w->d, w->w, nc, c, w->d->T_max)) { w->T[c] = w->d->T_max; continue; }
    double lo = w->d->T_min, hi = w->d->T_max;
    while (hi - lo > 1e-13 * lo) {
      double mid = 0.5 * (lo + hi);
      if (weighted_emission(w->d, w->w, nc, c, mid) < target) lo = mid;
      else hi = mid;
    }
    w->T[c] = 0.5 * (lo + hi);
  }
  return NULL;
}

int orc_dust_temperature_weighted(const orc_tree* t, const double* rhs, const double* weights, const orc_dust* d,
                                  int n_threads, double* T) {
  if (!t || !rhs || !weights || !d || !T || d->n_lambda <= 0 || !(d->T_min > 0) || !(d->T_max > d->T_min))
    return -1;
  int NT = n_threads > 0 ? n_threads : 1;
  wtemp_work* ws = (wtemp_work*)calloc((size_t)NT, sizeof(wtemp_work));
  pthread_t* th = (pthread_t*)calloc((size_t)NT, sizeof(pthread_t));
  for (int i = 0; i < NT; ++i) {
    ws[i].t = t; ws[i].rhs = rhs; ws[i].w = weights; ws[i].d = d; ws[i].T = T;
    ws[i].c0 = t->n_cells * i / NT;
    ws[i].c1 = t->n_cells * (i + 1) / NT;
  }
  if (NT == 1) wtemp_thread(&ws[0]);
  else {
    for (int i = 0; i < NT; ++i) pthread_create(&th[i], NULL, wtemp_thread, &ws[i]);
    for (int i = 0; i < NT; ++i) pthread_join(th[i], NULL);
  }
  free(ws); free(th);
  return 0;
}

int orc_dust_emission(const orc_tree* t, const double* T, const orc_dust* d, double* emission) {
  if (!t || !T || !d || !emission) return -1;
  int64_t nc = t->n_cells;
  for (int b = 0; b < d->n_lambda; ++b) {
    double nu = C_CGS / (d->lambda_um[b] * 1e-4);
    for (int64_t c = 0; c < nc; ++c) {
      const orc_node* n = &t->nodes[c];
      double v = 0.0;
      if (!n->child && T[c] > 0) {
        double h = t->h0 * n->size;
        v = 4.0 * ORC_PI * n->rho * h * h * h * d->kappa_abs[b] * planck_nu(nu, T[c]) * d->dnu[b];
      }
      emission[(int64_t)b * nc + c] = v;
    }
  }
  return 0;
}
