/*
 * rt_oracle.h -- FP64 CPU oracle for Monte Carlo radiative transfer on a
 * hierarchical (2x2x2-refined) cartesian grid.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, obviously-correct
 * restatement of the method of Lunttila & Juvela, "Radiative transfer on
 * hierarchial grids" (Sects. 2-3), written to check the CUDA library.  Only
 * the test-suite, the smoke check and the benchmark's CPU-baseline leg may
 * load it.  It shares no code, header or constant table with the library.
 *
 * Coordinates: internally the oracle works in root-cell units (a root cell is
 * 1 unit, a level-l cell 2^-l units); physical lengths are those units times
 * h0 = box/root (cm).  Every cell is half-open [lo, lo+size) except that a
 * point lying exactly on a face belongs to the cell the ray moves into.
 */
#ifndef RT_ORACLE_H
#define RT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_tree orc_tree;

/* Tree description, level order (Sect. 2.1 nested grids, restricted to
 * octree refinement).  density is g/cm^3 per cell; refined cells' values are
 * ignored. */
typedef struct {
  int root[3];
  double box[3];
  int n_levels;
  const int64_t* n_refined;
  const uint8_t* refine_flags;
  const double* density;
} orc_tree_desc;

/* Build the pointer octree.  Returns NULL on inconsistent input. */
orc_tree* orc_tree_build(const orc_tree_desc* d);
void orc_tree_free(orc_tree* t);
int64_t orc_tree_ncells(const orc_tree* t);
/* per-cell level (uint8) and leaf flag (1 = leaf) in level order */
void orc_tree_cells(const orc_tree* t, uint8_t* level, uint8_t* is_leaf);

/* Philox4x32-10 and Philox4x64-10 (Salmon et al. 2011, SC'11). */
void orc_philox4x32(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
/* draw j of a packet stream, as uint32 */
uint32_t orc_draw_u32(uint64_t seed, uint32_t job, uint32_t iter, uint32_t stream,
                      uint64_t pkt, uint64_t j);

/* Deterministic walk of one ray (Sect. 2.3 cell stepping), origin in cm.
 * Writes up to max_seg segments of positive length: leaf cell id, length
 * (cm) and a tie margin (distance of the exit point from the nearest other
 * cell face, in units of the smaller of the two cells).  Returns the number
 * of segments, or -1 if the origin is outside the box. */
int64_t orc_walk(const orc_tree* t, const double origin[3], const double dir[3],
                 int64_t max_seg, int64_t* cells, double* lengths, double* margins);

enum { ORC_SRC_POINT = 0, ORC_SRC_EXTERNAL = 1, ORC_SRC_DUST = 2, ORC_SRC_BEAM = 3 };
enum { ORC_EST_CONTINUOUS = 0, ORC_EST_ANALOG = 1 };

typedef struct {
  int kind;
  double pos[3];               /* cm: point / beam origin */
  double dir[3];               /* beam direction */
  const double* bin_energy;    /* [n_lambda] (point, external, beam) */
  const int64_t* packets;      /* [n_lambda] packets per bin (dust: the expected number) */
  const double* emission;      /* dust: [n_lambda][n_cells] energy per cell per bin */
  const double* package_energy; /* dust, optional: [n_lambda] energy of one package (default: the
                                 * bin's emission / packets) */
} orc_source;

typedef struct {
  int n_lambda;
  const double* kappa_ext;     /* cm^2/g */
  const double* albedo;
  const double* g_hg;
} orc_optics;

typedef struct {
  int n_obs;
  const double* dir;           /* [n_obs][3] */
  const double* up;            /* [n_obs][3] */
  int nx, ny;
  double fov[2];               /* cm */
} orc_observers;

typedef struct {
  uint64_t seed;
  uint32_t job, iter;
  int estimator;
  double rr_wmin;              /* roulette below rr_wmin * W0; <= 0 disables */
  double rr_p;
  int64_t step_limit;          /* max segments per packet, <= 0: none */
  double peel_tau_max;         /* <= 0: march to the boundary always */
  int per_lambda;              /* 1: outputs per bin; 0: summed */
  int n_threads;
  int64_t packet_offset;       /* package k of a (source, bin) draws the stream of index k + offset */
  int peel_block;              /* > 0: accelerated peel-off (Sect. 2.4) with blocks of this many root cells */
  int peel_tiles;              /*      and peel_tiles x peel_tiles tiles on each block face */
  /* Subiterations (Sect. 3.2, App. B): the grid of a cell at level l is the
   * set of 8 children of its parent (the root grid for l = 0).  A package
   * remembers the shallowest grid level it has been in: the level of its
   * emission cell at first, then, at each crossing, the level of the
   * shallowest grid on the way (one below the deepest common ancestor of the
   * two cells; 0 between root cells). */
  int per_level;               /* 1: absorbed is [n_levels][n_cells]: deposits by that level */
  int confine_level;           /* >= 0: a package that reaches a grid of this level or shallower
                                  (it left the subtree of its level-L ancestor) leaves the run,
                                  booked as escaped; < 0: no confinement */
  double* self_absorbed;       /* optional [n_lambda][n_cells]: energy a dust package deposits in its
                                  own emission cell, per bin and cell (the diagonal of Lambda, Eq. 3) */
  double* self_emitted;        /* with self_absorbed: [n_lambda][n_cells] energy of the dust packages
                                  emitted per bin and cell */
  double* self_count;          /* with self_absorbed: [n_cells] number of dust packages emitted per cell */
  /* Resampling at grid boundaries (Sect. 2.3): a package entering a cell dl
   * grid levels deeper than its last cell is split into split_factor^dl
   * packages; one leaving for a cell dl levels shallower survives with
   * probability split_factor^-dl.  Levels are capped at split_max_level. */
  int split_factor;            /* <= 1: off */
  int split_max_level;
  /* Polychromatic packages (Sect. 2.3): > 1: the wavelength bins form
   * consecutive groups of poly_group bins (the last may be shorter) and a
   * package carries one weight per bin of its group; its path is drawn at
   * the group's reference bin (the middle one) and each bin's weight carries
   * the likelihood ratio of that path.  Packages are counted per group, at
   * the group's first bin of `packets`. */
  int poly_group;
  /* Optional [n_obs][bins][ny][nx], with observers: per pixel, the sum over
   * packages of the square of each package's total contribution to it (the
   * Monte Carlo variance of the images, as sumsq is for absorbed). */
  double* image_sumsq;
} orc_params;

/* Dust packages per cell (Sect. 4.2: the number of packages a cell sends at
 * a frequency follows its emission there, and every package of the
 * frequency carries the same energy w_b = E_b / N_b).  Cell c sends
 * floor(E_bc / w_b + u_bc) packages, u_bc the uniform of word 0 of Philox
 * counter (c, 0x80000000 | (c >> 32), 0, (source << 16) | bin) under the
 * run's key: the expected count is E_bc / w_b, the count is within one of
 * it, and it does not change between runs with the same key unless E_bc / w_b
 * moves past the threshold.  Package j of cell c draws from counter
 * (j + packet_offset, 0x40000000 | c, draw >> 2, (source << 16) | bin).
 * Writes the packages per bin into per_bin (may be NULL); returns their
 * total, or -1 for a bad argument (cells beyond 2^30). */
int64_t orc_dust_packages(const orc_tree* t, const orc_source* src, int src_index, int n_lambda,
                          const orc_params* prm, int64_t* per_bin);

typedef struct {
  double emitted, absorbed, escaped, rr_gain, rr_loss, killed, peeled;
  double n_packets, n_cross, n_scatter, n_peel_cross, n_killed, n_peel_out;
  double n_split;              /* copies made by package splitting */
} orc_ledger;

/* Trace all packets of all sources.  absorbed [bins][n_cells] and images
 * [n_obs][bins][ny][nx] are accumulated into (caller zeroes).  Optional:
 * sumsq/hits [bins][n_cells] per-packet second moments and packet counts;
 * rec [n_packets][10] per-packet record (w_escaped, n_scatter, n_cross,
 * fate, x_exit[3] cm, d_exit[3]).  Returns 0 or a negative error. */
int orc_trace(const orc_tree* t, int n_src, const orc_source* src, const orc_optics* op,
              const orc_params* prm, const orc_observers* obs, double* absorbed,
              double* images, double* sumsq, double* hits, double* rec, orc_ledger* ledger);

/* Extinction tables of the accelerated peel-off (Sect. 2.4).  The root grid
 * is cut into blocks of `block` root cells per axis; each block face is cut
 * into tiles x tiles tiles.  For observer o and each face of each block
 * through which a ray along dir[o] can leave it (axes a with dir[o][a] != 0;
 * the face on the side the direction points to), the entry is the column
 * density (sum of density x path length, g/cm^3 x root-cell units) from the
 * tile centre along dir[o] to the border of the model; the tile centre is
 * taken on the part of the tile inside the model.  Layout: for o in order,
 * [n_blocks][n_axes(o)][tiles][tiles] (v along axis (a+2)%3, u along
 * (a+1)%3), blocks x-fastest.  A peel-off march then stops where it leaves
 * the block of the scattering point and adds kappa_ext h0 times the entry
 * of the tile it leaves through.  Returns the number of entries (out may be
 * NULL to query it) or a negative error. */
int64_t orc_peel_table(const orc_tree* t, const orc_observers* obs, int block, int tiles, double* out);

/* Single peel-off contribution of a scattering at x (cm) with incoming
 * direction din and weight W, into images [n_obs][bins][ny][nx]. */
int orc_peel_point(const orc_tree* t, const orc_optics* op, const orc_observers* obs, int bin,
                   int per_lambda, const double x_cm[3], const double din[3], double W, double* images);
/* Henyey-Greenstein cosine from one uniform, the phase function (sr^-1) and
 * the rotation of a direction by (mu, phi). */
double orc_hg_mu(double g, double u);
double orc_hg_phase(double g, double mu);
void orc_scatter_dir(const double d[3], double mu, double phi, double out[3]);

/* Dust model (Sects. 3.2 and 4: single-component equilibrium dust). */
typedef struct {
  int n_lambda;
  const double* lambda_um;
  const double* kappa_abs;     /* cm^2/g */
  const double* dnu;           /* Hz */
  double T_min, T_max;
} orc_dust;

/* Emission per unit mass 4 pi sum_i kappa_abs,i B_nu_i(T) dnu_i (erg/s/g). */
double orc_emission_per_mass(const orc_dust* d, double T);
/* Per leaf: solve rho V E(T) = absorbed.  T of refined cells is set to 0. */
int orc_dust_temperature(const orc_tree* t, const double* absorbed_total, const orc_dust* d,
                         int n_threads, double* T);
/* Per leaf and bin: 4 pi rho V kappa_abs,i B_nu_i(T) dnu_i, [n_lambda][n_cells]. */
int orc_dust_emission(const orc_tree* t, const double* T, const orc_dust* d, double* emission);
/* ALI with a per-frequency diagonal operator: per leaf, the T in
 * [T_min, T_max] with sum_b weights[b][c] E_b(T) = rhs[c] (E_b: the cell's
 * emission in bin b; weights = 1 - Lambda_b). */
int orc_dust_temperature_weighted(const orc_tree* t, const double* rhs, const double* weights, const orc_dust* d,
                                  int n_threads, double* T);

#ifdef __cplusplus
}
#endif
#endif
