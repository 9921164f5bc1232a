/*
 * rt.h -- C ABI of librt.so: GB300 (sm_103a) Monte Carlo continuum radiative
 * transfer on hierarchical 2x2x2-refined cartesian grids.
 *
 * Method: Lunttila & Juvela, "Radiative transfer on hierarchial grids".
 * Photon packages are emitted by sources (Sect. 2.3), followed cell by cell
 * through a tree of nested grids (Sect. 2.1) until they leave the outer
 * boundary of the root grid (Sect. 2.3), losing weight by continuous
 * absorption and optionally Russian roulette (Sect. 2.3); after every
 * scattering a peel-off contribution is sent to each observer (Sect. 2.4).
 * Dust temperatures follow from the balance of absorbed and emitted energy
 * (Sects. 3.2 and 4), iterated with the Lambda iteration of Eq. 2.
 *
 * Conventions (all entry points):
 *  - Every call returns an int status: RT_OK or a negative RT_ERR_* code;
 *    rt_last_error() returns a message for the calling thread.
 *  - Host pointers (structs, arrays marked "host") are read only during the
 *    call.  Pointers marked "device" are CUDA device pointers on the
 *    context's device; output device buffers belong to the caller.
 *  - cuda_stream is a cudaStream_t (NULL = legacy default stream).  Kernels
 *    run on that stream; calls that return a ledger wait for their own work
 *    on the stream (bounded by params.timeout_s, RT_ERR_TIMEOUT on expiry).
 *    Results are copied into the context's pinned memory and read only
 *    after the wait succeeded.  After RT_ERR_TIMEOUT the call's kernels keep
 *    running on the stream (they end by themselves, bounded by the step
 *    limit) and still use the context's scratch: until they have finished,
 *    every call on that context returns RT_ERR_BUSY.
 *  - Lengths are cm, densities g/cm^3, opacities cm^2/g (per unit mass).
 *    The model box is [0, box[0]] x [0, box[1]] x [0, box[2]].
 *  - Random numbers: Philox4x32-10 (Salmon et al. 2011) with
 *    key = (seed_lo ^ job, seed_hi ^ iter), counter = (pkt_lo, pkt_hi,
 *    draw >> 2, (source << 16) | bin); draw j of a package is word j & 3.
 *    Dust sources send their packages per cell (Sect. 4.2): every package
 *    of bin b carries w_b (the bin's emission over its packages), and cell c
 *    sends floor(E_bc / w_b + u_bc) of them, u_bc from word 0 of counter
 *    (c, 0x80000000, 0, (source << 16) | b); package j of cell c draws from
 *    counter (j + packet_offset, 0x40000000 | c, draw >> 2, (source << 16) |
 *    b): position in the cell (3 draws), direction (2), then the flight.
 *    A package keeps its random numbers when other cells' emission changes.
 */
#ifndef RT_H
#define RT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  RT_OK = 0,
  RT_ERR_INVALID = -1,    /* bad argument or inconsistent input */
  RT_ERR_OOM = -2,        /* device allocation failed */
  RT_ERR_CUDA = -3,       /* CUDA runtime error */
  RT_ERR_STEP_LIMIT = -4, /* some package hit the per-package step limit */
  RT_ERR_TIMEOUT = -5,    /* bounded wait for the device expired */
  RT_ERR_BUSY = -6        /* server: job does not fit the free budget/slots now;
                             context: an earlier call's timed-out work still runs */
};

typedef struct rt_ctx rt_ctx;
typedef struct rt_grid rt_grid;
typedef struct rt_server rt_server;

/* Create a context on CUDA device `device`.  Owns scratch memory and
 * device-side bookkeeping; one context may be used from one host thread at a
 * time (calls lock it). */
int rt_ctx_create(int device, rt_ctx** out);
void rt_ctx_destroy(rt_ctx* ctx);
/* Peel-off (Sect. 2.4) is deferred: each scattering appends one record
 * (48 B in FP32, 80 B in FP64) to a context-owned device queue, and a second
 * kernel marches every (record, observer) pair after the tracer.  The queue
 * holds min(max_records, 2 x packages of the launch) records (at least 2^20);
 * scatterings beyond it peel off inline in the tracer, with the same
 * results.  max_records = 0 disables deferral, < 0 restores the default
 * (2^27).  Takes effect at the next launch (and at rt_batch_create). */
int rt_ctx_set_peel_queue(rt_ctx* ctx, int64_t max_records);
/* Tiled tracing (the GPU form of the grid-by-grid processing of Sect. 2.2 and
 * App. A): for single-job rt_trace / rt_peel / rt_lambda_iterate launches the
 * root grid is cut into cubic tiles of tile_edge root cells (a power of
 * two); packages are traced in rounds, each round one (wavelength bin, tile)
 * after another, and a package that enters another tile continues in the
 * next round.  Results are those of the untiled tracer (the same package
 * histories; only the order of the FP64 additions differs).  tile_edge < 0:
 * automatic (tiles whose node words plus one bin's accumulators take at most
 * 48 MB, only when the whole grid's take more); 0: off.  Uses two record
 * buffers of up to 2^26 (FP32, 80 B each) or 2^25 (FP64, 144 B each)
 * records.  Returns RT_ERR_INVALID if tile_edge is not a power of two. */
int rt_ctx_set_tiles(rt_ctx* ctx, int tile_edge);
/* Capacity of the tiled tracer's record buffers, in records: the packages of
 * a launch are emitted in chunks of this many records (a quarter of it with
 * resampling) and traced round by round before the next chunk.  <= 0
 * restores the default (2^26 in FP32, 2^25 in FP64); larger values are
 * capped there.  Results do not depend on it (the same package histories);
 * small values let a small launch go through the many-chunk path of a large
 * one. */
int rt_ctx_set_tile_records(rt_ctx* ctx, int64_t max_records);
/* Message of the last failing call on this thread (static storage, valid
 * until the next call on the same thread). */
const char* rt_last_error(void);
/* Library version string. */
const char* rt_version(void);

/* ------------------------------------------------------------------------ */
/* Grid (Sect. 2.1 nested grids; Sect. 2.1 subgrid identification array)     */
/* ------------------------------------------------------------------------ */
/* Level-ordered tree description (host arrays).  Level 0 is the root grid
 * in x-fastest order ix + root[0]*(iy + root[1]*iz).  Level l+1 lists, for
 * each refined level-l cell in order, its 8 children in octant order
 * ox + 2*oy + 4*oz.  refine_flags: 1 byte per cell (1 = refined).
 * density: per cell (values of refined cells are ignored).  n_refined[l]:
 * refined cells on level l (the last level has 0).  Root cells must be
 * cubic: box[a]/root[a] equal on all axes. */
typedef struct {
  int root[3];
  double box[3];
  int n_levels;
  const int64_t* n_refined;
  const uint8_t* refine_flags;
  const double* density;
} rt_tree_desc;

/* Flatten the tree into level-ordered device arrays (structure of arrays):
 * density (f32; refined cells hold the mean of their children), child
 * (u32; 0 = leaf, else index of the first of 8 contiguous children), level
 * (u8), plus the tracer's packed node word (leaf: f32 density / rho_scale,
 * rho_scale = 2^-64 x the densest leaf; refined: 0x80000000 | child) and an
 * f64 density copy.  The library
 * owns the arrays; free with rt_grid_free.  Errors: RT_ERR_INVALID for
 * inconsistent counts, negative/NaN densities, non-cubic cells, more than
 * 2^31 cells or a finest lattice above 2^21 cells per axis; RT_ERR_OOM. */
int rt_build_grid(rt_ctx* ctx, const rt_tree_desc* desc, rt_grid** out);

typedef struct {
  int64_t n_cells, n_leaves;
  int depth;               /* deepest level index */
  int root[3];
  double box[3];
  size_t bytes;            /* device bytes held by the grid */
  const float* density;    /* device [n_cells] */
  const uint32_t* child;   /* device [n_cells] */
  const uint8_t* level;    /* device [n_cells] */
  const uint32_t* node;    /* device [n_cells] packed tracer word */
  const double* density64; /* device [n_cells] */
  const uint64_t* coord;   /* device [n_cells] x | y<<21 | z<<42 at the cell's level */
  double rho_scale;        /* leaf node density = density64 / rho_scale */
} rt_grid_info;
int rt_grid_get_info(const rt_grid* grid, rt_grid_info* out);
void rt_grid_free(rt_grid* grid);

/* New densities for an existing grid, the tree unchanged (Sect. 2.1: the
 * density arrays of the grids; a sequence of models on one mesh, or the same
 * model uploaded again each run).  density: host [n_cells] f64 in the
 * grid's level order, refined cells' values ignored (they get the mean of
 * their children); pinned host memory makes the copy asynchronous.  Work is
 * issued on cuda_stream (NULL = legacy default stream): the upload,
 * validation and densest leaf are read back (the call waits for them and
 * for earlier work on that stream), then the node words are rebuilt
 * stream-ordered; work on other streams that uses the grid must be ordered
 * after the stream by the caller.  Nothing is allocated.  Afterwards the
 * grid's arrays equal those rt_build_grid gives for the same tree and
 * densities.  Errors: RT_ERR_INVALID for NULL arguments, a grid of another
 * context, or a negative, NaN or infinite leaf density (the grid's
 * densities are then undefined until a successful call); RT_ERR_TIMEOUT,
 * RT_ERR_BUSY, RT_ERR_CUDA as for the other calls. */
int rt_grid_set_density(rt_ctx* ctx, rt_grid* grid, const double* density, void* cuda_stream);

/* ------------------------------------------------------------------------ */
/* Tracing (Sects. 2.3, 2.4)                                                 */
/* ------------------------------------------------------------------------ */
typedef struct {
  int n_lambda;            /* 1..256 wavelength bins */
  const double* kappa_ext; /* host [n_lambda], cm^2/g, >= 0 */
  const double* albedo;    /* host [n_lambda], in [0,1] */
  const double* g_hg;      /* host [n_lambda], Henyey-Greenstein g, |g| < 1 */
} rt_optics;

enum {
  RT_SRC_POINT = 0,        /* isotropic point source at pos */
  RT_SRC_EXTERNAL = 1,     /* isotropic external field entering the root box */
  RT_SRC_DUST = 2,         /* thermal dust emission from temperatures T_dev,
                              packages per cell (< 2^30 cells) */
  RT_SRC_BEAM = 3          /* parallel beam from pos along dir */
};

typedef struct {
  int n_lambda;
  const double* lambda_um; /* host [n_lambda] */
  const double* kappa_abs; /* host [n_lambda], cm^2/g; NULL in rt_lambda_iterate /
                              rt_lambda_subiterate: (1 - albedo) kappa_ext of their optics */
  const double* dnu;       /* host [n_lambda], Hz, bin widths */
  double T_min, T_max;     /* K, bracket of the temperature solve */
} rt_dust;

typedef struct {
  int kind;
  double pos[3];            /* cm (point, beam) */
  double dir[3];            /* beam direction (normalised by the library) */
  const double* bin_energy; /* host [n_lambda]: energy per bin (point, external, beam) */
  const double* T_dev;      /* device [n_cells] dust temperatures (dust) */
  const rt_dust* dust;      /* dust model (dust) */
} rt_source;

enum { RT_EST_CONTINUOUS = 0, RT_EST_ANALOG = 1 };

typedef struct {
  uint64_t seed;
  uint32_t job, iter;       /* mixed into the Philox key */
  int precision;            /* 32: f32 geometry + f64 accumulators; 64: f64 throughout */
  int estimator;            /* RT_EST_CONTINUOUS (default) or RT_EST_ANALOG */
  double rr_wmin;           /* roulette when W < rr_wmin * W0 (after a scattering); <= 0 off */
  double rr_p;              /* roulette kill probability */
  int64_t step_limit;       /* max cell segments per package; <= 0: 100000000 */
  double peel_tau_max;      /* stop a peel-off march once tau exceeds this; <= 0 never */
  int per_lambda;           /* 1: outputs per bin; 0: summed over bins */
  int64_t packets_per_bin;  /* > 0: packages for every (source, bin) */
  const int64_t* packets;   /* host [n_src][n_lambda] when packets_per_bin <= 0 and packets_total <= 0 */
  int64_t packets_total;    /* > 0: spread over (source, bin) in proportion to energy */
  double* packet_log_dev;   /* optional device [packet_log_rows][10], one row per package in
                               package order: w_escaped, n_scatter, n_cross, fate (0 escaped,
                               1 roulette, 2 step limit, 3 analog absorption), x_exit[3] (cm),
                               d_exit[3] */
  double timeout_s;         /* bounded wait for completion; <= 0: 3600 s */
  int block_size;           /* 0: tuned default */
  int refill_threshold;     /* 0: tuned default; dead lanes per warp before a refill */
  int blocks_per_sm;        /* 0: occupancy-derived */
  uint32_t* hits_dev;       /* optional device [n_cells]: deposits per cell are ADDED here
                               (continuous estimator, rt_trace only); NULL: not counted */
  int64_t packet_offset;    /* package k of a (source, bin) draws the random stream of package
                               k + packet_offset: launches with offsets 0, n, 2n, ... of n packages
                               each are shards of one run of their total (weights aside) */
  /* Resampling at grid boundaries (Sect. 2.3, Table 1).  The grid of a cell
   * of level l is the octet of its parent (the root grid for l = 0); grid
   * levels are capped at split_max_level.  A package that enters a cell dl
   * levels deeper than its last cell is split into M = split_factor^dl
   * packages of weight W/M at that point and direction (each copy with its
   * own random stream, named by three words the package draws, and a fresh
   * free path); one that enters a cell dl levels shallower survives with
   * probability 1/M and carries M W (booked as roulette gain and loss).
   * The roulette reference W0 follows the weight.  External-field packages
   * start in the root grid, the others in the grid of their first cell.
   * rt_trace / rt_peel of one job only, continuous estimator, no hit counts
   * or level arrays; split_factor^min(split_max_level, depth) <= 256.  Copies
   * are traced in the rounds of the tiled tracer; a split that finds no room
   * in its record buffer is skipped (counted in n_split_skipped). */
  int split_factor;         /* <= 1: off */
  int split_max_level;      /* < 0: the grid's depth */
  /* Polychromatic packages (Sect. 2.3, after Jonsson 2006): 2..8 groups the
   * bins into consecutive groups of poly_group bins (the last may be
   * shorter); a package carries one weight per bin of its group, its path is
   * drawn for the group's reference bin r (bin first + (size - 1) / 2) and
   * each weight carries the likelihood ratio of that path: e^{-(ks_j -
   * ks_r) rho s} along a segment without scattering, ks_j / ks_r at a
   * scattering, p_j(mu) / p_r(mu) for the new direction; a segment deposits
   * W_j ta_j (1 - e^{-x_j}) / x_j with x_j = (ka_j + ks_j - ks_r) rho s and
   * W_j <- W_j e^{-x_j}.  Packages are counted per group (packets_per_bin
   * per group; packets_total in proportion to the group's energy; packets:
   * the entry of the group's first bin); W0_j = E_j / N_group.  The random
   * stream of a group is that of the monochromatic package of its first
   * bin.  Roulette acts on all weights when max_j W_j / W0_j < rr_wmin.
   * One job, point / external / beam sources, continuous estimator, no hit
   * counts, levels, resampling or tabulated peel-off; the group's reference
   * bin must scatter if any bin of the group does; untiled, peel-off inline.
   * The ledger sums the bins; per package its energy balance holds in
   * expectation only (the likelihood ratios change the weights).  <= 1: off. */
  int poly_group;
  /* Rows of packet_log_dev (required with it): a launch whose packages
   * exceed it is refused (RT_ERR_INVALID) before anything runs.  A dust
   * source's package count depends on the emission (within one per emitting
   * cell and bin of the budget), so give its log room beyond the budget. */
  int64_t packet_log_rows;
  /* FP32 tracing: a near-vacuum cell, whose extinction per unit length lies
   * below the f32 normal range (about 1e-43 of the densest leaf's), takes
   * its deposit from the f64 density in the thin limit q = x instead of
   * none, so its temperature follows from its absorbed energy per unit mass
   * as in FP64.  Costs a read of the f64 density and FP64 arithmetic per
   * such crossing (the 9.2e6-cell disc traces 30 % slower).  0: off. */
  int thin_f64;
} rt_trace_params;

typedef struct {
  double emitted, absorbed, escaped, rr_gain, rr_loss, killed, peeled;
  uint64_t n_packets, n_cross, n_scatter, n_peel_cross, n_killed, n_peel_out;
  uint64_t n_peel_deferred; /* scatterings whose peel-off ran in the deferred peel-off kernel */
  int status;               /* RT_OK or RT_ERR_STEP_LIMIT */
  double kernel_ms;         /* device time of the tracer launch */
  double peel_ms;           /* device time of the deferred peel-off launch (0: none) */
  int64_t n_launches;       /* kernel launches of the call (tracer rounds, record sorts, peel-off) */
  int32_t n_tiles;          /* tiled tracing: tiles (0: untiled) */
  int32_t n_rounds;         /* tiled tracing: rounds after the emission round */
  uint64_t n_split;         /* resampling: copies made */
  uint64_t n_split_skipped; /* resampling: splits skipped for lack of record space */
} rt_ledger;

/* Trace every package of every source and accumulate the absorbed energy
 * per cell: absorbed_dev (device, [bins][n_cells] f64, bins = n_lambda if
 * per_lambda else 1) is ADDED to (zero it first).  The ledger (host, may be
 * NULL) receives the energy balance and counters.  Returns RT_OK,
 * RT_ERR_STEP_LIMIT if a package was killed by the step limit (results are
 * still written), or an error. */
int rt_trace(rt_ctx* ctx, const rt_grid* grid, int n_src, const rt_source* src,
             const rt_optics* optics, const rt_trace_params* params, double* absorbed_dev,
             rt_ledger* ledger, void* cuda_stream);

/* Observers for peel-off images (Sect. 2.4): orthographic projection
 * centred on the box centre; pixel (ix, iy) covers
 * [(ix - nx/2) fov[0]/nx, ...) along ex = normalise(up x dir), ey = dir x ex. */
typedef struct {
  int n_obs;               /* 1..16 */
  const double* dir;       /* host [n_obs][3] unit vectors towards the observers */
  const double* up;        /* host [n_obs][3] */
  int nx, ny;
  double fov[2];           /* cm */
} rt_observers;

/* As rt_trace, and after every scattering peel off W p_HG(mu) exp(-tau) to
 * each observer into images_dev (device, [n_obs][bins][ny][nx] f64, added
 * to).  absorbed_dev may be NULL. */
int rt_peel(rt_ctx* ctx, const rt_grid* grid, int n_src, const rt_source* src,
            const rt_optics* optics, const rt_trace_params* params, const rt_observers* obs,
            double* images_dev, double* absorbed_dev, rt_ledger* ledger, void* cuda_stream);

/* Accelerated peel-off (Sect. 2.4): before the simulation, the faces of
 * blocks of block_edge^3 root cells are cut into tiles_per_edge^2 tiles, and
 * for each observer the column density (sum of density x path length) from
 * every tile centre (of the part of the tile inside the model) along the
 * observer direction to the border of the model is stored, for the block
 * faces a ray along that direction can leave through.  A peel-off march then
 * follows the optical depth exactly only until it leaves the block of the
 * scattering point and adds kappa_ext times the entry of the tile it leaves
 * through: an approximation (the tile centre stands in for the exit point)
 * that is exact for observers along an axis on grids whose cells are not
 * refined below the tile size.  block_edge and tiles_per_edge are powers of
 * two, at most 1024 blocks per axis; the tables (FP64, device memory owned
 * by the returned object) take 8 bytes x observers x blocks x exit axes x
 * tiles_per_edge^2 and are built on `cuda_stream` (FP64 marches).  The
 * object refers to `grid`, which must outlive it. */
typedef struct rt_peel_tables rt_peel_tables;
int rt_peel_tables_create(rt_ctx* ctx, const rt_grid* grid, const rt_observers* obs, int block_edge,
                          int tiles_per_edge, rt_peel_tables** out, void* cuda_stream);
void rt_peel_tables_destroy(rt_peel_tables* tables);
/* Number of table entries; rt_peel_tables_read copies them to host memory
 * (n >= that number) in the layout: observers in order, then
 * [blocks x-fastest][exit axes in x, y, z order][v along axis (a+2)%3][u along (a+1)%3]. */
int64_t rt_peel_tables_size(const rt_peel_tables* tables);
int rt_peel_tables_read(const rt_peel_tables* tables, double* host, int64_t n);
/* rt_peel with the tables (same grid, same observer directions as at
 * creation, else RT_ERR_INVALID).  Scatterings that do not fit the deferred
 * peel-off queue are peeled off inline with exact marches. */
int rt_peel_tabulated(rt_ctx* ctx, const rt_grid* grid, int n_src, const rt_source* src,
                      const rt_optics* optics, const rt_trace_params* params, const rt_observers* obs,
                      const rt_peel_tables* tables, double* images_dev, double* absorbed_dev,
                      rt_ledger* ledger, void* cuda_stream);

/* ------------------------------------------------------------------------ */
/* Batches: many models in one persistent launch                            */
/* ------------------------------------------------------------------------ */
/* One job = one model traced (and optionally peeled off) exactly as rt_trace
 * / rt_peel would; a batch runs all jobs in one persistent launch that
 * shares the package counter, so short and long jobs keep every SM busy.
 * All jobs must use the same precision and estimator; the launch settings
 * (block size, refill threshold) are taken from the first job's params. */
typedef struct {
  const rt_grid* grid;
  int n_src;
  const rt_source* src;
  const rt_optics* optics;
  const rt_trace_params* params;
  const rt_observers* obs;  /* NULL: no images */
  double* images_dev;       /* device, as rt_peel (added to) */
  double* absorbed_dev;     /* device, as rt_trace (added to); may be NULL */
} rt_job;

/* One-shot batched launch; ledgers: host [n_jobs] (may be NULL). */
int rt_trace_batch(rt_ctx* ctx, int n_jobs, const rt_job* jobs, rt_ledger* ledgers, void* cuda_stream);

/* A batch prepared once and replayed: the job table (and any dust emission
 * tables, from the temperatures at creation) is uploaded into memory owned
 * by the batch, and one CUDA graph holds the zeroing of every job's outputs,
 * the ledger reset, the persistent tracer launch and the ledger read-back.
 * rt_batch_run replays it on `cuda_stream` and waits (bounded). */
typedef struct rt_batch rt_batch;
int rt_batch_create(rt_ctx* ctx, int n_jobs, const rt_job* jobs, rt_batch** out);
int rt_batch_run(rt_batch* batch, rt_ledger* ledgers, double timeout_s, void* cuda_stream);
void rt_batch_destroy(rt_batch* batch);

/* Autotuner: runs the jobs with their package counts scaled by
 * sample_fraction under every block size {128, 256} x refill threshold
 * {2, 4, 8, 12, 16}, keeps the fastest (cell crossings per ms) as the
 * context's default for this precision and peel-off mode, and zeroes the
 * jobs' outputs afterwards.  rt_tune_save / rt_tune_load persist the choices
 * per GPU architecture in a text file. */
typedef struct {
  int block_size, refill_threshold, blocks_per_sm;
  double crossings_per_ms;
} rt_tune_result;
int rt_autotune(rt_ctx* ctx, int n_jobs, const rt_job* jobs, double sample_fraction, rt_tune_result* best);
int rt_tune_save(const rt_ctx* ctx, const char* path);
int rt_tune_load(rt_ctx* ctx, const char* path);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching with admission by device-memory footprint    */
/* ------------------------------------------------------------------------ */
/* Models (density trees) are registered once by id; their grids are built on
 * first use and stay resident on the device until memory is needed (least
 * recently used first, never while a running job uses them).  A request is
 * admitted, in arrival order, when its footprint -- its grid unless resident
 * plus its accumulators -- fits the free part of hbm_budget.  max_slots
 * dispatcher threads, each with its own context and stream, run the
 * admitted requests in arrival order as batched persistent launches: a free
 * slot takes the next request and, after waiting batch_window_ms for
 * company, the requests behind it while the launch holds at most
 * max_batch_jobs jobs and max_batch_packets packages (a request larger than
 * that runs alone); requests arriving meanwhile join the next launch of
 * whichever slot frees first, so the slots' work overlaps on the device.
 * Results stay on the device (counted in the budget) until
 * rt_server_fetch. */
typedef struct {
  size_t hbm_budget;
  int max_slots;          /* 1..16 */
  int max_batch_jobs;
  double batch_window_ms;
  int64_t max_batch_packets; /* <= 0: no limit */
} rt_server_config;

typedef struct {
  uint64_t model_id;
  int n_src;
  const rt_source* src;   /* point, external or beam */
  const rt_optics* optics;
  const rt_trace_params* params;
  const rt_observers* obs; /* NULL: no images */
} rt_serve_job;

int rt_server_create(rt_ctx* ctx, const rt_server_config* cfg, rt_server** out);
/* Host tree copied; RT_ERR_INVALID if the id exists. */
int rt_server_add_model(rt_server* srv, uint64_t model_id, const rt_tree_desc* tree);
/* Queues a request (host data copied); RT_ERR_BUSY if it can never fit. */
int rt_server_submit(rt_server* srv, const rt_serve_job* job, uint64_t* ticket);
/* done = 1 once finished; latency_ms = submit to completion of its launch. */
int rt_server_poll(rt_server* srv, uint64_t ticket, int* done, rt_ledger* ledger, double* latency_ms);
int rt_server_wait(rt_server* srv, uint64_t ticket, double timeout_s);
/* Device time of the launch a finished request ran in, in ms after the
 * server's creation (CUDA events around the slot's launch): launches of
 * different slots whose intervals intersect ran on the device at the same
 * time.  -1 for a request not run (yet). */
int rt_server_job_times(rt_server* srv, uint64_t ticket, double* t_start_ms, double* t_end_ms);
/* Copies results to host arrays (either may be NULL) and releases the job. */
int rt_server_fetch(rt_server* srv, uint64_t ticket, double* absorbed_host, double* images_host);
int rt_server_stats(rt_server* srv, size_t* used_bytes, int* queued, int* running);
void rt_server_destroy(rt_server* srv);

/* ------------------------------------------------------------------------ */
/* Dust (Sects. 3.2, 4)                                                      */
/* ------------------------------------------------------------------------ */
/* Per leaf: solve rho V 4 pi sum_i kappa_abs,i B_nu_i(T) dnu_i = A for T in
 * [T_min, T_max] (clamped), A = sum over n_bins rows of absorbed_dev
 * (device [n_bins][n_cells]).  T_dev (device [n_cells]) receives T; refined
 * cells get 0.  FP64 safeguarded Newton on a tabulated bracket. */
int rt_dust_temperature(rt_ctx* ctx, const rt_grid* grid, const double* absorbed_dev, int n_bins,
                        const rt_dust* dust, double* T_dev, void* cuda_stream);

/* Lambda iteration (Eq. 2): J_{n+1} = Lambda S_n + J_0, S_{n+1} = f(J_{n+1}).
 * The field of the constant sources (`src`, e.g. a star) is traced once and
 * stored (Sect. 3.2); each iteration re-emits the dust with the current
 * temperatures (packages per bin in proportion to the bin emission, Sect. 4.2,
 * or an equal count), traces them and solves the new temperatures from the
 * sum of both fields.  The dust packages reuse the same random streams in
 * every iteration (key iter = params.iter + 1), and a package stays with its
 * cell (packages are sent per cell), so the change in T measures
 * convergence rather than Monte Carlo noise.  Stops when max |dT|/T over
 * leaves with at least min_hits deposits (counted during the constant-source
 * trace and the first dust trace) falls below tol, or after max_iter
 * iterations (the disc test of Sect. 4.2 stops at 30). */
typedef struct {
  int max_iter;                  /* 1..64 */
  double tol;                    /* stop threshold on max |dT|/T; 0: run max_iter */
  double min_hits;               /* cells with fewer deposits are left out of the stop rule */
  int64_t dust_packets_total;    /* packages per dust trace, spread over bins by emission */
  int64_t dust_packets_per_bin;  /* > 0: this many per bin instead */
} rt_lambda_params;

typedef struct {
  int n_iter;                    /* iterations taken */
  double history[64];            /* max |dT|/T after iteration i+1 */
  rt_ledger source_ledger;       /* the constant-source trace */
  rt_ledger dust_ledger;         /* the last dust trace */
  double ms;                     /* wall time of the whole iteration */
} rt_lambda_result;

/* src/params: the constant sources and their trace parameters (precision,
 * roulette, packages); dust: the dust model (same bins as optics); T_dev
 * (device [n_cells]) receives the final temperatures.  Library scratch:
 * three f64 and one u32 array of n_cells. */
int rt_lambda_iterate(rt_ctx* ctx, const rt_grid* grid, int n_src, const rt_source* src,
                      const rt_optics* optics, const rt_dust* dust, const rt_trace_params* params,
                      const rt_lambda_params* lp, double* T_dev, rt_lambda_result* result,
                      void* cuda_stream);

/* Lambda iteration with subiterations (Sect. 3.2, App. B).  The grid of a
 * cell at level l is the set of 8 children of its parent (the root grid for
 * l = 0); a package remembers the shallowest grid level it has reached (the
 * level of its emission cell at first; one below the deepest common
 * ancestor at every crossing out of a parent octet).  The dust field is kept
 * in one array per level (Eq. 9: a cell's field is the constant sources' plus
 * all its level arrays).  A step is
 *   full (0): dust emitted by every cell, all level arrays replaced;
 *   sub  (1): a subiteration of every subtree below the refined cells of level
 *             sub_level = L: dust emitted by the cells of level > L, packages
 *             leave the run where they reach a grid of level <= L (booked as
 *             escaped), the level arrays > L replaced.
 * A subiteration sends from each cell the packages a full step would, with
 * the same random streams: the package energy w_b is the full step's (the
 * whole model's emission in bin b over its packages).
 * After each step T follows from the summed field.  The dust packages reuse
 * the same random streams every step (key iter = params.iter + 1).  With an
 * explicit schedule the steps run as given (the run stops early when max
 * dT/T over cells with >= lp->min_hits hits drops below lp->tol); with
 * n_steps = 0, lp->max_iter steps are chosen automatically from the energy
 * balance (Sect. 3.3): the first step is full; then a full step whenever the
 * mass-weighted mean |absorbed - emitted| of the leaves at level <= L
 * (measured at the last full step) is at least select_frac times the larger
 * of it and that of the leaves below L (measured every step), or when the
 * dust emission below L has changed by flux_frac since the last full step
 * (Sect. 3.3: the flux a grid receives from its children has changed), else
 * a subiteration.  Library scratch: 7 f64 + 3 u32 arrays of n_cells and 2 f64
 * arrays of n_levels x n_cells. */
typedef struct {
  int sub_level;           /* L: subiterations cover the subtrees below the refined cells of level L */
  int n_steps;             /* > 0: explicit schedule of this length (<= 64); 0: automatic */
  const int* schedule;     /* host [n_steps]: 0 full step, 1 subiteration */
  double select_frac;      /* automatic choice threshold (0.25 in Sect. 4.2) */
  double flux_frac;        /* automatic: also a full step once the emission below L has changed by this
                              fraction since the last full step (the upper levels' field from below
                              is stale); <= 0: off */
  int ali;                 /* 1: accelerated Lambda iteration with the diagonal operator (Eq. 3), per
                              frequency bin b: each step tallies per cell and bin the energy its dust
                              packages leave in it (self_b) and the energy they carried (emitted_b),
                              and per cell their number; Lambda_b = self_b / emitted_b (capped at
                              ali_max_lambda) and T solves sum_b (1 - Lambda_b) E_b(T) =
                              A - sum_b Lambda_b emitted_b in the cells that sent at least
                              ali_min_packages packages; a bin such a cell did not sample takes the
                              largest Lambda_j of its sampled bins with kappa_abs,j <= kappa_abs,b
                              (0 if none); the other cells take the plain step */
  int ali_min_packages;    /* <= 1: every cell that sent a package */
  double ali_max_lambda;   /* cap of Lambda_b (it bounds the amplification 1 / (1 - Lambda_b) of the
                              cell's incoming field); outside (0, 1): 0.999 */
} rt_subiter_params;

typedef struct {
  rt_lambda_result lambda;       /* steps taken, max dT/T per step, ledgers, wall time */
  int step_kind[64];             /* 0 full, 1 subiteration */
  double imbalance[64][2];       /* after each step: mean |absorbed - emitted| per unit mass, levels <= L and > L */
  double step_ms[64];            /* wall time of each step */
} rt_subiter_result;

int rt_lambda_subiterate(rt_ctx* ctx, const rt_grid* grid, int n_src, const rt_source* src,
                         const rt_optics* optics, const rt_dust* dust, const rt_trace_params* params,
                         const rt_lambda_params* lp, const rt_subiter_params* sp, double* T_dev,
                         rt_subiter_result* result, void* cuda_stream);

/* Dust emission per leaf and bin, 4 pi rho V kappa_abs,i B_nu_i(T) dnu_i,
 * into emission_dev (device [n_lambda][n_cells]); bin totals to
 * bin_total_host (host [n_lambda], may be NULL; waits for the stream). */
int rt_dust_emission(rt_ctx* ctx, const rt_grid* grid, const double* T_dev, const rt_dust* dust,
                     double* emission_dev, double* bin_total_host, void* cuda_stream);

/* Hierarchical model built bottom-up from a full-resolution cube (Sect. 4.1:
 * cells are combined while the combined cell's V-band optical thickness is
 * <= 0.05 and the density contrast of the cells combined is < 30).
 * rho_dev: device [nz][ny][nx] f64 densities (g/cm^3, x fastest) with
 * n = root[i] * 2^n_fine_levels cells per axis; box: model size (cm, cubic
 * cells).  Eight cells of level l+1 are combined into their parent when all
 * eight are undivided, kappa * rho_mean * h_l <= tau_max (kappa: cm^2/g,
 * h_l: the parent's size) and rho_max < contrast_max * rho_min over the
 * full-resolution cells the parent covers (rho_min = 0: only if rho_max =
 * 0); the parent's density is the mean of the eight, added in octant order
 * o = ox + 2 oy + 4 oz.  Output (caller-owned host arrays): the level-ordered
 * description rt_build_grid takes -- refine_flags / density [cap_cells]
 * (root cells x-fastest, then the children of each divided cell in the
 * order of their parents, in octant order), n_refined [n_fine_levels + 1]
 * (divided cells per level), n_levels_out, n_cells_out.  If the
 * description has more than cap_cells cells nothing past cap_cells is
 * written, n_cells_out holds the size needed and the call returns
 * RT_ERR_INVALID.  Device scratch is allocated and freed inside the call
 * (~1.3 x the cube's bytes).  Synchronises the stream. */
int rt_merge_uniform(rt_ctx* ctx, const int* root, const double* box, int n_fine_levels, const double* rho_dev,
                     double kappa, double tau_max, double contrast_max, int64_t cap_cells,
                     uint8_t* refine_flags_host, double* density_host, int64_t* n_refined_host, int* n_levels_out,
                     int64_t* n_cells_out, void* cuda_stream);

/* ------------------------------------------------------------------------ */
/* Diagnostics used by the parity tests                                      */
/* ------------------------------------------------------------------------ */
/* Deterministic walks (Sect. 2.3 cell stepping) of n_rays rays with the
 * tracer's own stepping code.  origins/dirs: device [n_rays][3] f64 (cm;
 * converted to the working precision).  Outputs (device): cells
 * [n_rays][max_seg] int64, lengths [n_rays][max_seg] f64 (cm), counts
 * [n_rays] int64 (segments of positive length; -1 if the origin is outside). */
int rt_walk(rt_ctx* ctx, const rt_grid* grid, int64_t n_rays, const double* origins_dev,
            const double* dirs_dev, int precision, int64_t max_seg, int64_t* cells_dev,
            double* lengths_dev, int64_t* counts_dev, void* cuda_stream);

/* L2 read bandwidth in GB/s (diagnostic for the rooflines of L2-resident
 * work; no counterpart in the paper): buf_dev is a zeroed device buffer of
 * `bytes` (16-byte aligned, smaller than the L2), read `reps` times per
 * launch with 16-byte loads cached in L2 only; best of 5 timed launches
 * after one warm-up launch. */
int rt_l2_read_bandwidth(rt_ctx* ctx, void* buf_dev, int64_t bytes, int reps, double* gbs, void* cuda_stream);

/* Diagnostic: node descents since the last reset, counts[0] in the tracers'
 * own walks, counts[1] in peel-off marches; a descent is a global read of an
 * interior cell's child word (the 4 B per descent of the roofline unit).
 * Only builds compiled with RT_COUNT_DESCENTS=1 count (an atomic per
 * descent; the crossings and histories are those of the normal build);
 * others answer RT_ERR_INVALID.  Waits for the device; reset != 0 zeroes the
 * counters after reading.  counts: host [2]. */
int rt_descent_counts(rt_ctx* ctx, uint64_t* counts, int reset);

/* Philox4x32-10 blocks for n (counter, key) pairs: ctr_dev [n][4], key_dev
 * [n][2], out_dev [n][4] (device uint32). */
int rt_philox(rt_ctx* ctx, int64_t n, const uint32_t* ctr_dev, const uint32_t* key_dev,
              uint32_t* out_dev, void* cuda_stream);

/* ------------------------------------------------------------------------ */
/* Allocation-free tracing (no counterpart in the paper)                     */
/* ------------------------------------------------------------------------ */
/* rt_trace without a context and without any device allocation, for callers
 * that cannot let a library call cudaMalloc: applications whose device memory
 * is owned by their own pool or caching allocator, and latency-critical code
 * that cannot take the device synchronisation of cudaMalloc/cudaFree.  The
 * tracer's scratch (job table, ledger, package counter) lives in a 64 KiB
 * file-scope __device__ array that every GPU loading the library holds until
 * the process exits.  The caller passes the grid (built beforehand with
 * rt_build_grid), sources, optics, params and the output array exactly as for
 * rt_trace; the result is the same.  Limits (RT_ERR_INVALID beyond them):
 * 1..4 sources, 1..256 wavelength bins, point/external/beam sources only (a
 * dust source needs a cumulative-emission table larger than the scratch),
 * no observers.  The first call on a device looks up the scratch address
 * (cudaGetSymbolAddress) with that device current.  The call cannot be made
 * on a stream that is capturing a graph (RT_ERR_INVALID): it uploads the job
 * table from host memory, polls the stream and reads the ledger back.  It
 * waits (bounded by params->timeout_s) for the earlier work on the stream
 * before the upload and for its kernel after the launch; on RT_ERR_TIMEOUT
 * the kernel is still running and still uses the scratch, and the ledger is
 * not filled.  The scratch is cleared at the start of every call and shared
 * by all calls, which are serialised on the host: calls whose work overlaps
 * on the GPU (several streams, or a call after a timeout on another stream
 * before the first one's kernel finished) race on it and must be ordered by
 * the caller.  The host side uses a static staging area, not the stack.
 * ledger->kernel_ms is 0 (no timing events). */
int rt_trace_noalloc(const rt_grid* grid, int n_src, const rt_source* src, const rt_optics* optics,
                     const rt_trace_params* params, double* absorbed_dev, rt_ledger* ledger,
                     void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
