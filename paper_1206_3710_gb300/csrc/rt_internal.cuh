// rt_internal.cuh -- device-side data layout shared by the library's .cu files.
//
// The grid lives in HBM as level-ordered arrays (Sect. 2.1 nested grids,
// octree case).  The tracer reads one 32-bit word per cell visit: a leaf
// holds its density as a non-negative f32 (scaled by 1/rho_scale), a refined
// cell holds 0x80000000 | index-of-first-child.  This folds the "subgrid
// identification array" of Sect. 2.1 into the density array, as the
// footnote of Sect. 3.4 suggests.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include "rt.h"

#define RT_MAX_OBS 16
#define RT_MAX_LAMBDA 256
#define RT_INTERIOR 0x80000000u
#define RT_CHILD_MASK 0x7FFFFFFFu
#define RT_COORD_BITS 21
#define RT_COORD_MASK ((1ull << RT_COORD_BITS) - 1ull)

// per wavelength bin optics, scaled to the tracer's units
struct BinDev {
  double kext_d;   // kappa_ext * h0 (multiplies f64 density), per root-cell unit
  float kext_f;    // kappa_ext * h0 * rho_scale (multiplies the node's f32 density)
  float albedo;
  float g;
  float pad;
  double albedo_d, g_d;
};

// observer, in root-cell units
struct ObsDev {
  double k[3], ex[3], ey[3];
  double c[3];        // box centre
  double inv_pix[2];  // 1 / pixel size
  float kf[3], exf[3], eyf[3], cf[3], inv_pixf[2];  // the same in f32
  int nx, ny;
  // accelerated peel-off tables (Sect. 2.4): this observer's entries start
  // at tab_off; tab_slot[a] is the slot of axis a among its exit axes
  long long tab_off;
  int tab_slot[3];
  int tab_naxes;
};

struct LedgerDev {
  double emitted, absorbed, escaped, rr_gain, rr_loss, killed, peeled;
  unsigned long long n_packets, n_cross, n_scatter, n_peel_cross, n_killed, n_peel_out, n_peel_deferred;
  unsigned long long n_split, n_split_skipped;
  int status;
  int pad;
};

// Deferred peel-off (Sect. 2.4): at a scattering the tracer appends the
// scattering point, incoming direction and weight to a queue; a second
// kernel marches every (record, observer) pair to the grid edge.  The
// tracer's lanes then all trace, and the marches run in a kernel of their
// own.  meta = level | bin << 5 | job << 13.
struct PeelRec32 {
  uint32_t cx, cy, cz, idx;
  float fx, fy, fz, W;
  float dx, dy, dz;
  uint32_t meta;
};
struct PeelRec64 {
  uint32_t cx, cy, cz, idx;
  double fx, fy, fz, W;
  double dx, dy, dz;
  uint32_t meta, pad;
};
#define RT_PEEL_MAX_JOBS (1 << 19)

// Tiled tracing, the GPU form of the grid-by-grid processing of Sect. 2.2
// (App. A): the root grid is cut into tiles of 2^tsh root cells per axis.
// Packages are emitted into records, sorted by (bin, tile), and traced in
// rounds; a package that crosses into another tile is written back to a
// record for the next round, so the cells touched at any time belong to a
// few (bin, tile) pairs whose node words and accumulators stay in L2.
//
// aux = mlev | (plev + 1) << 8 | (sexp + 128) << 16: the subiterations'
// shallowest grid level, the resampling's grid level of the last cell (-1:
// none yet) and its split exponent (the weight reference W0 is the
// package's emitted W0 times split_factor^-sexp).  The wide records, used
// by the subiteration and resampling tracers, add the ALI emission cell and
// the random stream of a split copy (s3 bit 31 set; else the stream follows
// from gi).
struct TRec32 {
  uint32_t cx, cy, cz, meta;  // lattice coordinates at level; meta = lev | bin << 5 | job << 13
  float fx, fy, fz, W;
  float dx, dy, dz, tau;
  float pkt_abs;
  uint32_t next, nscat, ncross;
  unsigned long long gi;      // package index in the launch's package counter
  uint32_t npeel, aux;
};
struct TRec32W {
  TRec32 b;
  uint32_t orig, s0, s1, s3;
};
struct TRec64 {
  uint32_t cx, cy, cz, meta;
  double fx, fy, fz, W;
  double dx, dy, dz, tau;
  double pkt_abs;
  uint32_t next, nscat, ncross, npeel;
  unsigned long long gi;
  uint32_t aux, orig, s0, s1, s3, pad0;
  unsigned long long pad1;
};
struct TileRun {
  const void* in;               // run: records sorted by key
  void* out;                    // emit/run: records written for the next round
  uint32_t* out_key;            // their keys: bin * n_tiles + tile
  unsigned long long* n_out;    // records written
  long long cap_out;
  long long first;              // emit: index of the first package of the chunk
  int tsh, ntx, nty, n_tiles;
  int* status;                  // bit 0: record buffer overflow
  unsigned long long* n_split;  // resampling: copies written this round
  long long split_cap;          // resampling: copies the record buffer has room for this round
  int sbits;                    // records are also sorted by 2^sbits-per-axis blocks within a tile
  int pad;
};
struct PeelQueue {
  void* rec;                    // PeelRec32 or PeelRec64 [cap]
  unsigned long long* count;    // records requested (may exceed cap: the rest peel inline)
  long long cap;                // 0: no queue, every peel-off inline
};

struct JobDev {
  const uint32_t* node;
  const double* rho64;
  const uint64_t* coord;
  const uint8_t* level;
  uint32_t root[3];
  int depth;
  double h0;
  int n_lambda;
  int estimator;
  const BinDev* bins;
  long long n_cells;
  double* absorbed;
  int abs_bins;     // n_lambda or 1
  int img_bins;
  double* images;
  int n_obs;
  int pad0;
  const ObsDev* obs;
  LedgerDev* ledger;
  double* packet_log;
  unsigned long long seed;
  uint32_t job_id, iter;
  double rr_wmin, rr_p;
  long long step_limit;
  double peel_tau_max;
  unsigned int* hits;  // optional deposits per cell
  // f32 copies for the f32 tracer (GB300's FP64 pipe is narrow)
  float rr_wmin_f, rr_p_f, peel_tau_max_f;
  // the f32 tracer books ledger energies in 64-bit fixed point: value * 2^led_shift
  int led_shift;
  int thin64;  // f32 tracer: near-vacuum cells' deposits from the f64 density
  long long pkt_offset;  // added to the package index of the random streams
  // accelerated peel-off: column densities on block faces (NULL: exact
  // marches); blocks of 2^ptab_bsh root cells, 2^ptab_ssh tiles per face edge
  const double* ptab;
  int ptab_bsh, ptab_ssh, ptab_nbx, ptab_nby;
  // subiterations (Sect. 3.2, App. B): absorbed is [n_levels][n_cells] and a
  // deposit goes to the shallowest grid level the package has reached; a
  // package that reaches a grid of level <= sub_conf leaves the run
  int sub_conf;
  int pad2;
  // resampling at grid boundaries (Sect. 2.3): split factor (<= 1: off) and
  // the level at which grid levels are capped
  int split_n;
  int split_lmax;
  // polychromatic packages: bins per group (1: monochromatic)
  int poly_n;
  int pad3;
  // ALI (Eq. 3): energy a dust package leaves in its own emission cell, per
  // bin and cell [n_lambda][n_cells] (the diagonal of Lambda per
  // frequency), and the energy of the dust packages each cell emitted in
  // each bin; NULL: not tallied
  double* self_abs;
  double* self_emit;
  unsigned int* self_cnt;  // dust packages emitted per cell
};

// one (job, source) work item: a contiguous range of the global package counter
struct ItemDev {
  long long pkt_begin, pkt_end;
  long long log_offset;
  int job;
  int kind;
  uint32_t src_index;
  int pad;
  double pos[3];   // root-cell units
  double dir[3];
  const long long* bin_prefix;  // [n_lambda + 1] package prefix within the item
  const double* W0;             // [n_lambda]
  const long long* dust_first;  // dust: [n_lambda][n_cells + 1] first package of each cell
  const float* W0f;             // [n_lambda] f32 copy of W0
  float posf[3], dirf[3];       // f32 copies of pos, dir
  int pad2;
};

// Fixed-point scale of a job's ledger in the f32 tracer: the largest value a
// single booking can carry is bounded by the largest package weight, times
// the roulette survival gain; 40 fractional bits below that bound leave 24
// bits of headroom for the sum of a warp's bookings.
inline int ledger_shift(double w0_max, double rr_wmin, double rr_p) {
  double bound = w0_max;
  if (rr_wmin > 0.0 && rr_p < 1.0) bound *= std::max(1.0, rr_wmin / (1.0 - rr_p));
  if (!(bound > 0.0) || !std::isfinite(bound)) return 0;
  return 40 - (std::ilogb(bound) + 2);
}

// ------------------------------------------------------------------------
// host-side helpers implemented in rt_trace.cu / rt_dust.cu / rt_grid.cu
// ------------------------------------------------------------------------
namespace rtk {

// levels of the path above a leaf a tracer lane keeps in shared memory (a
// crossing out of a deeper octet re-descends from the root cell)
#define RT_ANC_MAX 12

struct LaunchCfg {
  int block;
  int blocks;        // grid of the untiled and emission launches
  int refill;
  int blocks_tiled;  // grid of the tiled rounds (their tracer is sized for fewer blocks per SM)
  int anc = 0;       // levels of the stored path per lane (0..RT_ANC_MAX): the grids' depth
};

// launch the persistent tracer over n_items items of total packages;
// mode 0 plain, 1 emit into tile records (packages [T.first, total)),
// 2 trace the records T.in[0, total) within their tiles
cudaError_t launch_trace(int precision, bool peel, int estimator, bool hits, const JobDev* jobs_dev,
                         const ItemDev* items_dev, int n_items, unsigned long long* counter_dev,
                         long long total, const LaunchCfg& cfg, const PeelQueue& q, cudaStream_t s,
                         int mode = 0, const TileRun* tiles = nullptr, bool levels = false, bool split = false);
size_t tile_record_bytes(int precision, bool wide);
// polychromatic tracer (groups of 2..8 bins), one job
cudaError_t launch_poly(int precision, int group, bool peel, const JobDev* jobs, const ItemDev* items, int n_items,
                        unsigned long long* counter, long long total, int sm_count, cudaStream_t s);
// counting sort of n records (rec_bytes each) by key (< n_keys) from in/key
// into out; hist_dev holds n_keys + 1 counters
cudaError_t tile_sort(const void* in, const uint32_t* key, long long n, int rec_bytes, int n_keys,
                      unsigned long long* hist_dev, void* out, cudaStream_t s);
cudaError_t trace_occupancy(int precision, bool peel, int block, int* blocks_per_sm, int mode = 0, int anc = 0);
// march the queued peel-off records (n_obs_max observers each); work_dev is a
// zeroed counter
cudaError_t launch_peel(int precision, const JobDev* jobs_dev, const PeelQueue& q, unsigned long long* work_dev,
                        int n_obs_max, int refill, cudaStream_t s, int anc = 0);
size_t peel_record_bytes(int precision);
// node-descent counters of builds compiled with RT_COUNT_DESCENTS=1
bool descents_counted();
cudaError_t descent_counts(unsigned long long out[2], bool reset);
// sort keys of n queued peel-off records: block of 2^bs root cells (x fastest)
cudaError_t peel_keys(int precision, const void* rec, long long n, int bs, int nbx, int nby, int nbz, uint32_t* key,
                      int sm_count, cudaStream_t s);
// peel-off kernel with the extinction tables of JobDev::ptab
cudaError_t launch_peel_tab(int precision, const JobDev* jobs_dev, const PeelQueue& q, unsigned long long* work_dev,
                            int n_obs_max, int refill, cudaStream_t s, int anc = 0);
// the extinction tables: column density from each block-face tile centre
// along each observer direction to the border of the model (FP64 marches)
struct PeelTabSpec {
  int n_obs;
  double k[RT_MAX_OBS][3];
  long long off[RT_MAX_OBS + 1];
  int axes[RT_MAX_OBS][3];  // exit axes of observer o, n_axes[o] of them
  int n_axes[RT_MAX_OBS];
  int block, tiles, nb[3];
};
cudaError_t build_peel_table(const JobDev* job_dev, const PeelTabSpec& spec, double* table, cudaStream_t s);

cudaError_t launch_walk(int precision, const JobDev* job_dev, long long n_rays, const double* origins,
                        const double* dirs, long long max_seg, long long* cells, double* lengths,
                        long long* counts, cudaStream_t s);
cudaError_t launch_philox(long long n, const uint32_t* ctr, const uint32_t* key, uint32_t* out,
                          cudaStream_t s);
// reads a zeroed device buffer `reps` times through L2 (bandwidth diagnostic)
cudaError_t launch_l2_read(const void* buf, long long bytes, int reps, int sm_count, cudaStream_t s);

// grid build kernels
cudaError_t scan_flags_u8(const uint8_t* flags, long long n, unsigned long long* excl, void* tmp,
                          size_t tmp_bytes, cudaStream_t s);
size_t scan_tmp_bytes(long long n);
cudaError_t build_children(const uint8_t* flags, const unsigned long long* excl, long long n,
                           long long n0, uint32_t* child, cudaStream_t s);
cudaError_t build_levels(const long long* level_off, int n_levels, uint8_t* level, cudaStream_t s);
cudaError_t build_coords(const uint32_t* child, long long lvl_begin, long long lvl_end, const int* root,
                         uint64_t* coord, cudaStream_t s);
cudaError_t build_density(const double* dens_in, const uint32_t* child, long long lvl_begin,
                          long long lvl_end, double* rho64, cudaStream_t s);
cudaError_t build_nodes(const double* rho64, const uint32_t* child, long long n, double inv_scale,
                        float* density, uint32_t* node, cudaStream_t s);
cudaError_t reduce_max_leaf(const double* rho64, const uint32_t* child, long long n, double* out,
                            cudaStream_t s);
cudaError_t validate_leaf_density(const double* rho64, const uint32_t* child, long long n, int* bad,
                                  cudaStream_t s);

// record an error message for rt_last_error and return code
int set_error(int code, const char* msg);
// the hierarchical model built bottom-up from a full-resolution cube
// (Sect. 4.1); see rt_merge_uniform in rt.h
int merge_uniform(const int* root, double h0, int L, const double* rho, double kappa, double tau_max, double cmax,
                  long long cap, uint8_t* flags_host, double* dens_host, long long* n_ref_host, int* n_levels,
                  long long* n_cells, cudaStream_t s);
// device of a context
int ctx_device(const rt_ctx* c);

// dust kernels
cudaError_t dust_table(const double* lam_um, const double* kabs, const double* dnu, int nl, double Tmin,
                       double Tmax, int n_table, double* table, cudaStream_t s);
cudaError_t dust_temperature(const double* absorbed, int n_bins, long long n_cells, const uint32_t* child,
                             const double* rho64, const uint8_t* level, double h0, const double* lam_um,
                             const double* kabs, const double* dnu, int nl, double Tmin, double Tmax,
                             const double* table, int n_table, double* T, cudaStream_t s);
cudaError_t dust_emission(const double* T, long long n_cells, const uint32_t* child, const double* rho64,
                          const uint8_t* level, double h0, const double* lam_um, const double* kabs,
                          const double* dnu, int nl, double* emission, cudaStream_t s);
// per-bin totals of dust_emission's emission into tot [nl] (device)
cudaError_t dust_emission_totals(const double* T, long long n_cells, const uint32_t* child, const double* rho64,
                                 const uint8_t* level, double h0, const double* lam, const double* kabs,
                                 const double* dnu, int nl, double* tot, cudaStream_t s);
// max over leaves with hits >= min_hits of |T - T_prev| / T_prev into *out
cudaError_t max_rel_change(const double* T, const double* T_prev, const unsigned int* hits, const uint32_t* child,
                           long long n, double min_hits, double* out, cudaStream_t s);
// subiterations: T of the cells below level L (0 elsewhere); A = A_star +
// sum of the level arrays; imbalance |A - rho V E(T)|, mass and emission
// rho V E(T) over the leaves at level <= L and below L (out[6]: imbalance,
// mass at <= L, imbalance, mass below L, emission at <= L, below L)
cudaError_t mask_levels(const double* T, const uint8_t* level, long long n, int L, double* out, cudaStream_t s);
cudaError_t sum_levels(const double* I, int n_levels, long long n, const double* A_star, double* A, cudaStream_t s);
// ALI per frequency (Eq. 3): weights w_b = 1 - Lambda_b [nl][n], the
// right-hand side A - sum_b Lambda_b emitted_b and the cells that use it;
// kabs [nl] orders the bins for the cells' unsampled bins
cudaError_t ali_weights(const double* A, const double* self, const double* emitted, const unsigned int* count,
                        const double* kabs, unsigned int min_count, double lam_max, int nl, long long n, double* rhs,
                        double* w, uint8_t* use, cudaStream_t s);
// the ALI cells' temperatures from sum_b w_b E_b(T) = rhs (starts from T)
cudaError_t dust_temperature_weighted(const double* rhs, const double* w, const uint8_t* use, long long n,
                                      const uint32_t* child, const double* rho64, const uint8_t* level, double h0,
                                      const double* lam, const double* kabs, const double* dnu, int nl, double Tmin,
                                      double Tmax, double* T, cudaStream_t s);
cudaError_t level_imbalance(const double* A, const double* T, const uint32_t* child, const double* rho64,
                            const uint8_t* level, double h0, const double* table, int n_table, long long n, int L,
                            double* out, cudaStream_t s);
// per-row sums of rows x n (f64) into out[rows] (device)
cudaError_t row_sums_f64(const double* data, int n_rows, long long n, double* out, cudaStream_t s);
// inclusive prefix sums of n_rows rows of length n (f64), in place
cudaError_t scan_rows_f64(double* data, int n_rows, long long n, void* tmp, size_t tmp_bytes,
                          cudaStream_t s);
size_t scan_rows_tmp_bytes(int n_rows, long long n);
// exclusive prefix sums of n_rows rows of length n (int64), in place
cudaError_t scan_rows_i64_excl(long long* data, int n_rows, long long n, void* tmp, size_t tmp_bytes,
                               cudaStream_t s);
// Dust packages per cell (Sect. 4.2): row b of first [nl][n + 1] gets, for
// each cell, floor(emission[b][c] / w[b] + u_bc) (u_bc: word 0 of Philox
// counter (c, 0x80000000, 0, (src << 16) | b) under key (k0, k1)), and 0 in
// the last column; an exclusive scan of the rows then gives each cell's
// first package and the bin's total.  w: device [nl]; w[b] <= 0: no packages
cudaError_t dust_counts(const double* emission, long long n, int nl, const double* w, uint32_t k0, uint32_t k1,
                        uint32_t src, long long* first, cudaStream_t s);

}  // namespace rtk
