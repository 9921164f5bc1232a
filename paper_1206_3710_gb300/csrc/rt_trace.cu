// rt_trace.cu -- persistent Monte Carlo package tracer for hierarchical grids.
//
// One CUDA thread follows one photon package at a time (Sect. 2.3): emit,
// locate the leaf, step cell by cell, lose weight by continuous absorption
// (Sect. 2.3, Lucy 1999) or by analog absorption events, scatter with the
// Henyey-Greenstein phase function, peel off scattered light towards each
// observer after every scattering (Sect. 2.4), play Russian roulette
// (Sect. 2.3), and leave at the outer boundary of the root grid.
//
// GPU design (not the paper's grid-by-grid CPU scheme, App. A):
//  * persistent grid; each warp refills its finished lanes in one batch from
//    a global package counter (one atomicAdd per refill), so warps stay full
//    while packages of very different lengths finish;
//  * the trace and the peel-off march share one cell-stepping loop: a lane
//    is either tracing or marching towards observer o, so scattering events
//    do not serialise the warp on a nested loop;
//  * geometry runs in leaf-local coordinates (cell = 1 unit, Sect. 2.3) plus
//    integer lattice coordinates at the leaf's level, so FP32 keeps its
//    precision at deep levels; a face crossing moves to the sibling in the
//    same octet with one load, otherwise re-descends from the root;
//  * one 32-bit node word per visit (density or child index), absorbed
//    energy by FP64 atomics (RED) into [bin][cell].
#include <math_constants.h>

#include "philox.cuh"
#include "rt_internal.cuh"

namespace rtk {

template <typename R>
struct Num;

template <>
struct Num<float> {
  // u32 -> (0,1): ((x >> 9) + 0.5) 2^-23, exact in f32
  static __device__ __forceinline__ float uni(uint32_t x) {
    return (float)(x >> 9) * 1.1920928955078125e-07f + 5.9604644775390625e-08f;
  }
  static __device__ __forceinline__ float log_(float x) { return logf(x); }
  static __device__ __forceinline__ float expm1_(float x) { return expm1f(x); }
  static __device__ __forceinline__ float exp_(float x) { return expf(x); }
  static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
  static __device__ __forceinline__ float floor_(float x) { return floorf(x); }
  static __device__ __forceinline__ float ldexp_(float x, int e) { return ldexpf(x, e); }
  static __device__ __forceinline__ void sincos2pi(float u, float* s, float* c) { sincospif(2.0f * u, s, c); }
  static __device__ __forceinline__ float inf() { return CUDART_INF_F; }
  static __device__ __forceinline__ float leaf_rho(const JobDev& J, uint32_t w, uint32_t) {
    return __uint_as_float(w);
  }
  static __device__ __forceinline__ float kext(const BinDev& b) { return b.kext_f; }
  static __device__ __forceinline__ float alb(const BinDev& b) { return b.albedo; }
  static __device__ __forceinline__ float gg(const BinDev& b) { return b.g; }
};

template <>
struct Num<double> {
  static __device__ __forceinline__ double uni(uint32_t x) { return ((double)x + 0.5) * 2.3283064365386963e-10; }
  static __device__ __forceinline__ double log_(double x) { return log(x); }
  static __device__ __forceinline__ double expm1_(double x) { return expm1(x); }
  static __device__ __forceinline__ double exp_(double x) { return exp(x); }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double floor_(double x) { return floor(x); }
  static __device__ __forceinline__ double ldexp_(double x, int e) { return ldexp(x, e); }
  static __device__ __forceinline__ void sincos2pi(double u, double* s, double* c) { sincospi(2.0 * u, s, c); }
  static __device__ __forceinline__ double inf() { return CUDART_INF; }
  static __device__ __forceinline__ double leaf_rho(const JobDev& J, uint32_t, uint32_t idx) {
    return __ldg(J.rho64 + idx);
  }
  static __device__ __forceinline__ double kext(const BinDev& b) { return b.kext_d; }
  static __device__ __forceinline__ double alb(const BinDev& b) { return b.albedo_d; }
  static __device__ __forceinline__ double gg(const BinDev& b) { return b.g_d; }
};

// position of a package: leaf at level `lev` with lattice coordinates c and
// in-leaf offsets f in [0,1]; idx is the leaf's array index
template <typename R>
struct Geo {
  uint32_t cx, cy, cz;
  int lev;
  uint32_t idx;
  R fx, fy, fz;
  R rho;
};

__device__ __forceinline__ uint32_t load_node(const uint32_t* node, uint32_t i) { return __ldg(node + i); }

// point on a face belongs to the child the direction points into
template <typename R>
__device__ __forceinline__ uint32_t upper_half(R f, R d) {
  return (f > R(0.5)) | ((f == R(0.5)) & (d >= R(0)));
}

// descend from a refined node word w at the current (c, lev) using offsets
template <typename R>
__device__ __forceinline__ void descend(const JobDev& J, Geo<R>& g, uint32_t w, R dx, R dy, R dz) {
  while (w & RT_INTERIOR) {
    const uint32_t bx = upper_half(g.fx, dx), by = upper_half(g.fy, dy), bz = upper_half(g.fz, dz);
    g.fx = R(2) * g.fx - R(bx);
    g.fy = R(2) * g.fy - R(by);
    g.fz = R(2) * g.fz - R(bz);
    g.cx = 2u * g.cx + bx;
    g.cy = 2u * g.cy + by;
    g.cz = 2u * g.cz + bz;
    g.lev += 1;
    g.idx = (w & RT_CHILD_MASK) + (bx | (by << 1) | (bz << 2));
    w = load_node(J.node, g.idx);
  }
  g.rho = Num<R>::leaf_rho(J, w, g.idx);
}

// find the leaf holding (c, f) at level lev by descending from the root;
// returns false if the point is outside the root grid
template <typename R>
__device__ __forceinline__ bool locate_root(const JobDev& J, Geo<R>& g, R dx, R dy, R dz) {
  const uint32_t rx = g.cx >> g.lev, ry = g.cy >> g.lev, rz = g.cz >> g.lev;
  if (rx >= J.root[0] || ry >= J.root[1] || rz >= J.root[2]) return false;
  uint32_t idx = rx + J.root[0] * (ry + J.root[1] * rz);
  uint32_t w = load_node(J.node, idx);
  int l = 0;
  while (l < g.lev && (w & RT_INTERIOR)) {
    ++l;
    const int sh = g.lev - l;
    const uint32_t o = ((g.cx >> sh) & 1u) | (((g.cy >> sh) & 1u) << 1) | (((g.cz >> sh) & 1u) << 2);
    idx = (w & RT_CHILD_MASK) + o;
    w = load_node(J.node, idx);
  }
  g.idx = idx;
  if (l < g.lev) {  // the leaf is coarser than the lattice level: re-express offsets
    const int k = g.lev - l;
    const uint32_t m = (1u << k) - 1u;
    const R s = Num<R>::ldexp_(R(1), -k);
    g.fx = (R(g.cx & m) + g.fx) * s;
    g.fy = (R(g.cy & m) + g.fy) * s;
    g.fz = (R(g.cz & m) + g.fz) * s;
    g.cx >>= k;
    g.cy >>= k;
    g.cz >>= k;
    g.lev = l;
    g.rho = Num<R>::leaf_rho(J, w, idx);
  } else {
    descend(J, g, w, dx, dy, dz);
  }
  return true;
}

// place a point given in root-cell units (root level), faces belong to the
// cell the direction points into
template <typename R>
__device__ __forceinline__ bool place_root_units(const JobDev& J, Geo<R>& g, R px, R py, R pz, R dx, R dy,
                                                 R dz) {
  if (!(px >= R(0) && py >= R(0) && pz >= R(0) && px <= (R)J.root[0] && py <= (R)J.root[1] &&
        pz <= (R)J.root[2]))
    return false;
  R fl = Num<R>::floor_(px);
  g.cx = (uint32_t)fl;
  g.fx = px - fl;
  if (g.fx == R(0) && dx < R(0)) { g.cx -= 1u; g.fx = R(1); }
  fl = Num<R>::floor_(py);
  g.cy = (uint32_t)fl;
  g.fy = py - fl;
  if (g.fy == R(0) && dy < R(0)) { g.cy -= 1u; g.fy = R(1); }
  fl = Num<R>::floor_(pz);
  g.cz = (uint32_t)fl;
  g.fz = pz - fl;
  if (g.fz == R(0) && dz < R(0)) { g.cz -= 1u; g.fz = R(1); }
  g.lev = 0;
  return locate_root(J, g, dx, dy, dz);
}

// exit distance (leaf-local units) and axis; ties -> lowest axis.  Axes with
// d == 0 give NaN or inf and are never selected.
template <typename R>
__device__ __forceinline__ R exit_dist(const Geo<R>& g, R dx, R dy, R dz, R ix, R iy, R iz, int& axis) {
  const R tx = (dx > R(0) ? R(1) - g.fx : g.fx) * ix;
  const R ty = (dy > R(0) ? R(1) - g.fy : g.fy) * iy;
  const R tz = (dz > R(0) ? R(1) - g.fz : g.fz) * iz;
  R t = Num<R>::inf();
  int a = -1;
  if (tx < t) { t = tx; a = 0; }
  if (ty < t) { t = ty; a = 1; }
  if (tz < t) { t = tz; a = 2; }
  axis = a;
  return t;
}

template <typename R>
__device__ __forceinline__ R clamp01(R v) {
  return v < R(0) ? R(0) : (v > R(1) ? R(1) : v);
}

// Cross the exit face on axis a and find the next leaf.  Returns false when
// the package leaves the root grid.
template <typename R>
__device__ __forceinline__ bool cross_face(const JobDev& J, Geo<R>& g, int a, R t, R dx, R dy, R dz) {
  uint32_t cold, cnew;
  bool plus;
  if (a == 0) {
    plus = dx > R(0);
    g.fy = clamp01(g.fy + t * dy);
    g.fz = clamp01(g.fz + t * dz);
    cold = g.cx;
    g.cx = plus ? g.cx + 1u : g.cx - 1u;
    g.fx = plus ? R(0) : R(1);
    cnew = g.cx;
  } else if (a == 1) {
    plus = dy > R(0);
    g.fx = clamp01(g.fx + t * dx);
    g.fz = clamp01(g.fz + t * dz);
    cold = g.cy;
    g.cy = plus ? g.cy + 1u : g.cy - 1u;
    g.fy = plus ? R(0) : R(1);
    cnew = g.cy;
  } else {
    plus = dz > R(0);
    g.fx = clamp01(g.fx + t * dx);
    g.fy = clamp01(g.fy + t * dy);
    cold = g.cz;
    g.cz = plus ? g.cz + 1u : g.cz - 1u;
    g.fz = plus ? R(0) : R(1);
    cnew = g.cz;
  }
  uint32_t step;
  if (g.lev == 0) {
    if (cnew >= J.root[a]) return false;
    step = (a == 0) ? 1u : (a == 1 ? J.root[0] : J.root[0] * J.root[1]);
  } else if ((cold >> 1) == (cnew >> 1)) {
    step = 1u << a;  // sibling in the same octet
  } else {
    return locate_root(J, g, dx, dy, dz);
  }
  g.idx = plus ? g.idx + step : g.idx - step;
  const uint32_t w = load_node(J.node, g.idx);
  if (w & RT_INTERIOR) descend(J, g, w, dx, dy, dz);
  else g.rho = Num<R>::leaf_rho(J, w, g.idx);
  return true;
}

template <typename R>
__device__ __forceinline__ R hg_mu(R g, R u) {
  R mu;
  if (g == R(0)) {
    mu = R(2) * u - R(1);
  } else {
    const R s = (R(1) - g * g) / (R(1) - g + R(2) * g * u);
    mu = (R(1) + g * g - s * s) / (R(2) * g);
  }
  return mu > R(1) ? R(1) : (mu < R(-1) ? R(-1) : mu);
}

template <typename R>
__device__ __forceinline__ R hg_phase(R g, R mu) {
  const R den = R(1) + g * g - R(2) * g * mu;
  return (R(1) - g * g) / (R(4) * R(CUDART_PI) * den * Num<R>::sqrt_(den));
}

// rotate direction d by polar cosine mu and azimuth 2 pi u (the usual
// Monte Carlo transport rotation), renormalised
template <typename R>
__device__ __forceinline__ void scatter_dir(R& dx, R& dy, R& dz, R mu, R u) {
  R sp, cp;
  Num<R>::sincos2pi(u, &sp, &cp);
  const R st = Num<R>::sqrt_(fmax(R(0), R(1) - mu * mu));
  R nx, ny, nz;
  if (fabs(dz) > R(0.99999)) {
    nx = st * cp;
    ny = st * sp;
    nz = dz > R(0) ? mu : -mu;
  } else {
    const R den = Num<R>::sqrt_(R(1) - dz * dz);
    nx = st * (dx * dz * cp - dy * sp) / den + dx * mu;
    ny = st * (dy * dz * cp + dx * sp) / den + dy * mu;
    nz = -st * cp * den + dz * mu;
  }
  const R nrm = Num<R>::sqrt_(nx * nx + ny * ny + nz * nz);
  dx = nx / nrm;
  dy = ny / nrm;
  dz = nz / nrm;
}

template <typename R>
__device__ __forceinline__ void iso_dir(R u1, R u2, R& dx, R& dy, R& dz) {
  const R mu = R(2) * u1 - R(1);
  const R st = Num<R>::sqrt_(fmax(R(0), R(1) - mu * mu));
  R s, c;
  Num<R>::sincos2pi(u2, &s, &c);
  dx = st * c;
  dy = st * s;
  dz = mu;
}

template <typename R>
__device__ __forceinline__ R inv_abs(R d) {
  return R(1) / fabs(d);
}

struct LaneLedger {
  double emitted, absorbed, escaped, rr_gain, rr_loss, killed, peeled;
  unsigned long long n_packets, n_cross, n_scatter, n_peel_cross, n_killed, n_peel_out;
  __device__ void zero() {
    emitted = absorbed = escaped = rr_gain = rr_loss = killed = peeled = 0.0;
    n_packets = n_cross = n_scatter = n_peel_cross = n_killed = n_peel_out = 0ull;
  }
  __device__ void flush(LedgerDev* L) {
    if (emitted != 0.0) atomicAdd(&L->emitted, emitted);
    if (absorbed != 0.0) atomicAdd(&L->absorbed, absorbed);
    if (escaped != 0.0) atomicAdd(&L->escaped, escaped);
    if (rr_gain != 0.0) atomicAdd(&L->rr_gain, rr_gain);
    if (rr_loss != 0.0) atomicAdd(&L->rr_loss, rr_loss);
    if (killed != 0.0) atomicAdd(&L->killed, killed);
    if (peeled != 0.0) atomicAdd(&L->peeled, peeled);
    if (n_packets) atomicAdd(&L->n_packets, n_packets);
    if (n_cross) atomicAdd(&L->n_cross, n_cross);
    if (n_scatter) atomicAdd(&L->n_scatter, n_scatter);
    if (n_peel_cross) atomicAdd(&L->n_peel_cross, n_peel_cross);
    if (n_killed) atomicAdd(&L->n_killed, n_killed);
    if (n_peel_out) atomicAdd(&L->n_peel_out, n_peel_out);
    zero();
  }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}
__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

enum { ST_DEAD = 0, ST_TRACE = 1, ST_PEEL = 2, ST_DONE = 3 };

template <typename R, bool PEEL>
__global__ void __launch_bounds__(256) trace_kernel(const JobDev* __restrict__ jobs,
                                                    const ItemDev* __restrict__ items, int n_items,
                                                    unsigned long long* __restrict__ counter,
                                                    long long total, int refill_thr) {
  const unsigned FULL = 0xFFFFFFFFu;
  const int lane = threadIdx.x & 31;

  int st = ST_DEAD;
  int job = -1, acc_job = -1;
  LaneLedger acc;
  acc.zero();

  Geo<R> g;
  g.cx = g.cy = g.cz = 0u;
  g.lev = 0;
  g.idx = 0u;
  g.fx = g.fy = g.fz = R(0);
  g.rho = R(0);
  R dx = R(0), dy = R(0), dz = R(1), ix = R(0), iy = R(0), iz = R(0);
  R W = R(0), W0 = R(0), tau = R(0), pkt_abs = R(0);
  R kext = R(0), alb = R(0), gpar = R(0);
  double* absb = nullptr;
  const JobDev* Jp = jobs;
  PhiloxStream rng;
  rng.init(0ull, 0u, 0u, 0u, 0ull);
  long long steps = 0, log_index = -1;
  uint32_t nscat = 0u, ncross = 0u;
  int bin = 0;
  // peel-off state (observer march)
  int obs_i = 0;
  R taup = R(0), pw = R(0);
  long long pix = -1;
  Geo<R> sg = g;
  R sdx = R(0), sdy = R(0), sdz = R(0);

  // after a scattering (and its peel-off): new direction from the phase
  // function, Russian roulette when the weight is low, next free path.
  // Returns a fate (1 = roulette kill) or -1.
  auto finish_scatter = [&](const JobDev& J) -> int {
    const R mu = hg_mu(gpar, Num<R>::uni(rng.u32()));
    scatter_dir(dx, dy, dz, mu, Num<R>::uni(rng.u32()));
    ix = inv_abs(dx);
    iy = inv_abs(dy);
    iz = inv_abs(dz);
    if (J.rr_wmin > 0.0 && W < (R)J.rr_wmin * W0) {
      const R ur = Num<R>::uni(rng.u32());
      if (ur < (R)J.rr_p) {
        acc.rr_loss += (double)W;
        W = R(0);
        return 1;
      }
      const R Wn = W / (R(1) - (R)J.rr_p);
      acc.rr_gain += (double)(Wn - W);
      W = Wn;
    }
    tau = -Num<R>::log_(Num<R>::uni(rng.u32()));
    return -1;
  };

  for (;;) {
    // ---------------------------------------------------------------- refill
    const unsigned dead = __ballot_sync(FULL, st == ST_DEAD);
    const unsigned busy = __ballot_sync(FULL, st == ST_TRACE || st == ST_PEEL);
    if (dead != 0u && (__popc(dead) >= refill_thr || busy == 0u)) {
      const int leader = __ffs(dead) - 1;
      unsigned long long base = 0ull;
      if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(dead));
      base = __shfl_sync(FULL, base, leader);
      if (st == ST_DEAD) {
        const long long gi = (long long)base + __popc(dead & ((1u << lane) - 1u));
        if (gi >= total) {
          st = ST_DONE;
        } else {
          // ------------------------------------------------ emission (Sect. 2.3)
          int lo = 0, hi = n_items - 1;
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (items[mid].pkt_begin <= gi) lo = mid;
            else hi = mid - 1;
          }
          const ItemDev& I = items[lo];
          job = I.job;
          if (job != acc_job) {
            if (acc_job >= 0) acc.flush(jobs[acc_job].ledger);
            acc_job = job;
          }
          Jp = jobs + job;
          const JobDev& J = *Jp;
          const long long p = gi - I.pkt_begin;
          int blo = 0, bhi = J.n_lambda - 1;
          while (blo < bhi) {
            const int mid = (blo + bhi + 1) >> 1;
            if (I.bin_prefix[mid] <= p) blo = mid;
            else bhi = mid - 1;
          }
          bin = blo;
          const long long k = p - I.bin_prefix[bin];
          log_index = J.packet_log ? I.log_offset + p : -1;
          rng.init(J.seed, J.job_id, J.iter, (I.src_index << 16) | (uint32_t)bin, (unsigned long long)k);
          const BinDev& B = J.bins[bin];
          kext = Num<R>::kext(B);
          alb = Num<R>::alb(B);
          gpar = Num<R>::gg(B);
          absb = J.absorbed ? J.absorbed + (long long)(J.abs_bins > 1 ? bin : 0) * J.n_cells : nullptr;
          W0 = (R)I.W0[bin];
          W = W0;
          pkt_abs = R(0);
          steps = 0;
          nscat = ncross = 0u;
          acc.emitted += (double)W0;
          acc.n_packets += 1ull;
          bool inside;
          if (I.kind == RT_SRC_POINT || I.kind == RT_SRC_BEAM) {
            if (I.kind == RT_SRC_POINT) {
              const R u1 = Num<R>::uni(rng.u32()), u2 = Num<R>::uni(rng.u32());
              iso_dir(u1, u2, dx, dy, dz);
            } else {
              dx = (R)I.dir[0];
              dy = (R)I.dir[1];
              dz = (R)I.dir[2];
            }
            inside = place_root_units(J, g, (R)I.pos[0], (R)I.pos[1], (R)I.pos[2], dx, dy, dz);
          } else if (I.kind == RT_SRC_EXTERNAL) {
            // face by area, uniform point on it, cosine-weighted inward direction
            const double ax = (double)J.root[1] * J.root[2], ay = (double)J.root[0] * J.root[2],
                         az = (double)J.root[0] * J.root[1];
            const R u0 = Num<R>::uni(rng.u32());
            const R tot = R(2) * (R)(ax + ay + az);
            const R v = u0 * tot;
            int face = 5;
            R cum = R(0);
            const R ar[3] = {(R)ax, (R)ay, (R)az};
#pragma unroll
            for (int f = 0; f < 6; ++f) {
              cum += ar[f >> 1];
              if (face == 5 && v < cum) face = f;
            }
            const int a = face >> 1;
            const R u1 = Num<R>::uni(rng.u32()), u2 = Num<R>::uni(rng.u32());
            const R u3 = Num<R>::uni(rng.u32()), u4 = Num<R>::uni(rng.u32());
            const R mu = Num<R>::sqrt_(u3), st_ = Num<R>::sqrt_(fmax(R(0), R(1) - mu * mu));
            R sp, cp;
            Num<R>::sincos2pi(u4, &sp, &cp);
            const R dn = (face & 1) ? -mu : mu;
            R px, py, pz;
            if (a == 0) {
              px = (face & 1) ? (R)J.root[0] : R(0);
              py = u1 * (R)J.root[1];
              pz = u2 * (R)J.root[2];
              dx = dn; dy = st_ * cp; dz = st_ * sp;
            } else if (a == 1) {
              py = (face & 1) ? (R)J.root[1] : R(0);
              px = u1 * (R)J.root[0];
              pz = u2 * (R)J.root[2];
              dy = dn; dx = st_ * cp; dz = st_ * sp;
            } else {
              pz = (face & 1) ? (R)J.root[2] : R(0);
              px = u1 * (R)J.root[0];
              py = u2 * (R)J.root[1];
              dz = dn; dx = st_ * cp; dy = st_ * sp;
            }
            inside = place_root_units(J, g, px, py, pz, dx, dy, dz);
          } else {
            // dust emission: cell from this bin's cumulative emission
            const double* cdf = I.cdf + (long long)bin * J.n_cells;
            const double totE = cdf[J.n_cells - 1];
            const double target = (double)Num<R>::uni(rng.u32()) * totE;
            long long clo = 0, chi = J.n_cells - 1;
            while (clo < chi) {
              const long long mid = clo + ((chi - clo) >> 1);
              if (cdf[mid] > target) chi = mid;
              else clo = mid + 1;
            }
            const uint64_t cw = J.coord[clo];
            g.cx = (uint32_t)(cw & RT_COORD_MASK);
            g.cy = (uint32_t)((cw >> RT_COORD_BITS) & RT_COORD_MASK);
            g.cz = (uint32_t)((cw >> (2 * RT_COORD_BITS)) & RT_COORD_MASK);
            g.lev = J.level[clo];
            g.idx = (uint32_t)clo;
            g.fx = Num<R>::uni(rng.u32());
            g.fy = Num<R>::uni(rng.u32());
            g.fz = Num<R>::uni(rng.u32());
            g.rho = Num<R>::leaf_rho(J, load_node(J.node, g.idx), g.idx);
            const R u4 = Num<R>::uni(rng.u32()), u5 = Num<R>::uni(rng.u32());
            iso_dir(u4, u5, dx, dy, dz);
            inside = true;
          }
          ix = inv_abs(dx);
          iy = inv_abs(dy);
          iz = inv_abs(dz);
          tau = -Num<R>::log_(Num<R>::uni(rng.u32()));
          if (inside) {
            st = ST_TRACE;
          } else {
            acc.escaped += (double)W;
            if (log_index >= 0) {
              double* r = J.packet_log + log_index * 10;
              r[0] = (double)W; r[1] = 0.0; r[2] = 0.0; r[3] = 0.0;
              r[4] = r[5] = r[6] = 0.0;
              r[7] = (double)dx; r[8] = (double)dy; r[9] = (double)dz;
            }
            st = ST_DEAD;
          }
        }
      }
    }
    {
      const unsigned still = __ballot_sync(FULL, st != ST_DONE);
      if (still == 0u) break;
    }
    if (st != ST_TRACE && st != ST_PEEL) continue;

    // ------------------------------------------------------------------ step
    const JobDev& J = *Jp;
    int fate = -1;  // >= 0: the package ends with this fate
    if (st == ST_TRACE && steps >= J.step_limit) {
      acc.killed += (double)W;
      acc.n_killed += 1ull;
      atomicOr(&J.ledger->status, 1);
      fate = 2;
    } else {
      int a;
      const R t = exit_dist(g, dx, dy, dz, ix, iy, iz, a);
      if (a < 0) {  // degenerate direction: cannot happen for |d| = 1
        if (st == ST_TRACE) {
          acc.killed += (double)W;
          acc.n_killed += 1ull;
          atomicOr(&J.ledger->status, 2);
          fate = 2;
        } else {
          pix = -1;  // abandon this observer
        }
      } else {
        const R kl = kext * g.rho * Num<R>::ldexp_(R(1), -g.lev);  // extinction per local unit
        bool inside_event = false;
        R tseg = t;
        if (st == ST_TRACE) {
          ++steps;
          if (J.estimator == RT_EST_CONTINUOUS) {
            const R ksca = alb * kl;
            const R tsc = ksca * t;
            if (ksca > R(0) && tsc >= tau) {
              inside_event = true;
              tseg = tau / ksca;
            } else {
              tau -= tsc;
            }
            const R q = -Num<R>::expm1_(-(kl - ksca) * tseg);
            const R dep = W * q;
            W -= dep;
            if (dep > R(0)) {
              pkt_abs += dep;
              if (absb) atomicAdd(absb + g.idx, (double)dep);
            }
          } else {
            const R te = kl * t;
            if (kl > R(0) && te >= tau) {
              inside_event = true;
              tseg = tau / kl;
            } else {
              tau -= te;
            }
          }
          if (tseg > R(0)) ++ncross;
        } else {
          taup += kl * t;
          if (t > R(0)) acc.n_peel_cross += 1ull;
        }

        if (inside_event) {
          // ------------------------------------------- interaction in this cell
          g.fx = clamp01(g.fx + tseg * dx);
          g.fy = clamp01(g.fy + tseg * dy);
          g.fz = clamp01(g.fz + tseg * dz);
          bool scatter = true;
          if (J.estimator == RT_EST_ANALOG) {
            const R ua = Num<R>::uni(rng.u32());
            if (ua >= alb) {
              scatter = false;
              if (absb) atomicAdd(absb + g.idx, (double)W);
              pkt_abs += W;
              W = R(0);
              fate = 3;
            }
          }
          if (scatter) {
            ++nscat;
            acc.n_scatter += 1ull;
            if (PEEL && J.n_obs > 0) {
              // save the scattering point and march towards each observer in
              // turn (observer selection below); the new direction is drawn
              // after the last observer
              sg = g;
              sdx = dx; sdy = dy; sdz = dz;
              obs_i = -1;
              pix = -1;
              st = ST_PEEL;
            } else {
              fate = finish_scatter(J);
            }
          }
        } else if (st == ST_PEEL && J.peel_tau_max > 0.0 && taup > (R)J.peel_tau_max) {
          pix = -1;  // cut: this observer gets nothing; select the next one below
        } else {
          const bool in = cross_face(J, g, a, t, dx, dy, dz);
          if (!in) {
            if (st == ST_TRACE) {
              acc.escaped += (double)W;
              fate = 0;
            } else {
              // peel-off contribution reaches the observer
              if (pix >= 0) {
                const double c = (double)pw * (double)Num<R>::exp_(-taup);
                atomicAdd(J.images + pix, c);
                acc.peeled += c;
              }
              pix = -1;
            }
          }
        }
      }
    }

    // -------------------------------------------- peel-off observer selection
    if (PEEL && st == ST_PEEL && pix < 0) {
      // choose the next observer whose pixel is inside the image
      bool started = false;
      while (!started) {
        ++obs_i;
        if (obs_i >= J.n_obs) break;
        const ObsDev& O = J.obs[obs_i];
        // scattering point in root-cell units
        const R s = Num<R>::ldexp_(R(1), -sg.lev);
        const R Px = ((R)sg.cx + sg.fx) * s - (R)O.c[0];
        const R Py = ((R)sg.cy + sg.fy) * s - (R)O.c[1];
        const R Pz = ((R)sg.cz + sg.fz) * s - (R)O.c[2];
        const R u = (Px * (R)O.ex[0] + Py * (R)O.ex[1] + Pz * (R)O.ex[2]) * (R)O.inv_pix[0] + R(0.5) * (R)O.nx;
        const R v = (Px * (R)O.ey[0] + Py * (R)O.ey[1] + Pz * (R)O.ey[2]) * (R)O.inv_pix[1] + R(0.5) * (R)O.ny;
        const R fu = Num<R>::floor_(u), fv = Num<R>::floor_(v);
        if (!(fu >= R(0) && fv >= R(0) && fu < (R)O.nx && fv < (R)O.ny)) {
          acc.n_peel_out += 1ull;
          continue;
        }
        const R kx = (R)O.k[0], ky = (R)O.k[1], kz = (R)O.k[2];
        pw = W * hg_phase(gpar, sdx * kx + sdy * ky + sdz * kz);
        pix = (((long long)obs_i * J.img_bins + (J.img_bins > 1 ? bin : 0)) * O.ny + (long long)fv) * O.nx +
              (long long)fu;
        g = sg;
        dx = kx; dy = ky; dz = kz;
        ix = inv_abs(dx); iy = inv_abs(dy); iz = inv_abs(dz);
        taup = R(0);
        started = true;
      }
      if (!started) {
        // all observers done: restore the package and finish the scattering
        g = sg;
        dx = sdx; dy = sdy; dz = sdz;
        st = ST_TRACE;
        fate = finish_scatter(J);
      }
    }

    if (fate >= 0) {
      acc.absorbed += (double)pkt_abs;
      acc.n_cross += ncross;
      if (log_index >= 0) {
        double* r = J.packet_log + log_index * 10;
        const R s = Num<R>::ldexp_(R(1), -g.lev);
        r[0] = fate == 0 ? (double)W : 0.0;
        r[1] = (double)nscat;
        r[2] = (double)ncross;
        r[3] = (double)fate;
        r[4] = ((double)g.cx + (double)g.fx) * (double)s * J.h0;
        r[5] = ((double)g.cy + (double)g.fy) * (double)s * J.h0;
        r[6] = ((double)g.cz + (double)g.fz) * (double)s * J.h0;
        r[7] = (double)dx; r[8] = (double)dy; r[9] = (double)dz;
      }
      st = ST_DEAD;
    }
  }

  // ------------------------------------------------------------ final ledger
  const int j0 = __shfl_sync(FULL, acc_job, 0);
  if (__all_sync(FULL, acc_job == j0)) {
    if (j0 >= 0) {
      double v[7] = {acc.emitted, acc.absorbed, acc.escaped, acc.rr_gain, acc.rr_loss, acc.killed, acc.peeled};
      unsigned long long u[6] = {acc.n_packets, acc.n_cross, acc.n_scatter, acc.n_peel_cross, acc.n_killed,
                                 acc.n_peel_out};
#pragma unroll
      for (int i = 0; i < 7; ++i) v[i] = warp_sum(v[i]);
#pragma unroll
      for (int i = 0; i < 6; ++i) u[i] = warp_sum(u[i]);
      if (lane == 0) {
        acc.emitted = v[0]; acc.absorbed = v[1]; acc.escaped = v[2]; acc.rr_gain = v[3];
        acc.rr_loss = v[4]; acc.killed = v[5]; acc.peeled = v[6];
        acc.n_packets = u[0]; acc.n_cross = u[1]; acc.n_scatter = u[2]; acc.n_peel_cross = u[3];
        acc.n_killed = u[4]; acc.n_peel_out = u[5];
        acc.flush(jobs[j0].ledger);
      }
    }
  } else if (acc_job >= 0) {
    acc.flush(jobs[acc_job].ledger);
  }
}

// ------------------------------------------------------------------------
// deterministic walk (diagnostic): the tracer's own stepping, no physics
// ------------------------------------------------------------------------
template <typename R>
__global__ void walk_kernel(const JobDev* __restrict__ job, long long n_rays, const double* __restrict__ origins,
                            const double* __restrict__ dirs, long long max_seg, long long* __restrict__ cells,
                            double* __restrict__ lengths, long long* __restrict__ counts) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rays) return;
  const JobDev& J = *job;
  const R dx = (R)dirs[3 * r], dy = (R)dirs[3 * r + 1], dz = (R)dirs[3 * r + 2];
  Geo<R> g;
  if (!place_root_units(J, g, (R)(origins[3 * r] / J.h0), (R)(origins[3 * r + 1] / J.h0),
                        (R)(origins[3 * r + 2] / J.h0), dx, dy, dz)) {
    counts[r] = -1;
    return;
  }
  const R ix = inv_abs(dx), iy = inv_abs(dy), iz = inv_abs(dz);
  long long k = 0;
  for (long long guard = 0; guard < 64ll * (1ll << 22); ++guard) {
    int a;
    const R t = exit_dist(g, dx, dy, dz, ix, iy, iz, a);
    if (a < 0) break;
    if (t > R(0)) {
      if (k < max_seg) {
        cells[r * max_seg + k] = g.idx;
        lengths[r * max_seg + k] = (double)t * ldexp(1.0, -g.lev) * J.h0;
      }
      ++k;
    }
    if (!cross_face(J, g, a, t, dx, dy, dz)) break;
  }
  counts[r] = k;
}

__global__ void philox_kernel(long long n, const uint32_t* __restrict__ ctr, const uint32_t* __restrict__ key,
                              uint32_t* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
  const uint4 o = philox4x32_10(c, key[2 * i], key[2 * i + 1]);
  out[4 * i] = o.x;
  out[4 * i + 1] = o.y;
  out[4 * i + 2] = o.z;
  out[4 * i + 3] = o.w;
}

// ------------------------------------------------------------------------
// host launchers
// ------------------------------------------------------------------------
template <typename R, bool PEEL>
static cudaError_t launch_t(const JobDev* jobs, const ItemDev* items, int n_items, unsigned long long* counter,
                            long long total, const LaunchCfg& cfg, cudaStream_t s) {
  trace_kernel<R, PEEL><<<cfg.blocks, cfg.block, 0, s>>>(jobs, items, n_items, counter, total, cfg.refill);
  return cudaGetLastError();
}

cudaError_t launch_trace(int precision, bool peel, const JobDev* jobs_dev, const ItemDev* items_dev, int n_items,
                         unsigned long long* counter_dev, long long total, const LaunchCfg& cfg, cudaStream_t s) {
  if (precision == 64) {
    return peel ? launch_t<double, true>(jobs_dev, items_dev, n_items, counter_dev, total, cfg, s)
                : launch_t<double, false>(jobs_dev, items_dev, n_items, counter_dev, total, cfg, s);
  }
  return peel ? launch_t<float, true>(jobs_dev, items_dev, n_items, counter_dev, total, cfg, s)
              : launch_t<float, false>(jobs_dev, items_dev, n_items, counter_dev, total, cfg, s);
}

cudaError_t trace_occupancy(int precision, bool peel, int block, int* blocks_per_sm) {
  if (precision == 64) {
    return peel ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, trace_kernel<double, true>, block, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, trace_kernel<double, false>, block, 0);
  }
  return peel ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, trace_kernel<float, true>, block, 0)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, trace_kernel<float, false>, block, 0);
}

cudaError_t launch_walk(int precision, const JobDev* job_dev, long long n_rays, const double* origins,
                        const double* dirs, long long max_seg, long long* cells, double* lengths, long long* counts,
                        cudaStream_t s) {
  const int B = 128;
  const unsigned G = (unsigned)((n_rays + B - 1) / B);
  if (G == 0) return cudaSuccess;
  if (precision == 64) walk_kernel<double><<<G, B, 0, s>>>(job_dev, n_rays, origins, dirs, max_seg, cells, lengths, counts);
  else walk_kernel<float><<<G, B, 0, s>>>(job_dev, n_rays, origins, dirs, max_seg, cells, lengths, counts);
  return cudaGetLastError();
}

cudaError_t launch_philox(long long n, const uint32_t* ctr, const uint32_t* key, uint32_t* out, cudaStream_t s) {
  const int B = 256;
  const unsigned G = (unsigned)((n + B - 1) / B);
  if (G == 0) return cudaSuccess;
  philox_kernel<<<G, B, 0, s>>>(n, ctr, key, out);
  return cudaGetLastError();
}

}  // namespace rtk
