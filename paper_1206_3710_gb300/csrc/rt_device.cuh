// rt_device.cuh -- device-side building blocks of the tracers: number
// traits for the FP32 / FP64 paths, the octree cursor (one node word per
// step: descend, settle on a leaf, cross a face), the exit distance in
// leaf-local units, Henyey-Greenstein sampling, cached node loads and
// accumulator reductions, observer geometry.
#pragma once

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
  // q = 1 - exp(-x) and e = exp(-x) for x >= 0, both without cancellation:
  // Taylor series of q through x^6 below 1/8 (relative remainder < 1e-9)
  // with e = 1 - q; expf above, where q = 1 - e >= 0.117
  static __device__ __forceinline__ void absorb_pair(float x, float& q, float& e) {
    const float p = x * (1.0f - x * (0.5f - x * (1.0f / 6.0f - x * (1.0f / 24.0f - x * (1.0f / 120.0f - x * (1.0f / 720.0f))))));
    const bool small = x < 0.125f;
    // expf only where some lane needs it (most segments are thin): a branch,
    // so a warp without thick segments skips it (tracer 1 % faster on the
    // 256^3 cloud than computing it for every segment)
    float ex = 0.0f;
    if (!small) ex = expf(-x);
    q = small ? p : 1.0f - ex;
    e = small ? 1.0f - p : ex;
  }
  static __device__ __forceinline__ float exp_(float x) { return expf(x); }
  static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
  static __device__ __forceinline__ float floor_(float x) { return floorf(x); }
  static __device__ __forceinline__ float ldexp_(float x, int e) { return ldexpf(x, e); }
  static __device__ __forceinline__ void sincos2pi(float u, float* s, float* c) { sincospif(2.0f * u, s, c); }
  static __device__ __forceinline__ float inf() { return CUDART_INF_F; }
  // 2^-l for 0 <= l <= 126, exact
  static __device__ __forceinline__ float pow2m(int l) { return __int_as_float((127 - l) << 23); }
  static __device__ __forceinline__ float leaf_rho(uint32_t w, double) { return __uint_as_float(w); }
  static __device__ __forceinline__ double load_rho64(const double*, uint32_t) { return 0.0; }
  static __device__ __forceinline__ float kext(const BinDev& b) { return b.kext_f; }
  static __device__ __forceinline__ float w0(const ItemDev& I, int bin) { return I.W0f[bin]; }
  static __device__ __forceinline__ float pos(const ItemDev& I, int a) { return I.posf[a]; }
  static __device__ __forceinline__ float dir(const ItemDev& I, int a) { return I.dirf[a]; }
  static __device__ __forceinline__ float rr_wmin(const JobDev& J) { return J.rr_wmin_f; }
  static __device__ __forceinline__ float rr_p(const JobDev& J) { return J.rr_p_f; }
  static __device__ __forceinline__ float tau_max(const JobDev& J) { return J.peel_tau_max_f; }
  static __device__ __forceinline__ float alb(const BinDev& b) { return b.albedo; }
  static __device__ __forceinline__ float gg(const BinDev& b) { return b.g; }
};

template <>
struct Num<double> {
  static __device__ __forceinline__ double uni(uint32_t x) { return ((double)x + 0.5) * 2.3283064365386963e-10; }
  static __device__ __forceinline__ double log_(double x) { return log(x); }
  static __device__ __forceinline__ double expm1_(double x) { return expm1(x); }
  static __device__ __forceinline__ void absorb_pair(double x, double& q, double& e) {
    if (x < 0.125) {
      q = -expm1(-x);
      e = 1.0 - q;
    } else {
      e = exp(-x);
      q = 1.0 - e;
    }
  }
  static __device__ __forceinline__ double exp_(double x) { return exp(x); }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double floor_(double x) { return floor(x); }
  static __device__ __forceinline__ double ldexp_(double x, int e) { return ldexp(x, e); }
  static __device__ __forceinline__ void sincos2pi(double u, double* s, double* c) { sincospi(2.0 * u, s, c); }
  static __device__ __forceinline__ double inf() { return CUDART_INF; }
  static __device__ __forceinline__ double pow2m(int l) { return __longlong_as_double((long long)(1023 - l) << 52); }
  static __device__ __forceinline__ double leaf_rho(uint32_t, double r64) { return r64; }
  static __device__ __forceinline__ double load_rho64(const double* p, uint32_t i) { return __ldg(p + i); }
  static __device__ __forceinline__ double kext(const BinDev& b) { return b.kext_d; }
  static __device__ __forceinline__ double w0(const ItemDev& I, int bin) { return I.W0[bin]; }
  static __device__ __forceinline__ double pos(const ItemDev& I, int a) { return I.pos[a]; }
  static __device__ __forceinline__ double dir(const ItemDev& I, int a) { return I.dir[a]; }
  static __device__ __forceinline__ double rr_wmin(const JobDev& J) { return J.rr_wmin; }
  static __device__ __forceinline__ double rr_p(const JobDev& J) { return J.rr_p; }
  static __device__ __forceinline__ double tau_max(const JobDev& J) { return J.peel_tau_max; }
  static __device__ __forceinline__ double alb(const BinDev& b) { return b.albedo_d; }
  static __device__ __forceinline__ double gg(const BinDev& b) { return b.g_d; }
};


// Position of a package: a leaf at level `lev` with lattice coordinates c at
// that level and in-leaf offsets f in [0,1] (cell = 1 unit, Sect. 2.3).
template <typename R>
struct Geo {
  uint32_t cx, cy, cz;
  int lev;
  uint32_t idx;
  R fx, fy, fz;
  R rho;
};

// The next node to visit: `pending` is an array index whose node sits at
// level k on the path to the package's leaf.  Every loop iteration loads
// exactly one node word; a refined node advances one level, a leaf ends the
// search.  Lanes therefore never wait on another lane's multi-level descent.
struct Cursor {
  uint32_t pending;
  int k;
};

// The path above the current leaf (Sect. 2.3: a package that leaves a grid
// goes up to the enclosing grid and from there down into its neighbour):
// a[l * stride] is the index of the node of level l on the leaf's path from
// its root cell, kept for the levels l < cap.  n is cap while the stored
// path is the current leaf's (it was reached by a descent from its root
// cell or from a stored ancestor) and 0 for a package placed directly in a
// leaf; a move out of an octet then re-descends from the root cell, which
// stores the path again.  cap = 0 keeps no path.
struct AncPath {
  uint32_t* a;
  int stride;
  int cap;
  int n;
};

__device__ __forceinline__ AncPath no_path() {
  AncPath P;
  P.a = nullptr;
  P.stride = 0;
  P.cap = 0;
  P.n = 0;
  return P;
}

// grid geometry needed on the hot path, held in registers
struct GridRegs {
  const uint32_t* node;
  const double* rho64;
  uint32_t rx, ry, rz;
};

// a point on a face belongs to the child the direction points into
template <typename R>
__device__ __forceinline__ uint32_t upper_half(R f, R d) {
  return (f > R(0.5)) | ((f == R(0.5)) & (d >= R(0)));
}

// one level of descent below a refined node word w at cursor level k
template <typename R>
__device__ __forceinline__ void descend_step(Geo<R>& g, Cursor& cur, uint32_t w, R dx, R dy, R dz) {
  // above the lattice level: follow the lattice bits; at or below it: split
  // the leaf-local offsets
  const bool by_lattice = cur.k < g.lev;
  const int sh = by_lattice ? g.lev - cur.k - 1 : 0;
  const uint32_t ol = ((g.cx >> sh) & 1u) | (((g.cy >> sh) & 1u) << 1) | (((g.cz >> sh) & 1u) << 2);
  const uint32_t bx = upper_half(g.fx, dx), by = upper_half(g.fy, dy), bz = upper_half(g.fz, dz);
  if (!by_lattice) {
    g.fx = R(2) * g.fx - R(bx);
    g.fy = R(2) * g.fy - R(by);
    g.fz = R(2) * g.fz - R(bz);
    g.cx = 2u * g.cx + bx;
    g.cy = 2u * g.cy + by;
    g.cz = 2u * g.cz + bz;
    g.lev += 1;
  }
  const uint32_t o = by_lattice ? ol : (bx | (by << 1) | (bz << 2));
  cur.pending = (w & RT_CHILD_MASK) + o;
  cur.k += 1;
}

// descend_step() that also records the refined node on the path
template <typename R>
__device__ __forceinline__ void descend_step(Geo<R>& g, Cursor& cur, uint32_t w, R dx, R dy, R dz, const AncPath& P) {
  if (P.cap > 0 && cur.k < P.cap) P.a[cur.k * P.stride] = cur.pending;
  descend_step(g, cur, w, dx, dy, dz);
}

// Where the search for the neighbour starts after a crossing on axis a that
// changed the lattice coordinate from cold to cnew (only bits below hb + 1
// changed, hb the highest): the neighbour shares the ancestors above level
// lev - hb, and its ancestor at that level m is the sibling of ours on axis a
// (index +-2^a, the octet's children being in octant order).  hb = 0 is the
// sibling of the leaf itself; m <= 0 (the root coordinate changed) starts at
// the root cell.  Sets cur; the path stays the leaf's (a search from a stored
// ancestor or the root cell rewrites the levels below its start).
__device__ __forceinline__ void neighbour_start(const GridRegs& G, int lev, uint32_t idx, uint32_t cx, uint32_t cy,
                                                uint32_t cz, int a, bool plus, uint32_t moved, AncPath& P,
                                                Cursor& cur) {
  const bool a0 = a == 0, a1 = a == 1;
  const bool root_level = lev == 0;
  const bool near = root_level || moved < 2u;  // root-level neighbour or sibling: one load
  const uint32_t rx = cx >> lev, ry = cy >> lev, rz = cz >> lev;
  if (P.cap > 0 && !near) {
    // a branch, not selects: few crossings leave their octet on most grids
    // (with no path, cap = 0 at compile time, this block is not compiled)
    const int m = lev - (31 - __clz((int)moved));
    const bool up = m >= 1 && m < P.n;
    const uint32_t am = up ? P.a[m * P.stride] : 0u;
    cur.pending = up ? (plus ? am + (1u << a) : am - (1u << a)) : rx + G.rx * (ry + G.ry * rz);
    cur.k = up ? m : 0;
    P.n = up ? P.n : P.cap;
  } else {
    const uint32_t step = root_level ? (a0 ? 1u : (a1 ? G.rx : G.rx * G.ry)) : (1u << a);
    cur.pending = near ? (plus ? idx + step : idx - step) : rx + G.rx * (ry + G.ry * rz);
    cur.k = near ? lev : 0;
  }
}

// the node at the cursor is a leaf: if it is coarser than the lattice level,
// re-express the offsets in its units
template <typename R>
__device__ __forceinline__ void settle_leaf(Geo<R>& g, const Cursor& cur, uint32_t w, double r64) {
  if (cur.k < g.lev) {
    const int kk = g.lev - cur.k;
    const uint32_t m = (1u << kk) - 1u;
    const R s = Num<R>::pow2m(kk);
    g.fx = (R(g.cx & m) + g.fx) * s;
    g.fy = (R(g.cy & m) + g.fy) * s;
    g.fz = (R(g.cz & m) + g.fz) * s;
    g.cx >>= kk;
    g.cy >>= kk;
    g.cz >>= kk;
    g.lev = cur.k;
  }
  g.idx = cur.pending;
  g.rho = Num<R>::leaf_rho(w, r64);
}

// start at a point given in root-cell units (faces belong to the cell the
// direction points into); false if outside the root grid
template <typename R>
__device__ __forceinline__ bool place_root(const GridRegs& G, Geo<R>& g, Cursor& cur, R px, R py, R pz, R dx,
                                           R dy, R dz) {
  if (!(px >= R(0) && py >= R(0) && pz >= R(0) && px <= (R)G.rx && py <= (R)G.ry && pz <= (R)G.rz))
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
  if (g.cx >= G.rx || g.cy >= G.ry || g.cz >= G.rz) return false;
  cur.pending = g.cx + G.rx * (g.cy + G.ry * g.cz);
  cur.k = 0;
  return true;
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

// Cross the exit face on axis a; aim the cursor at the neighbour (the
// sibling in the same octet or the root-level neighbour with one load,
// otherwise a descent from the sibling of the deepest stored ancestor the
// neighbour does not share, or from the root cell: neighbour_start).  False
// when the package leaves the root grid.  Written with selects only: lanes
// crossing different axes do not diverge.  `moved` gets the bits of the lattice coordinate on axis a
// that changed (bit l + s set: the crossing left a block of 2^s cells of
// level l on that axis, e.g. a tile).
template <typename R>
__device__ __forceinline__ bool advance(const GridRegs& G, Geo<R>& g, Cursor& cur, int a, R t, R dx, R dy, R dz,
                                        uint32_t& moved, AncPath& P) {
  const bool a0 = a == 0, a1 = a == 1;
  const R da = a0 ? dx : (a1 ? dy : dz);
  const bool plus = da > R(0);
  const R fnew = plus ? R(0) : R(1);
  const R nfx = clamp01(g.fx + t * dx), nfy = clamp01(g.fy + t * dy), nfz = clamp01(g.fz + t * dz);
  g.fx = a0 ? fnew : nfx;
  g.fy = a1 ? fnew : nfy;
  g.fz = (!a0 && !a1) ? fnew : nfz;
  const uint32_t cold = a0 ? g.cx : (a1 ? g.cy : g.cz);
  const uint32_t cnew = plus ? cold + 1u : cold - 1u;
  g.cx = a0 ? cnew : g.cx;
  g.cy = a1 ? cnew : g.cy;
  g.cz = (!a0 && !a1) ? cnew : g.cz;
  moved = cold ^ cnew;
  // only axis a moved: inside while its root coordinate stays below the
  // root grid's size (a step below 0 wraps to a huge unsigned value)
  const bool inside = (cnew >> g.lev) < (a0 ? G.rx : (a1 ? G.ry : G.rz));
  neighbour_start(G, g.lev, g.idx, g.cx, g.cy, g.cz, a, plus, moved, P, cur);
  return inside;
}
template <typename R>
__device__ __forceinline__ bool advance(const GridRegs& G, Geo<R>& g, Cursor& cur, int a, R t, R dx, R dy, R dz,
                                        uint32_t& moved) {
  AncPath P = no_path();
  return advance(G, g, cur, a, t, dx, dy, dz, moved, P);
}
template <typename R>
__device__ __forceinline__ bool advance(const GridRegs& G, Geo<R>& g, Cursor& cur, int a, R t, R dx, R dy, R dz) {
  uint32_t moved;
  return advance(G, g, cur, a, t, dx, dy, dz, moved);
}

// advance() for a direction along axis a (the other two components zero):
// the offsets on the other axes do not move, so only axis a is updated
// (the same results as advance() with that direction)
template <typename R>
__device__ __forceinline__ bool advance_axis(const GridRegs& G, Geo<R>& g, Cursor& cur, int a, bool plus,
                                             AncPath& P) {
  const bool a0 = a == 0, a1 = a == 1;
  const R fnew = plus ? R(0) : R(1);
  g.fx = a0 ? fnew : g.fx;
  g.fy = a1 ? fnew : g.fy;
  g.fz = (!a0 && !a1) ? fnew : g.fz;
  const uint32_t cold = a0 ? g.cx : (a1 ? g.cy : g.cz);
  const uint32_t cnew = plus ? cold + 1u : cold - 1u;
  g.cx = a0 ? cnew : g.cx;
  g.cy = a1 ? cnew : g.cy;
  g.cz = (!a0 && !a1) ? cnew : g.cz;
  const bool inside = (cnew >> g.lev) < (a0 ? G.rx : (a1 ? G.ry : G.rz));
  neighbour_start(G, g.lev, g.idx, g.cx, g.cy, g.cz, a, plus, cold ^ cnew, P, cur);
  return inside;
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


// L2 residency hints (createpolicy + .L2::cache_hint): 0 none, 1 evict_last,
// 2 evict_first.  The node words of the grid are read at every crossing; the
// accumulator lines take a few consecutive deposits and are then not touched
// for a long time, so they are marked evict_first and do not push the node
// words out.
#ifndef RT_NODE_HINT
#define RT_NODE_HINT 1
#endif
#ifndef RT_RED_HINT
#define RT_RED_HINT 2
#endif
__device__ __forceinline__ uint32_t ld_node(const uint32_t* p) {
#if RT_NODE_HINT == 0
  return __ldg(p);
#else
  uint64_t pol;
#if RT_NODE_HINT == 1
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
#else
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
#endif
  uint32_t w;
  asm("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(w) : "l"(p), "l"(pol));
  return w;
#endif
}
__device__ __forceinline__ void red_acc(double* p, double v) {
#if RT_RED_HINT == 0
  atomicAdd(p, v);
#else
  uint64_t pol;
#if RT_RED_HINT == 1
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
#else
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
#endif
  asm volatile("red.global.add.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(pol) : "memory");
#endif
}

// f32 -> f64 for the accumulator reductions (one conversion per deposit;
// measured as fast as assembling the f64 bits on the integer pipe)
__device__ __forceinline__ double widen(float v) { return (double)v; }
__device__ __forceinline__ double widen(double v) { return v; }

template <typename R>
struct ObsGeom;
template <>
struct ObsGeom<float> {
  static __device__ __forceinline__ float k(const ObsDev& O, int a) { return O.kf[a]; }
  static __device__ __forceinline__ float ex(const ObsDev& O, int a) { return O.exf[a]; }
  static __device__ __forceinline__ float ey(const ObsDev& O, int a) { return O.eyf[a]; }
  static __device__ __forceinline__ float c(const ObsDev& O, int a) { return O.cf[a]; }
  static __device__ __forceinline__ float ip(const ObsDev& O, int a) { return O.inv_pixf[a]; }
};
template <>
struct ObsGeom<double> {
  static __device__ __forceinline__ double k(const ObsDev& O, int a) { return O.k[a]; }
  static __device__ __forceinline__ double ex(const ObsDev& O, int a) { return O.ex[a]; }
  static __device__ __forceinline__ double ey(const ObsDev& O, int a) { return O.ey[a]; }
  static __device__ __forceinline__ double c(const ObsDev& O, int a) { return O.c[a]; }
  static __device__ __forceinline__ double ip(const ObsDev& O, int a) { return O.inv_pix[a]; }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

}  // namespace rtk
