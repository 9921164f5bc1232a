// rt_dust.cu -- equilibrium dust temperatures and dust emission (Sects. 3.2
// and 4: a single dust component in equilibrium with the local radiation
// field; the emission of every cell is recomputed from its temperature in
// each Lambda-iteration step, Eq. 2).
//
// Per leaf the solve finds T with rho V E(T) = A, where
//   E(T) = 4 pi sum_i kappa_abs,i B_nu(nu_i, T) dnu_i     (erg/s/g)
// is the same for every cell.  It is tabulated once per call (log E and its
// slope on a uniform log-T grid, FP64) and each leaf inverts the cubic
// Hermite interpolant, so no leaf evaluates the Planck sum (GB300's FP64
// pipe is narrow); where E underflows at the cold end the exact sum is
// solved by safeguarded Newton instead.
#include "philox.cuh"
#include "rt_internal.cuh"

namespace rtk {

#define C_CGS 2.99792458e10
#define H_CGS 6.62607015e-27
#define K_CGS 1.380649e-16
#define FOUR_PI 12.566370614359172

// B_nu(T) and its temperature derivative
__device__ __forceinline__ void planck_and_deriv(double nu, double T, double* B, double* dB) {
  const double x = H_CGS * nu / (K_CGS * T);
  const double em1 = expm1(x);
  if (!(em1 < HUGE_VAL)) {  // Wien tail below the double range
    *B = 0.0;
    *dB = 0.0;
    return;
  }
  const double b = 2.0 * H_CGS * nu * nu * nu / (C_CGS * C_CGS) / em1;
  *B = b;
  *dB = b * x * (1.0 + 1.0 / em1) / T;
}

__device__ __forceinline__ double emission_per_mass(const double* lam, const double* kabs, const double* dnu, int nl,
                                                    double T, double* dEdT) {
  double s = 0.0, ds = 0.0;
  for (int i = 0; i < nl; ++i) {
    const double nu = C_CGS / (lam[i] * 1e-4);
    double B, dB;
    planck_and_deriv(nu, T, &B, &dB);
    s += kabs[i] * B * dnu[i];
    ds += kabs[i] * dB * dnu[i];
  }
  if (dEdT) *dEdT = FOUR_PI * ds;
  return FOUR_PI * s;
}

// Table of the emission per unit mass on a uniform grid in log T:
// tab[3i] = log T_i, tab[3i+1] = log E(T_i), tab[3i+2] = d log E / d log T.
// log E(log T) is smooth, so cubic Hermite interpolation between nodes
// (spacing ~1e-3 in log T for 8192 nodes) inverts it to ~1e-13 in T.
__global__ void table_kernel(const double* __restrict__ lam, const double* __restrict__ kabs,
                             const double* __restrict__ dnu, int nl, double Tmin, double Tmax, int n,
                             double* __restrict__ table) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = log(Tmin) + log(Tmax / Tmin) * (double)i / (double)(n - 1);
  const double T = exp(x);
  double dE;
  const double E = emission_per_mass(lam, kabs, dnu, nl, T, &dE);
  table[3 * i] = x;
  table[3 * i + 1] = E > 0.0 ? log(E) : -HUGE_VAL;
  table[3 * i + 2] = E > 0.0 ? T * dE / E : 0.0;
}

cudaError_t dust_table(const double* lam, const double* kabs, const double* dnu, int nl, double Tmin, double Tmax,
                       int n_table, double* table, cudaStream_t s) {
  const int B = 128;
  table_kernel<<<(n_table + B - 1) / B, B, 0, s>>>(lam, kabs, dnu, nl, Tmin, Tmax, n_table, table);
  return cudaGetLastError();
}

// exact safeguarded Newton on E(T) = target inside [Tl, Th] (used where the
// table has no finite logarithm, i.e. E underflows to 0 at the cold end)
__device__ double solve_exact(const double* lam, const double* kabs, const double* dnu, int nl, double target,
                              double Tl, double Th) {
  double T = 0.5 * (Tl + Th);
  for (int it = 0; it < 200; ++it) {
    double dE;
    const double E = emission_per_mass(lam, kabs, dnu, nl, T, &dE);
    const double f = E - target;
    if (f < 0.0) Tl = T;
    else Th = T;
    double Tn = dE > 0.0 ? T - f / dE : 0.5 * (Tl + Th);
    if (!(Tn > Tl && Tn < Th)) Tn = 0.5 * (Tl + Th);
    const double step = fabs(Tn - T);
    T = Tn;
    if (step <= 1e-14 * T || (Th - Tl) <= 1e-14 * Tl) break;
  }
  return T;
}

__global__ void temperature_kernel(const double* __restrict__ absorbed, int n_bins, long long n,
                                   const uint32_t* __restrict__ child, const double* __restrict__ rho64,
                                   const uint8_t* __restrict__ level, double h0, const double* __restrict__ lam,
                                   const double* __restrict__ kabs, const double* __restrict__ dnu, int nl,
                                   double Tmin, double Tmax, const double* __restrict__ table, int n_table,
                                   double* __restrict__ Tout) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  if (child[c]) {
    Tout[c] = 0.0;
    return;
  }
  double A = 0.0;
  for (int b = 0; b < n_bins; ++b) A += absorbed[(long long)b * n + c];
  const double h = ldexp(h0, -(int)level[c]);
  const double mass = rho64[c] * h * h * h;
  if (!(mass > 0.0) || !(A > 0.0)) {
    Tout[c] = Tmin;
    return;
  }
  const double Y = log(A / mass);
  if (!(Y > table[1])) {
    Tout[c] = Tmin;
    return;
  }
  if (Y >= table[3 * (n_table - 1) + 1]) {
    Tout[c] = Tmax;
    return;
  }
  // bracket: y_lo <= Y < y_hi (log E is increasing in log T)
  int lo = 0, hi = n_table - 1;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (table[3 * mid + 1] <= Y) lo = mid;
    else hi = mid;
  }
  const double x0 = table[3 * lo], y0 = table[3 * lo + 1], s0 = table[3 * lo + 2];
  const double x1 = table[3 * hi], y1 = table[3 * hi + 1], s1 = table[3 * hi + 2];
  if (!(y0 > -HUGE_VAL)) {
    Tout[c] = solve_exact(lam, kabs, dnu, nl, A / mass, exp(x0), exp(x1));
    return;
  }
  // invert the cubic Hermite interpolant p(t), t in [0,1], by Newton
  const double hx = x1 - x0;
  const double m0 = s0 * hx, m1 = s1 * hx;
  double t = (Y - y0) / (y1 - y0);
  for (int it = 0; it < 6; ++it) {
    const double t2 = t * t, t3 = t2 * t;
    const double p = (2 * t3 - 3 * t2 + 1) * y0 + (t3 - 2 * t2 + t) * m0 + (-2 * t3 + 3 * t2) * y1 + (t3 - t2) * m1;
    const double dp = (6 * t2 - 6 * t) * y0 + (3 * t2 - 4 * t + 1) * m0 + (-6 * t2 + 6 * t) * y1 + (3 * t2 - 2 * t) * m1;
    double tn = dp > 0.0 ? t - (p - Y) / dp : t;
    tn = tn < 0.0 ? 0.0 : (tn > 1.0 ? 1.0 : tn);
    const bool done = fabs(tn - t) < 1e-15;
    t = tn;
    if (done) break;
  }
  Tout[c] = exp(x0 + t * hx);
}

cudaError_t dust_temperature(const double* absorbed, int n_bins, long long n_cells, const uint32_t* child,
                             const double* rho64, const uint8_t* level, double h0, const double* lam, const double* kabs,
                             const double* dnu, int nl, double Tmin, double Tmax, const double* table, int n_table,
                             double* T, cudaStream_t s) {
  const unsigned B = 128;
  temperature_kernel<<<(unsigned)((n_cells + B - 1) / B), B, 0, s>>>(absorbed, n_bins, n_cells, child, rho64, level,
                                                                     h0, lam, kabs, dnu, nl, Tmin, Tmax, table,
                                                                     n_table, T);
  return cudaGetLastError();
}

__global__ void emission_kernel(const double* __restrict__ T, long long n, const uint32_t* __restrict__ child,
                                const double* __restrict__ rho64, const uint8_t* __restrict__ level, double h0,
                                const double* __restrict__ lam, const double* __restrict__ kabs,
                                const double* __restrict__ dnu, int nl, double* __restrict__ em) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const double Tc = T[c];
  double pref = 0.0;
  if (!child[c] && Tc > 0.0) {
    const double h = ldexp(h0, -(int)level[c]);
    pref = FOUR_PI * rho64[c] * h * h * h;
  }
  for (int b = 0; b < nl; ++b) {
    double v = 0.0;
    if (pref > 0.0) {
      double B, dB;
      planck_and_deriv(C_CGS / (lam[b] * 1e-4), Tc, &B, &dB);
      v = pref * kabs[b] * B * dnu[b];
    }
    em[(long long)b * n + c] = v;
  }
}

cudaError_t dust_emission(const double* T, long long n_cells, const uint32_t* child, const double* rho64,
                          const uint8_t* level, double h0, const double* lam, const double* kabs, const double* dnu,
                          int nl, double* emission, cudaStream_t s) {
  const unsigned B = 128;
  emission_kernel<<<(unsigned)((n_cells + B - 1) / B), B, 0, s>>>(T, n_cells, child, rho64, level, h0, lam, kabs, dnu,
                                                                  nl, emission);
  return cudaGetLastError();
}

// per-bin totals of the emission of emission_kernel, without storing it
__global__ void emission_totals_kernel(const double* __restrict__ T, long long n, const uint32_t* __restrict__ child,
                                       const double* __restrict__ rho64, const uint8_t* __restrict__ level, double h0,
                                       const double* __restrict__ lam, const double* __restrict__ kabs,
                                       const double* __restrict__ dnu, int nl, double* __restrict__ tot) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double pref = 0.0, Tc = 0.0;
  if (c < n) {
    Tc = T[c];
    if (!child[c] && Tc > 0.0) {
      const double h = ldexp(h0, -(int)level[c]);
      pref = FOUR_PI * rho64[c] * h * h * h;
    }
  }
  for (int b = 0; b < nl; ++b) {
    double v = 0.0;
    if (pref > 0.0) {
      double B, dB;
      planck_and_deriv(C_CGS / (lam[b] * 1e-4), Tc, &B, &dB);
      v = pref * kabs[b] * B * dnu[b];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(tot + b, v);
  }
}

cudaError_t dust_emission_totals(const double* T, long long n_cells, const uint32_t* child, const double* rho64,
                                 const uint8_t* level, double h0, const double* lam, const double* kabs,
                                 const double* dnu, int nl, double* tot, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(tot, 0, sizeof(double) * (size_t)nl, s);
  if (e != cudaSuccess || n_cells <= 0) return e;
  const unsigned B = 128;
  emission_totals_kernel<<<(unsigned)((n_cells + B - 1) / B), B, 0, s>>>(T, n_cells, child, rho64, level, h0, lam,
                                                                         kabs, dnu, nl, tot);
  return cudaGetLastError();
}

__global__ void max_rel_change_kernel(const double* __restrict__ T, const double* __restrict__ Tp,
                                      const unsigned int* __restrict__ hits, const uint32_t* __restrict__ child,
                                      long long n, double min_hits, double* out) {
  double m = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (child[i] || (hits && (double)hits[i] < min_hits)) continue;
    const double tp = Tp[i];
    if (tp > 0.0) m = fmax(m, fabs(T[i] - tp) / tp);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
  // non-negative doubles order like their bit patterns
  if ((threadIdx.x & 31) == 0 && m > 0.0)
    atomicMax(reinterpret_cast<unsigned long long*>(out), (unsigned long long)__double_as_longlong(m));
}

cudaError_t max_rel_change(const double* T, const double* T_prev, const unsigned int* hits, const uint32_t* child,
                           long long n, double min_hits, double* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  max_rel_change_kernel<<<1024, 256, 0, s>>>(T, T_prev, hits, child, n, min_hits, out);
  return cudaGetLastError();
}

__global__ void dust_counts_kernel(const double* __restrict__ em, long long n, const double* __restrict__ w,
                                   uint32_t k0, uint32_t k1, uint32_t src, long long* __restrict__ first) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (c > n) return;
  long long* row = first + (long long)b * (n + 1);
  if (c == n) {
    row[n] = 0;
    return;
  }
  const double e = em[(long long)b * n + c];
  const double wb = w[b];
  long long k = 0;
  if (e > 0.0 && wb > 0.0) {
    const uint4 r = philox4x32_10(make_uint4((uint32_t)c, 0x80000000u, 0u, (src << 16) | (uint32_t)b), k0, k1);
    const double u = ((double)r.x + 0.5) * 2.3283064365386963e-10;
    k = (long long)floor(e / wb + u);
  }
  row[c] = k;
}

cudaError_t dust_counts(const double* emission, long long n, int nl, const double* w, uint32_t k0, uint32_t k1,
                        uint32_t src, long long* first, cudaStream_t s) {
  if (n <= 0 || nl <= 0) return cudaSuccess;
  const unsigned B = 256;
  dust_counts_kernel<<<dim3((unsigned)((n + 1 + B - 1) / B), (unsigned)nl), B, 0, s>>>(emission, n, w, k0, k1, src,
                                                                                      first);
  return cudaGetLastError();
}

__global__ void row_sum_kernel(const double* __restrict__ data, long long n, double* __restrict__ out) {
  const long long row = blockIdx.y;
  double v = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    v += data[row * n + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(out + row, v);
}

cudaError_t row_sums_f64(const double* data, int n_rows, long long n, double* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * (size_t)n_rows, s);
  if (e != cudaSuccess) return e;
  long long blocks = (n + 255) / 256;
  if (blocks > 512) blocks = 512;
  if (blocks < 1) blocks = 1;
  row_sum_kernel<<<dim3((unsigned)blocks, n_rows), 256, 0, s>>>(data, n, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------
// subiterations (Sect. 3.2, App. B)
// ------------------------------------------------------------------------
// temperatures that emit in a subiteration: the cells below level L
__global__ void mask_levels_kernel(const double* __restrict__ T, const uint8_t* __restrict__ level, long long n,
                                   int L, double* __restrict__ out) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n) out[c] = (int)level[c] > L ? T[c] : 0.0;
}

cudaError_t mask_levels(const double* T, const uint8_t* level, long long n, int L, double* out, cudaStream_t s) {
  mask_levels_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(T, level, n, L, out);
  return cudaGetLastError();
}

// Eq. 9: the field of a cell, constant sources plus the dust field of every
// level array (a cell holds nothing above its own level)
__global__ void sum_levels_kernel(const double* __restrict__ I, int n_levels, long long n,
                                  const double* __restrict__ A_star, double* __restrict__ A) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  double v = A_star[c];
  for (int i = 0; i < n_levels; ++i) v += I[(long long)i * n + c];
  A[c] = v;
}

cudaError_t sum_levels(const double* I, int n_levels, long long n, const double* A_star, double* A, cudaStream_t s) {
  sum_levels_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(I, n_levels, n, A_star, A);
  return cudaGetLastError();
}

// emission per unit mass E(T) from the table of log E(log T) (cubic Hermite)
__device__ __forceinline__ double table_emission(double T, const double* __restrict__ table, int n_table) {
  if (!(T > 0.0)) return 0.0;
  const double x0 = table[0], hx = table[3] - table[0];
  const double x = log(T);
  int i = (int)floor((x - x0) / hx);
  i = i < 0 ? 0 : (i > n_table - 2 ? n_table - 2 : i);
  const double y0 = table[3 * i + 1], y1 = table[3 * i + 4];
  if (!(y0 > -HUGE_VAL)) return 0.0;
  const double tt = (x - table[3 * i]) / hx, m0 = table[3 * i + 2] * hx, m1 = table[3 * i + 5] * hx;
  const double t2 = tt * tt, t3 = t2 * tt;
  return exp((2 * t3 - 3 * t2 + 1) * y0 + (t3 - 2 * t2 + tt) * m0 + (-2 * t3 + 3 * t2) * y1 + (t3 - t2) * m1);
}

// Eq. 3 with a diagonal operator per frequency (Sect. 3.1: the system
// decouples into one equation per cell, with one unknown per frequency):
// Lambda_b of a cell is the fraction of the energy its own bin-b packages
// carried that they left in it (self_b / emitted_b, two tallies of the same
// packages), capped at lam_max; the cell's temperature then solves
//   sum_b (1 - Lambda_b) E_b(T) = A - sum_b Lambda_b emitted_b.
// Only cells that sent at least min_count packages use it (flag 1); the
// others keep the plain step E(T) = A.  A bin in which such a cell sent no
// package takes the largest Lambda_j of the cell's sampled bins with
// kabs_j <= kabs_b (0 if none): self-absorption grows with opacity, and a
// weight of 1 would count that bin's emission at the new T as escaping.
__device__ __forceinline__ double ali_lambda(const double* __restrict__ self, const double* __restrict__ emitted,
                                             double lam_max, long long n, long long c, int b) {
  const double e = emitted[(long long)b * n + c];
  return e > 0.0 ? fmin(self[(long long)b * n + c] / e, lam_max) : -1.0;
}

__global__ void ali_weights_kernel(const double* __restrict__ A, const double* __restrict__ self,
                                   const double* __restrict__ emitted, const unsigned int* __restrict__ count,
                                   const double* __restrict__ kabs, unsigned int min_count, double lam_max, int nl,
                                   long long n, double* __restrict__ rhs, double* __restrict__ w,
                                   uint8_t* __restrict__ use) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const bool on = count[c] >= min_count;
  double r = A[c];
  for (int b = 0; b < nl; ++b) {
    double lam = on ? ali_lambda(self, emitted, lam_max, n, c, b) : 0.0;
    if (lam >= 0.0) {
      r -= lam * emitted[(long long)b * n + c];
    } else {
      lam = 0.0;
      for (int j = 0; j < nl; ++j)
        if (kabs[j] <= kabs[b]) lam = fmax(lam, ali_lambda(self, emitted, lam_max, n, c, j));
    }
    w[(long long)b * n + c] = 1.0 - lam;
  }
  rhs[c] = r;
  use[c] = on ? 1 : 0;
}

cudaError_t ali_weights(const double* A, const double* self, const double* emitted, const unsigned int* count,
                        const double* kabs, unsigned int min_count, double lam_max, int nl, long long n, double* rhs,
                        double* w, uint8_t* use, cudaStream_t s) {
  ali_weights_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(A, self, emitted, count, kabs, min_count, lam_max, nl,
                                                                  n, rhs, w, use);
  return cudaGetLastError();
}

// sum_b w_b E_b(T) per unit mass and its derivative
__device__ __forceinline__ double weighted_emission(const double* lam, const double* kabs, const double* dnu,
                                                    const double* __restrict__ w, long long n, long long c, int nl,
                                                    double T, double* dEdT) {
  double s = 0.0, ds = 0.0;
  for (int b = 0; b < nl; ++b) {
    double B, dB;
    planck_and_deriv(C_CGS / (lam[b] * 1e-4), T, &B, &dB);
    const double k = w[(long long)b * n + c] * kabs[b] * dnu[b];
    s += k * B;
    ds += k * dB;
  }
  *dEdT = FOUR_PI * ds;
  return FOUR_PI * s;
}

// The ALI cells' temperatures: safeguarded Newton (bisection when a step
// leaves the bracket) on sum_b w_b E_b(T) = rhs / (rho V), starting from the
// plain solve's T; T_min / T_max where the target lies outside.
__global__ void temperature_weighted_kernel(const double* __restrict__ rhs, const double* __restrict__ w,
                                            const uint8_t* __restrict__ use, long long n,
                                            const uint32_t* __restrict__ child, const double* __restrict__ rho64,
                                            const uint8_t* __restrict__ level, double h0,
                                            const double* __restrict__ lam, const double* __restrict__ kabs,
                                            const double* __restrict__ dnu, int nl, double Tmin, double Tmax,
                                            double* __restrict__ T) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n || !use[c] || child[c]) return;
  const double h = ldexp(h0, -(int)level[c]);
  const double mass = rho64[c] * h * h * h;
  if (!(mass > 0.0) || !(rhs[c] > 0.0)) {
    T[c] = Tmin;
    return;
  }
  const double target = rhs[c] / mass;
  double d;
  if (target <= weighted_emission(lam, kabs, dnu, w, n, c, nl, Tmin, &d)) {
    T[c] = Tmin;
    return;
  }
  if (target >= weighted_emission(lam, kabs, dnu, w, n, c, nl, Tmax, &d)) {
    T[c] = Tmax;
    return;
  }
  double lo = Tmin, hi = Tmax;
  double t = T[c] > Tmin && T[c] < Tmax ? T[c] : sqrt(Tmin * Tmax);
  for (int it = 0; it < 200; ++it) {
    double dE;
    const double f = weighted_emission(lam, kabs, dnu, w, n, c, nl, t, &dE) - target;
    if (f < 0.0) lo = t;
    else hi = t;
    double tn = dE > 0.0 ? t - f / dE : 0.5 * (lo + hi);
    if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
    const double step = fabs(tn - t);
    t = tn;
    if (step <= 1e-14 * t || (hi - lo) <= 1e-14 * lo) break;
  }
  T[c] = t;
}

cudaError_t dust_temperature_weighted(const double* rhs, const double* w, const uint8_t* use, long long n,
                                      const uint32_t* child, const double* rho64, const uint8_t* level, double h0,
                                      const double* lam, const double* kabs, const double* dnu, int nl, double Tmin,
                                      double Tmax, double* T, cudaStream_t s) {
  temperature_weighted_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(rhs, w, use, n, child, rho64, level, h0, lam,
                                                                          kabs, dnu, nl, Tmin, Tmax, T);
  return cudaGetLastError();
}

// Energy imbalance |absorbed - emitted|, mass and emission, summed over the
// leaves at level <= L (out[0], out[1], out[4]) and below L (out[2], out[3],
// out[5]).  The emission is rho V E(T) with E from the tabulated
// log E(log T) (cubic Hermite).
__global__ void imbalance_kernel(const double* __restrict__ A, const double* __restrict__ T,
                                 const uint32_t* __restrict__ child, const double* __restrict__ rho64,
                                 const uint8_t* __restrict__ level, double h0, const double* __restrict__ table,
                                 int n_table, long long n, int L, double* __restrict__ out) {
  double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    if (child[c]) continue;
    const double h = ldexp(h0, -(int)level[c]);
    const double mass = rho64[c] * h * h * h;
    const double E = table_emission(T[c], table, n_table);
    const int gi = (int)level[c] > L ? 2 : 0;
    v[gi] += fabs(A[c] - mass * E);
    v[gi + 1] += mass;
    v[4 + gi / 2] += mass * E;
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    double x = v[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
    if ((threadIdx.x & 31) == 0 && x != 0.0) atomicAdd(out + k, x);
  }
}

cudaError_t level_imbalance(const double* A, const double* T, const uint32_t* child, const double* rho64,
                            const uint8_t* level, double h0, const double* table, int n_table, long long n, int L,
                            double* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, 6 * sizeof(double), s);
  if (e != cudaSuccess) return e;
  imbalance_kernel<<<1024, 256, 0, s>>>(A, T, child, rho64, level, h0, table, n_table, n, L, out);
  return cudaGetLastError();
}

}  // namespace rtk
