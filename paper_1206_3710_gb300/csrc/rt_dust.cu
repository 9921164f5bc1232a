// rt_dust.cu -- equilibrium dust temperatures and dust emission (Sects. 3.2
// and 4: a single dust component in equilibrium with the local radiation
// field; the emission of every cell is recomputed from its temperature in
// each Lambda-iteration step, Eq. 2).
//
// Per leaf the solve finds T with rho V E(T) = A, where
//   E(T) = 4 pi sum_i kappa_abs,i B_nu(nu_i, T) dnu_i     (erg/s/g)
// is the same for every cell.  A tabulated E on a log-T grid gives the
// bracket; a safeguarded Newton iteration in FP64 on the exact sum
// finishes to 1e-13 relative.
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

__global__ void table_kernel(const double* __restrict__ lam, const double* __restrict__ kabs,
                             const double* __restrict__ dnu, int nl, double Tmin, double Tmax, int n,
                             double* __restrict__ table) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double T = Tmin * exp(log(Tmax / Tmin) * (double)i / (double)(n - 1));
  table[i] = emission_per_mass(lam, kabs, dnu, nl, T, nullptr);
}

cudaError_t dust_table(const double* lam, const double* kabs, const double* dnu, int nl, double Tmin, double Tmax,
                       int n_table, double* table, cudaStream_t s) {
  const int B = 128;
  table_kernel<<<(n_table + B - 1) / B, B, 0, s>>>(lam, kabs, dnu, nl, Tmin, Tmax, n_table, table);
  return cudaGetLastError();
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
  const double target = A / mass;
  if (target <= table[0]) {
    Tout[c] = Tmin;
    return;
  }
  if (target >= table[n_table - 1]) {
    Tout[c] = Tmax;
    return;
  }
  // bracket from the table (E is increasing in T)
  int lo = 0, hi = n_table - 1;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (table[mid] <= target) lo = mid;
    else hi = mid;
  }
  const double lr = log(Tmax / Tmin) / (double)(n_table - 1);
  double Tl = Tmin * exp(lr * lo), Th = Tmin * exp(lr * hi);
  if (lo == 0) Tl = Tmin;
  if (hi == n_table - 1) Th = Tmax;
  // start by log-log interpolation inside the bracket
  double T = Tl * exp(log(Th / Tl) * log(target / table[lo]) / log(table[hi] / table[lo]));
  if (!(T > Tl && T < Th)) T = 0.5 * (Tl + Th);
  for (int it = 0; it < 100; ++it) {
    double dE;
    const double E = emission_per_mass(lam, kabs, dnu, nl, T, &dE);
    const double f = E - target;
    if (f < 0.0) Tl = T;
    else Th = T;
    double Tn = T - f / dE;
    if (!(Tn > Tl && Tn < Th)) Tn = 0.5 * (Tl + Th);
    const double step = fabs(Tn - T);
    T = Tn;
    if (step <= 1e-13 * T || (Th - Tl) <= 1e-13 * Tl) break;
  }
  Tout[c] = T;
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

}  // namespace rtk
