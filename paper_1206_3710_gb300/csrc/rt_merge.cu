// rt_merge.cu -- the hierarchical model built bottom-up from a
// full-resolution cube (Sect. 4.1).
//
// Eight cells of level l+1 are combined into their level-l parent when all
// eight are undivided, the parent's optical thickness kappa * rho_mean * h_l
// is at most tau_max (0.05 in the V band in Sect. 4.1) and the density
// contrast rho_max / rho_min over the full-resolution cells it covers is
// below contrast_max (30 in Sect. 4.1).  The combined density is the mean of
// the eight, summed in octant order o = ox + 2 oy + 4 oz.
//
// Pass 1 (bottom-up, one launch per level): mean, min, max and the
// "undivided" flag of every cell of every level on full lattices.
// Pass 2 (top-down): the level-ordered tree description -- the root cells
// x-fastest, then the children of each divided cell in the order of their
// parents, in octant order -- by one exclusive scan of the divide flags per
// level.
#include "rt_internal.cuh"

#include <vector>

namespace rtk {

template <bool FINEST>
__global__ void merge_up_kernel(const double* __restrict__ cm, const double* __restrict__ cmn,
                                const double* __restrict__ cmx, const uint8_t* __restrict__ cleaf, int nx, int ny,
                                int nz, double kappa, double h, double tau_max, double cmax, double* __restrict__ m,
                                double* __restrict__ mn, double* __restrict__ mx, uint8_t* __restrict__ leaf) {
  const long long n = (long long)nx * ny * nz;
  const long long cnx = 2ll * nx, cny = 2ll * ny;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long x = i % nx, r = i / nx, y = r % ny, z = r / ny;
    double acc = 0.0, lo = 0.0, hi = 0.0;
    bool all = true;
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      const long long c = (2 * x + (o & 1)) + cnx * ((2 * y + ((o >> 1) & 1)) + cny * (2 * z + ((o >> 2) & 1)));
      const double v = cm[c];
      const double a = FINEST ? v : cmn[c], b = FINEST ? v : cmx[c];
      if (o == 0) {
        acc = v;
        lo = a;
        hi = b;
      } else {
        acc = acc + v;
        lo = fmin(lo, a);
        hi = fmax(hi, b);
      }
      if (!FINEST) all = all && cleaf[c] != 0;
    }
    const double mean = acc / 8.0;
    const double tau = kappa * mean * h;
    const bool tau_ok = tau <= tau_max;
    const bool c_ok = lo > 0.0 ? hi < cmax * lo : hi == 0.0;
    m[i] = mean;
    mn[i] = lo;
    mx[i] = hi;
    leaf[i] = (all && tau_ok && c_ok) ? 1 : 0;
  }
}

// the cells of one level of the description (lattice indices in list):
// divide flag and density
__global__ void merge_emit_kernel(const unsigned long long* __restrict__ list, long long n,
                                  const uint8_t* __restrict__ leaf, const double* __restrict__ mean,
                                  uint8_t* __restrict__ flags, double* __restrict__ dens) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long c = list[i];
  flags[i] = leaf ? (leaf[c] ? 0 : 1) : 0;
  dens[i] = mean[c];
}

// the eight children of every divided cell, at 8 * (divided cells before it)
__global__ void merge_expand_kernel(const unsigned long long* __restrict__ list, long long n,
                                    const uint8_t* __restrict__ flags, const unsigned long long* __restrict__ excl,
                                    int nx, int ny, unsigned long long* __restrict__ child) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !flags[i]) return;
  const unsigned long long c = list[i];
  const unsigned long long x = c % (unsigned)nx, r = c / (unsigned)nx, y = r % (unsigned)ny, z = r / (unsigned)ny;
  const unsigned long long cnx = 2ull * nx, cny = 2ull * ny;
  const unsigned long long b = 8ull * excl[i];
#pragma unroll
  for (int o = 0; o < 8; ++o)
    child[b + o] = (2 * x + (o & 1)) + cnx * ((2 * y + ((o >> 1) & 1)) + cny * (2 * z + ((o >> 2) & 1)));
}

__global__ void iota_kernel(unsigned long long* __restrict__ out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (unsigned long long)i;
}

static unsigned grid_of(long long n) { return (unsigned)std::min<long long>((n + 255) / 256, 1ll << 20); }

int merge_uniform(const int* root, double h0, int L, const double* rho, double kappa, double tau_max, double cmax,
                  long long cap, uint8_t* flags_host, double* dens_host, long long* n_ref_host, int* n_levels,
                  long long* n_cells, cudaStream_t s) {
  const long long n0 = (long long)root[0] * root[1] * root[2];
  std::vector<long long> nl(L + 1);
  for (int l = 0; l <= L; ++l) nl[l] = n0 << (3 * l);
  std::vector<void*> owned;
  auto alloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(bytes, 256)) != cudaSuccess) return nullptr;
    owned.push_back(p);
    return p;
  };
  auto cleanup = [&]() {
    for (void* p : owned) cudaFree(p);
  };
  // pass 1: levels L-1 .. 0
  std::vector<double*> m(L + 1), mn(L + 1), mx(L + 1);
  std::vector<uint8_t*> lf(L + 1, nullptr);
  m[L] = const_cast<double*>(rho);
  for (int l = L - 1; l >= 0; --l) {
    m[l] = static_cast<double*>(alloc(sizeof(double) * nl[l]));
    mn[l] = static_cast<double*>(alloc(sizeof(double) * nl[l]));
    mx[l] = static_cast<double*>(alloc(sizeof(double) * nl[l]));
    lf[l] = static_cast<uint8_t*>(alloc(nl[l]));
    if (!m[l] || !mn[l] || !mx[l] || !lf[l]) {
      cleanup();
      return set_error(RT_ERR_OOM, "rt_merge_uniform: device allocation failed");
    }
    const int nx = root[0] << l, ny = root[1] << l, nz = root[2] << l;
    const double h = std::ldexp(h0, -l);
    if (l == L - 1)
      merge_up_kernel<true><<<grid_of(nl[l]), 256, 0, s>>>(m[l + 1], nullptr, nullptr, nullptr, nx, ny, nz, kappa, h,
                                                            tau_max, cmax, m[l], mn[l], mx[l], lf[l]);
    else
      merge_up_kernel<false><<<grid_of(nl[l]), 256, 0, s>>>(m[l + 1], mn[l + 1], mx[l + 1], lf[l + 1], nx, ny, nz,
                                                             kappa, h, tau_max, cmax, m[l], mn[l], mx[l], lf[l]);
    if (cudaGetLastError() != cudaSuccess) {
      cleanup();
      return set_error(RT_ERR_CUDA, "rt_merge_uniform: merge kernel launch failed");
    }
  }
  // pass 2: level-ordered description
  const long long nmax = nl[L];
  unsigned long long* list_a = static_cast<unsigned long long*>(alloc(sizeof(unsigned long long) * nmax));
  unsigned long long* list_b = static_cast<unsigned long long*>(alloc(sizeof(unsigned long long) * nmax));
  unsigned long long* excl = static_cast<unsigned long long*>(alloc(sizeof(unsigned long long) * nmax));
  uint8_t* fl = static_cast<uint8_t*>(alloc(nmax));
  double* de = static_cast<double*>(alloc(sizeof(double) * nmax));
  const size_t tb = scan_tmp_bytes(nmax);
  void* tmp = alloc(tb);
  if (!list_a || !list_b || !excl || !fl || !de || !tmp) {
    cleanup();
    return set_error(RT_ERR_OOM, "rt_merge_uniform: device allocation failed");
  }
  iota_kernel<<<grid_of(n0), 256, 0, s>>>(list_a, n0);
  long long n = n0, off = 0;
  int lev = 0;
  for (int l = 0; l <= L; ++l) {
    lev = l + 1;
    if (off + n > cap) {
      // keep counting the cells without writing them
      flags_host = nullptr;
      dens_host = nullptr;
    }
    merge_emit_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(list_a, n, l < L ? lf[l] : nullptr, m[l], fl, de);
    unsigned long long tot = 0;
    cudaError_t e = cudaSuccess;
    if (l < L) {
      e = scan_flags_u8(fl, n, excl, tmp, tb, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(&tot, excl + (n - 1), sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    }
    uint8_t last = 0;
    if (e == cudaSuccess && l < L) e = cudaMemcpyAsync(&last, fl + (n - 1), 1, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && flags_host) e = cudaMemcpyAsync(flags_host + off, fl, n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && dens_host)
      e = cudaMemcpyAsync(dens_host + off, de, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      cleanup();
      return set_error(RT_ERR_CUDA, "rt_merge_uniform: CUDA error in the ordering pass");
    }
    const long long n_div = l < L ? (long long)tot + last : 0;
    n_ref_host[l] = n_div;
    off += n;
    if (n_div == 0) break;
    merge_expand_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(list_a, n, fl, excl, root[0] << l, root[1] << l,
                                                                    list_b);
    std::swap(list_a, list_b);
    n = 8 * n_div;
  }
  cudaError_t e = cudaStreamSynchronize(s);
  cleanup();
  if (e != cudaSuccess) return set_error(RT_ERR_CUDA, "rt_merge_uniform: CUDA error");
  *n_levels = lev;
  *n_cells = off;
  if (off > cap) return set_error(RT_ERR_INVALID, "rt_merge_uniform: the description needs more cells than cap_cells");
  return RT_OK;
}

}  // namespace rtk
