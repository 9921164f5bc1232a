// rt_grid.cu -- flattening the nested-grid tree into device arrays, and
// the prefix scans used by the grid build and the emission sampler.
//
// Sect. 2.1 builds a subgrid identification array per grid before the
// simulation; here the whole octree is one level-ordered array set.  With
// the children of the k-th refined cell (counted over all levels in level
// order) stored at n0 + 8k, a single exclusive scan of the refine flags
// gives every child pointer.
#include "rt_internal.cuh"

namespace rtk {

static constexpr int SCAN_THREADS = 256;
static constexpr int SCAN_ITEMS = 16;
static constexpr long long SCAN_CHUNK = (long long)SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T n = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

// block-wide exclusive scan of one value per thread; returns the block total
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* total) {
  __shared__ T warp_tot[SCAN_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const T inc = warp_incl_scan(v);
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T w = lane < SCAN_THREADS / 32 ? warp_tot[lane] : T(0);
    const T wi = warp_incl_scan(w);
    if (lane < SCAN_THREADS / 32) warp_tot[lane] = wi - w;
    if (lane == SCAN_THREADS / 32 - 1) *total = wi;
  }
  __syncthreads();
  const T res = inc - v + warp_tot[wid];
  __syncthreads();
  return res;
}

// per row (blockIdx.y): scan chunks of SCAN_CHUNK elements; out gets the
// in-chunk prefix (exclusive or inclusive), sums[row][chunk] the chunk total
template <typename Tin, typename Tout, bool INCL>
__global__ void __launch_bounds__(SCAN_THREADS) scan_chunks(const Tin* __restrict__ in, long long n,
                                                            Tout* __restrict__ out, Tout* __restrict__ sums,
                                                            long long n_chunks) {
  __shared__ Tout tot;
  const long long row = blockIdx.y;
  const Tin* rin = in + row * n;
  Tout* rout = out + row * n;
  const long long base = (long long)blockIdx.x * SCAN_CHUNK + (long long)threadIdx.x * SCAN_ITEMS;
  Tout v[SCAN_ITEMS];
  Tout s = Tout(0);
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const long long j = base + i;
    v[i] = j < n ? (Tout)rin[j] : Tout(0);
    s += v[i];
  }
  Tout run = block_excl_scan<Tout>(s, &tot);
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const long long j = base + i;
    if (INCL) run += v[i];
    if (j < n) rout[j] = run;
    if (!INCL) run += v[i];
  }
  if (threadIdx.x == 0) sums[row * n_chunks + blockIdx.x] = tot;
}

template <typename T>
__global__ void add_chunk_offsets(T* __restrict__ out, long long n, const T* __restrict__ offs, long long n_chunks) {
  const long long row = blockIdx.y;
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  out[row * n + j] += offs[row * n_chunks + j / SCAN_CHUNK];
}

static long long chunks_of(long long n) { return (n + SCAN_CHUNK - 1) / SCAN_CHUNK; }

// bytes of temporary storage for an exclusive/inclusive scan of rows x n
template <typename T>
static size_t scan_tmp(int rows, long long n) {
  size_t bytes = 0;
  long long m = n;
  while (true) {
    const long long c = chunks_of(m);
    bytes += (size_t)rows * (size_t)c * sizeof(T) * 2 + 256;
    if (c <= 1) break;
    m = c;
  }
  return bytes;
}

// scan rows x n; chunk totals are scanned recursively (exclusive) and added
template <typename Tin, typename T, bool INCL>
static cudaError_t scan_rows(const Tin* in, T* out, int rows, long long n, char* tmp, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const long long c = chunks_of(n);
  T* sums = reinterpret_cast<T*>(tmp);
  T* offs = sums + (size_t)rows * c;
  char* next = reinterpret_cast<char*>(offs + (size_t)rows * c);
  next += (256 - ((uintptr_t)next & 255)) & 255;
  scan_chunks<Tin, T, INCL><<<dim3((unsigned)c, rows), SCAN_THREADS, 0, s>>>(in, n, out, sums, c);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || c == 1) return e;
  e = scan_rows<T, T, false>(sums, offs, rows, c, next, s);
  if (e != cudaSuccess) return e;
  const unsigned B = 256;
  add_chunk_offsets<T><<<dim3((unsigned)((n + B - 1) / B), rows), B, 0, s>>>(out, n, offs, c);
  return cudaGetLastError();
}

size_t scan_tmp_bytes(long long n) { return scan_tmp<unsigned long long>(1, n) + 512; }

cudaError_t scan_flags_u8(const uint8_t* flags, long long n, unsigned long long* excl, void* tmp, size_t tmp_bytes,
                          cudaStream_t s) {
  if (tmp_bytes < scan_tmp_bytes(n)) return cudaErrorInvalidValue;
  char* t = reinterpret_cast<char*>(tmp);
  t += (256 - ((uintptr_t)t & 255)) & 255;
  return scan_rows<uint8_t, unsigned long long, false>(flags, excl, 1, n, t, s);
}

size_t scan_rows_tmp_bytes(int n_rows, long long n) { return scan_tmp<double>(n_rows, n) + 512; }

cudaError_t scan_rows_i64_excl(long long* data, int n_rows, long long n, void* tmp, size_t tmp_bytes, cudaStream_t s) {
  if (tmp_bytes < scan_rows_tmp_bytes(n_rows, n)) return cudaErrorInvalidValue;
  char* t = reinterpret_cast<char*>(tmp);
  t += (256 - ((uintptr_t)t & 255)) & 255;
  return scan_rows<long long, long long, false>(data, data, n_rows, n, t, s);
}

cudaError_t scan_rows_f64(double* data, int n_rows, long long n, void* tmp, size_t tmp_bytes, cudaStream_t s) {
  if (tmp_bytes < scan_rows_tmp_bytes(n_rows, n)) return cudaErrorInvalidValue;
  char* t = reinterpret_cast<char*>(tmp);
  t += (256 - ((uintptr_t)t & 255)) & 255;
  // in-place is safe: each chunk reads its inputs into registers before writing
  return scan_rows<double, double, true>(data, data, n_rows, n, t, s);
}

// ------------------------------------------------------------------------
__global__ void children_kernel(const uint8_t* __restrict__ flags, const unsigned long long* __restrict__ excl,
                                long long n, long long n0, uint32_t* __restrict__ child) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  child[i] = flags[i] ? (uint32_t)(n0 + 8ll * (long long)excl[i]) : 0u;
}

cudaError_t build_children(const uint8_t* flags, const unsigned long long* excl, long long n, long long n0,
                           uint32_t* child, cudaStream_t s) {
  const unsigned B = 256;
  children_kernel<<<(unsigned)((n + B - 1) / B), B, 0, s>>>(flags, excl, n, n0, child);
  return cudaGetLastError();
}

cudaError_t build_levels(const long long* level_off, int n_levels, uint8_t* level, cudaStream_t s) {
  for (int l = 0; l < n_levels; ++l) {
    const long long cnt = level_off[l + 1] - level_off[l];
    if (cnt <= 0) continue;
    cudaError_t e = cudaMemsetAsync(level + level_off[l], l, (size_t)cnt, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

__global__ void root_coords_kernel(long long n0, int rx, int ry, uint64_t* __restrict__ coord) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n0) return;
  const uint64_t x = (uint64_t)(i % rx), y = (uint64_t)((i / rx) % ry), z = (uint64_t)(i / ((long long)rx * ry));
  coord[i] = x | (y << RT_COORD_BITS) | (z << (2 * RT_COORD_BITS));
}

__global__ void child_coords_kernel(const uint32_t* __restrict__ child, long long b, long long e,
                                    uint64_t* __restrict__ coord) {
  const long long i = b + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= e) return;
  const uint32_t c = child[i];
  if (!c) return;
  const uint64_t w = coord[i];
  const uint64_t x = 2 * (w & RT_COORD_MASK), y = 2 * ((w >> RT_COORD_BITS) & RT_COORD_MASK),
                 z = 2 * ((w >> (2 * RT_COORD_BITS)) & RT_COORD_MASK);
#pragma unroll
  for (int o = 0; o < 8; ++o)
    coord[c + o] = (x + (o & 1)) | ((y + ((o >> 1) & 1)) << RT_COORD_BITS) | ((z + ((o >> 2) & 1)) << (2 * RT_COORD_BITS));
}

cudaError_t build_coords(const uint32_t* child, long long lvl_begin, long long lvl_end, const int* root,
                         uint64_t* coord, cudaStream_t s) {
  const unsigned B = 256;
  if (lvl_begin == 0 && root) {
    root_coords_kernel<<<(unsigned)((lvl_end + B - 1) / B), B, 0, s>>>(lvl_end, root[0], root[1], coord);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const long long n = lvl_end - lvl_begin;
  if (n <= 0) return cudaSuccess;
  child_coords_kernel<<<(unsigned)((n + B - 1) / B), B, 0, s>>>(child, lvl_begin, lvl_end, coord);
  return cudaGetLastError();
}

__global__ void mean_children_kernel(const uint32_t* __restrict__ child, long long b, long long e,
                                     double* __restrict__ rho) {
  const long long i = b + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= e) return;
  const uint32_t c = child[i];
  if (!c) return;
  double s = 0.0;
#pragma unroll
  for (int o = 0; o < 8; ++o) s += rho[c + o];
  rho[i] = 0.125 * s;
}

cudaError_t build_density(const double*, const uint32_t* child, long long lvl_begin, long long lvl_end, double* rho64,
                          cudaStream_t s) {
  const long long n = lvl_end - lvl_begin;
  if (n <= 0) return cudaSuccess;
  const unsigned B = 256;
  mean_children_kernel<<<(unsigned)((n + B - 1) / B), B, 0, s>>>(child, lvl_begin, lvl_end, rho64);
  return cudaGetLastError();
}

__global__ void nodes_kernel(const double* __restrict__ rho64, const uint32_t* __restrict__ child, long long n,
                             double inv_scale, float* __restrict__ density, uint32_t* __restrict__ node) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double r = rho64[i];
  density[i] = (float)r;
  const uint32_t c = child[i];
  if (c) {
    node[i] = RT_INTERIOR | c;
  } else {
    float v = (float)(r * inv_scale);
    if (!(v > 0.0f)) v = 0.0f;
    node[i] = __float_as_uint(v);
  }
}

cudaError_t build_nodes(const double* rho64, const uint32_t* child, long long n, double inv_scale, float* density,
                        uint32_t* node, cudaStream_t s) {
  const unsigned B = 256;
  nodes_kernel<<<(unsigned)((n + B - 1) / B), B, 0, s>>>(rho64, child, n, inv_scale, density, node);
  return cudaGetLastError();
}

__device__ __forceinline__ void atomic_max_nonneg(double* p, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(p), (unsigned long long)__double_as_longlong(v));
}

__global__ void max_leaf_kernel(const double* __restrict__ rho64, const uint32_t* __restrict__ child, long long n,
                                double* out) {
  double m = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (!child[i]) m = fmax(m, rho64[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0) atomic_max_nonneg(out, m);
}

cudaError_t reduce_max_leaf(const double* rho64, const uint32_t* child, long long n, double* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  max_leaf_kernel<<<1024, 256, 0, s>>>(rho64, child, n, out);
  return cudaGetLastError();
}

__global__ void validate_kernel(const double* __restrict__ rho64, const uint32_t* __restrict__ child, long long n,
                                int* bad) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (child[i]) continue;
    const double r = rho64[i];
    if (!(r >= 0.0) || !isfinite(r)) atomicOr(bad, 1);
  }
}

cudaError_t validate_leaf_density(const double* rho64, const uint32_t* child, long long n, int* bad, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  validate_kernel<<<1024, 256, 0, s>>>(rho64, child, n, bad);
  return cudaGetLastError();
}

}  // namespace rtk
