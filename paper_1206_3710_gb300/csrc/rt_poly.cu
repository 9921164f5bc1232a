// rt_poly.cu -- polychromatic photon packages (Sect. 2.3: a package may
// stand for several wavelengths, after Jonsson 2006).
//
// The wavelength bins form consecutive groups of F bins.  A package carries
// one weight per bin of its group; its free paths and scattering directions
// are drawn for the group's reference bin r (the middle one), and each bin's
// weight carries the likelihood ratio of that path for its own bin:
//   * along a segment of length s with no scattering, e^{-(ks_j - ks_r) rho s};
//   * at a scattering, ks_j / ks_r (the event), then p_j(mu) / p_r(mu) (the
//     new direction drawn from the reference phase function).
// Absorption stays continuous: over a segment the bin-j deposit is
//   W_j ta_j (1 - e^{-x_j}) / x_j,  x_j = (ka_j + ks_j - ks_r) rho s,
// the integral of W_j(t) ka_j rho over the segment, and W_j <- W_j e^{-x_j}.
// For j = r every ratio is 1: the reference bin is the monochromatic
// package, with the random stream of the group's first bin.
//
// One thread follows one package at a time (packages from a global
// counter); peel-off marches run inline, one column density per observer
// serving every bin of the group.  Single job, point / external / beam
// sources, continuous estimator, untiled.
#include "rt_device.cuh"
#include "rt_internal.cuh"

namespace rtk {

template <typename R>
struct PolyNum;
template <>
struct PolyNum<float> {
  // (1 - e^{-x}) / x and e^{-x}, with a series near 0 (x may be negative)
  static __device__ __forceinline__ void phi_e(float x, float& phi, float& e) {
    e = expf(-x);
    if (fabsf(x) < 0.125f)
      phi = 1.0f - x * (0.5f - x * (1.0f / 6.0f - x * (1.0f / 24.0f - x * (1.0f / 120.0f - x * (1.0f / 720.0f)))));
    else
      phi = (1.0f - e) / x;
  }
  static __device__ __forceinline__ float ka(const BinDev& b) { return b.kext_f * (1.0f - b.albedo); }
  static __device__ __forceinline__ float ks(const BinDev& b) { return b.kext_f * b.albedo; }
};
template <>
struct PolyNum<double> {
  static __device__ __forceinline__ void phi_e(double x, double& phi, double& e) {
    e = exp(-x);
    phi = x != 0.0 ? -expm1(-x) / x : 1.0;
  }
  static __device__ __forceinline__ double ka(const BinDev& b) { return b.kext_d * (1.0 - b.albedo_d); }
  static __device__ __forceinline__ double ks(const BinDev& b) { return b.kext_d * b.albedo_d; }
};

// the lane's own Philox stream, with the last block cached
struct PolyStream {
  uint32_t k0, k1, c0, c1, c3, next, tag;
  uint4 blk;
  __device__ __forceinline__ uint32_t word() {
    const uint32_t j = next++;
    if (tag != (j >> 2)) {
      blk = philox4x32_10(make_uint4(c0, c1, j >> 2, c3), k0, k1);
      tag = j >> 2;
    }
    const uint32_t w = j & 3u;
    return w == 0u ? blk.x : (w == 1u ? blk.y : (w == 2u ? blk.z : blk.w));
  }
};

template <typename R, int F, bool PEEL>
__global__ void __launch_bounds__(256) poly_kernel(const JobDev* __restrict__ jobs, const ItemDev* __restrict__ items,
                                                   int n_items, unsigned long long* __restrict__ counter,
                                                   long long total) {
  double l_emit = 0.0, l_abs = 0.0, l_esc = 0.0, l_rrg = 0.0, l_rrl = 0.0, l_kill = 0.0, l_peel = 0.0;
  unsigned long long u_pk = 0, u_cross = 0, u_scat = 0, u_pcross = 0, u_kill = 0, u_pout = 0;
  int status = 0;
  const JobDev& J = jobs[0];
  GridRegs G;
  G.node = J.node;
  G.rho64 = J.rho64;
  G.rx = J.root[0];
  G.ry = J.root[1];
  G.rz = J.root[2];
  const uint32_t step_limit = (uint32_t)min(J.step_limit, (long long)0xFFFFFFFFll);
  for (;;) {
    const long long gi = (long long)atomicAdd(counter, 1ull);
    if (gi >= total) break;
    int lo = 0, hi = n_items - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (items[mid].pkt_begin <= gi) lo = mid;
      else hi = mid - 1;
    }
    const ItemDev& I = items[lo];
    const long long p = gi - I.pkt_begin;
    int blo = 0, bhi = J.n_lambda - 1;
    while (blo < bhi) {
      const int mid = (blo + bhi + 1) >> 1;
      if (I.bin_prefix[mid] <= p) blo = mid;
      else bhi = mid - 1;
    }
    const int first = blo;  // packages sit at the first bin of their group
    const int size = min(J.poly_n, J.n_lambda - first);
    const int rb = first + (size - 1) / 2;
    const unsigned long long k = (unsigned long long)(p - I.bin_prefix[first] + J.pkt_offset);
    PolyStream S;
    S.k0 = (uint32_t)J.seed ^ J.job_id;
    S.k1 = (uint32_t)(J.seed >> 32) ^ J.iter;
    S.c0 = (uint32_t)k;
    S.c1 = (uint32_t)(k >> 32);
    S.c3 = (I.src_index << 16) | (uint32_t)first;
    S.next = 0u;
    S.tag = 0xFFFFFFFFu;
    R W[F], W0[F], ka[F], ks[F];
    R W0sum = R(0);
#pragma unroll
    for (int j = 0; j < F; ++j) {
      const bool in = j < size;
      const BinDev& B = J.bins[in ? first + j : rb];
      W0[j] = in ? Num<R>::w0(I, first + j) : R(0);
      W[j] = W0[j];
      W0sum += W0[j];
      ka[j] = PolyNum<R>::ka(B);
      ks[j] = PolyNum<R>::ks(B);
    }
    const BinDev& BR = J.bins[rb];
    const R ksr = PolyNum<R>::ks(BR), gr = Num<R>::gg(BR);
    l_emit += (double)W0sum;
    u_pk += 1;
    // emission: the monochromatic package's draws and arithmetic
    Geo<R> g;
    Cursor cur;
    R dx, dy, dz;
    bool inside;
    if (I.kind == RT_SRC_POINT || I.kind == RT_SRC_BEAM) {
      if (I.kind == RT_SRC_POINT) {
        const R u1 = Num<R>::uni(S.word()), u2 = Num<R>::uni(S.word());
        iso_dir(u1, u2, dx, dy, dz);
      } else {
        dx = Num<R>::dir(I, 0);
        dy = Num<R>::dir(I, 1);
        dz = Num<R>::dir(I, 2);
      }
      inside = place_root(G, g, cur, Num<R>::pos(I, 0), Num<R>::pos(I, 1), Num<R>::pos(I, 2), dx, dy, dz);
    } else {
      const R ax = (R)G.ry * (R)G.rz, ay = (R)G.rx * (R)G.rz, az = (R)G.rx * (R)G.ry;
      const R v = Num<R>::uni(S.word()) * (R(2) * (ax + ay + az));
      int face = 5;
      R cum = R(0);
      const R ar[3] = {ax, ay, az};
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        cum += ar[f >> 1];
        if (face == 5 && v < cum) face = f;
      }
      const int a = face >> 1;
      const R u1 = Num<R>::uni(S.word()), u2 = Num<R>::uni(S.word());
      const R u3 = Num<R>::uni(S.word()), u4 = Num<R>::uni(S.word());
      const R mu = Num<R>::sqrt_(u3), st_ = Num<R>::sqrt_(fmax(R(0), R(1) - mu * mu));
      R sp, cp;
      Num<R>::sincos2pi(u4, &sp, &cp);
      const R dn = (face & 1) ? -mu : mu;
      R px, py, pz;
      if (a == 0) {
        px = (face & 1) ? (R)G.rx : R(0);
        py = u1 * (R)G.ry;
        pz = u2 * (R)G.rz;
        dx = dn; dy = st_ * cp; dz = st_ * sp;
      } else if (a == 1) {
        py = (face & 1) ? (R)G.ry : R(0);
        px = u1 * (R)G.rx;
        pz = u2 * (R)G.rz;
        dy = dn; dx = st_ * cp; dz = st_ * sp;
      } else {
        pz = (face & 1) ? (R)G.rz : R(0);
        px = u1 * (R)G.rx;
        py = u2 * (R)G.ry;
        dz = dn; dx = st_ * cp; dy = st_ * sp;
      }
      inside = place_root(G, g, cur, px, py, pz, dx, dy, dz);
    }
    R ix = inv_abs(dx), iy = inv_abs(dy), iz = inv_abs(dz);
    R tau = -Num<R>::log_(Num<R>::uni(S.word()));
    R pkt_abs = R(0);
    uint32_t ncross = 0u;
    int nscat = 0, fate = 0;
    double* absb = J.absorbed;
    const bool per_bin = J.abs_bins > 1;
    if (!inside) fate = 0;
    while (inside) {
      const uint32_t w = ld_node(G.node + cur.pending);
      const double r64 = Num<R>::load_rho64(G.rho64, cur.pending);
      if (w & RT_INTERIOR) {
        descend_step(g, cur, w, dx, dy, dz);
        continue;
      }
      settle_leaf(g, cur, w, r64);
      int a;
      const R tx = exit_dist(g, dx, dy, dz, ix, iy, iz, a);
      if (ncross >= step_limit || a < 0) {
        R s = R(0);
#pragma unroll
        for (int j = 0; j < F; ++j) s += W[j];
        l_kill += (double)s;
        u_kill += 1;
        status = 1;
        fate = 2;
#pragma unroll
        for (int j = 0; j < F; ++j) W[j] = R(0);
        break;
      }
      const R scale = g.rho * Num<R>::pow2m(g.lev);  // density x root-cell units per local unit
      const R kr = ksr * scale;
      const R tsc = kr * tx;
      const bool ev = kr > R(0) && tsc >= tau;
      const R tseg = ev ? tau / kr : tx;
      tau = ev ? R(0) : tau - tsc;
      R dsum = R(0);  // summed output: one accumulator update for the group
#pragma unroll
      for (int j = 0; j < F; ++j) {
        if (j < size) {
          const R xj = (ka[j] + ks[j] - ksr) * scale * tseg;
          R phi, e;
          PolyNum<R>::phi_e(xj, phi, e);
          const R dep = W[j] * (ka[j] * scale * tseg) * phi;
          W[j] *= e;
          if (dep > R(0)) {
            pkt_abs += dep;
            if (per_bin) {
              if (absb) red_acc(absb + (long long)(first + j) * J.n_cells + g.idx, widen(dep));
            } else {
              dsum += dep;
            }
          }
        }
      }
      if (!per_bin && absb && dsum > R(0)) red_acc(absb + g.idx, widen(dsum));
      ncross += tseg > R(0) ? 1u : 0u;
      if (ev) {
        g.fx = clamp01(g.fx + tseg * dx);
        g.fy = clamp01(g.fy + tseg * dy);
        g.fz = clamp01(g.fz + tseg * dz);
        cur.pending = g.idx;
        cur.k = g.lev;
        nscat += 1;
#pragma unroll
        for (int j = 0; j < F; ++j) W[j] = j < size ? W[j] * (ks[j] / ksr) : R(0);
        if (PEEL && J.n_obs > 0) {
          // peel-off: one column density per observer serves every bin
          for (int o = 0; o < J.n_obs; ++o) {
            const ObsDev& O = J.obs[o];
            const R s = Num<R>::pow2m(g.lev);
            const R Px = ((R)g.cx + g.fx) * s - ObsGeom<R>::c(O, 0);
            const R Py = ((R)g.cy + g.fy) * s - ObsGeom<R>::c(O, 1);
            const R Pz = ((R)g.cz + g.fz) * s - ObsGeom<R>::c(O, 2);
            const R u = (Px * ObsGeom<R>::ex(O, 0) + Py * ObsGeom<R>::ex(O, 1) + Pz * ObsGeom<R>::ex(O, 2)) *
                            ObsGeom<R>::ip(O, 0) + R(0.5) * (R)O.nx;
            const R v = (Px * ObsGeom<R>::ey(O, 0) + Py * ObsGeom<R>::ey(O, 1) + Pz * ObsGeom<R>::ey(O, 2)) *
                            ObsGeom<R>::ip(O, 1) + R(0.5) * (R)O.ny;
            const R fu = Num<R>::floor_(u), fv = Num<R>::floor_(v);
            if (!(fu >= R(0) && fv >= R(0) && fu < (R)O.nx && fv < (R)O.ny)) {
              u_pout += 1;
              continue;
            }
            const R kx = ObsGeom<R>::k(O, 0), ky = ObsGeom<R>::k(O, 1), kz = ObsGeom<R>::k(O, 2);
            Geo<R> g2 = g;
            Cursor c2;
            c2.pending = g.idx;
            c2.k = g.lev;
            const R jx = inv_abs(kx), jy = inv_abs(ky), jz = inv_abs(kz);
            R col = R(0);
            for (;;) {
              const uint32_t w2 = ld_node(G.node + c2.pending);
              const double q64 = Num<R>::load_rho64(G.rho64, c2.pending);
              if (w2 & RT_INTERIOR) {
                descend_step(g2, c2, w2, kx, ky, kz);
                continue;
              }
              settle_leaf(g2, c2, w2, q64);
              int a2;
              const R t2 = exit_dist(g2, kx, ky, kz, jx, jy, jz, a2);
              if (a2 < 0) break;
              col += g2.rho * Num<R>::pow2m(g2.lev) * t2;
              u_pcross += t2 > R(0) ? 1u : 0u;
              if (!advance(G, g2, c2, a2, t2, kx, ky, kz)) break;
            }
            const R mu_o = dx * kx + dy * ky + dz * kz;
            const long long pix0 = ((long long)fv) * O.nx + (long long)fu;
#pragma unroll
            for (int j = 0; j < F; ++j) {
              if (j < size) {
                const BinDev& B = J.bins[first + j];
                const R c = W[j] * hg_phase(Num<R>::gg(B), mu_o) * Num<R>::exp_(-Num<R>::kext(B) * col);
                if (c > R(0)) {
                  const long long im = ((long long)o * J.img_bins + (J.img_bins > 1 ? first + j : 0)) * O.ny;
                  atomicAdd(J.images + im * O.nx + pix0, widen(c));
                  l_peel += (double)c;
                }
              }
            }
          }
        }
        const R mu = hg_mu(gr, Num<R>::uni(S.word()));
        scatter_dir(dx, dy, dz, mu, Num<R>::uni(S.word()));
        ix = inv_abs(dx);
        iy = inv_abs(dy);
        iz = inv_abs(dz);
        const R pr = hg_phase(gr, mu);
        R rmax = R(0);
#pragma unroll
        for (int j = 0; j < F; ++j) {
          if (j < size) {
            W[j] *= hg_phase(Num<R>::gg(J.bins[first + j]), mu) / pr;
            const R q = W[j] / W0[j];
            rmax = q > rmax ? q : rmax;
          }
        }
        const R wmin = Num<R>::rr_wmin(J);
        if (wmin > R(0) && rmax < wmin) {
          const R ur = Num<R>::uni(S.word());
          const R rp = Num<R>::rr_p(J);
          if (ur < rp) {
            R s = R(0);
#pragma unroll
            for (int j = 0; j < F; ++j) {
              s += W[j];
              W[j] = R(0);
            }
            l_rrl += (double)s;
            fate = 1;
            break;
          }
#pragma unroll
          for (int j = 0; j < F; ++j) {
            const R Wn = W[j] / (R(1) - rp);
            l_rrg += (double)(Wn - W[j]);
            W[j] = Wn;
          }
        }
        tau = -Num<R>::log_(Num<R>::uni(S.word()));
      } else if (!advance(G, g, cur, a, tx, dx, dy, dz)) {
        R s = R(0);
#pragma unroll
        for (int j = 0; j < F; ++j) s += W[j];
        l_esc += (double)s;
        fate = 0;
        break;
      }
    }
    if (!inside) {
      R s = R(0);
#pragma unroll
      for (int j = 0; j < F; ++j) s += W[j];
      l_esc += (double)s;
    }
    l_abs += (double)pkt_abs;
    u_cross += ncross;
    u_scat += (unsigned long long)nscat;
    if (J.packet_log) {
      double* r = J.packet_log + (I.log_offset + p) * 10;
      R s = R(0);
#pragma unroll
      for (int j = 0; j < F; ++j) s += W[j];
      const double hs = (double)Num<R>::pow2m(g.lev) * J.h0;
      r[0] = fate == 0 ? (double)s : 0.0;
      r[1] = (double)nscat;
      r[2] = (double)ncross;
      r[3] = (double)fate;
      r[4] = ((double)(int)g.cx + (double)g.fx) * hs;
      r[5] = ((double)(int)g.cy + (double)g.fy) * hs;
      r[6] = ((double)(int)g.cz + (double)g.fz) * hs;
      r[7] = (double)dx; r[8] = (double)dy; r[9] = (double)dz;
    }
  }
  // ledger: warp sums, one atomic per warp and quantity
  const double dv[7] = {l_emit, l_abs, l_esc, l_rrg, l_rrl, l_kill, l_peel};
  const unsigned long long uv[6] = {u_pk, u_cross, u_scat, u_pcross, u_kill, u_pout};
  LedgerDev* L = J.ledger;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    const double v = warp_sum(dv[i]);
    if (lane == 0 && v != 0.0) atomicAdd(&L->emitted + i, v);
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    unsigned long long v = uv[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if (lane == 0 && v) atomicAdd(&L->n_packets + i, v);
  }
  if (__any_sync(0xFFFFFFFFu, status) && lane == 0) atomicOr(&L->status, 1);
}

template <typename R, int F>
static cudaError_t launch_poly_f(bool peel, const JobDev* jobs, const ItemDev* items, int n_items,
                                 unsigned long long* counter, long long total, int blocks, cudaStream_t s) {
  if (peel)
    poly_kernel<R, F, true><<<blocks, 256, 0, s>>>(jobs, items, n_items, counter, total);
  else
    poly_kernel<R, F, false><<<blocks, 256, 0, s>>>(jobs, items, n_items, counter, total);
  return cudaGetLastError();
}

template <typename R>
static cudaError_t launch_poly_r(int group, bool peel, const JobDev* jobs, const ItemDev* items, int n_items,
                                 unsigned long long* counter, long long total, int blocks, cudaStream_t s) {
  if (group <= 2) return launch_poly_f<R, 2>(peel, jobs, items, n_items, counter, total, blocks, s);
  if (group <= 4) return launch_poly_f<R, 4>(peel, jobs, items, n_items, counter, total, blocks, s);
  return launch_poly_f<R, 8>(peel, jobs, items, n_items, counter, total, blocks, s);
}

cudaError_t launch_poly(int precision, int group, bool peel, const JobDev* jobs, const ItemDev* items, int n_items,
                        unsigned long long* counter, long long total, int sm_count, cudaStream_t s) {
  if (group < 2 || group > 8) return cudaErrorInvalidValue;
  const int blocks = sm_count * 4;
  return precision == 64 ? launch_poly_r<double>(group, peel, jobs, items, n_items, counter, total, blocks, s)
                         : launch_poly_r<float>(group, peel, jobs, items, n_items, counter, total, blocks, s);
}

}  // namespace rtk
