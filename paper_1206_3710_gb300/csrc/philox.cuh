// philox.cuh -- Philox4x32-10 counter-based generator for device code.
//
// Written from the published definition (Salmon, Moraes, Dror & Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of a
// substitution-permutation network on four 32-bit words.  Each round forms
// the 64-bit products of words 0 and 2 with two fixed multipliers; the new
// block is (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0)).
// The two key words are advanced by two Weyl constants between rounds.
#pragma once
#include <stdint.h>

namespace rtk {

__device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint32_t k0, uint32_t k1) {
  constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(M0, x.x), lo0 = M0 * x.x;
    const uint32_t hi1 = __umulhi(M1, x.z), lo1 = M1 * x.z;
    x = make_uint4(hi1 ^ x.y ^ k0, lo1, hi0 ^ x.w ^ k1, lo0);
    k0 += W0;
    k1 += W1;
  }
  return x;
}

// Sequential draws of one package stream: draw j = word (j & 3) of the block
// with counter (pkt_lo, pkt_hi, j >> 2, stream).
struct PhiloxStream {
  uint32_t k0, k1, c0, c1, c3;
  uint32_t next;
  uint32_t blk;
  uint4 cache;

  __device__ __forceinline__ void init(unsigned long long seed, uint32_t job, uint32_t iter,
                                       uint32_t stream, unsigned long long pkt) {
    k0 = (uint32_t)seed ^ job;
    k1 = (uint32_t)(seed >> 32) ^ iter;
    c0 = (uint32_t)pkt;
    c1 = (uint32_t)(pkt >> 32);
    c3 = stream;
    next = 0;
    blk = 0xFFFFFFFFu;
  }
  __device__ __forceinline__ uint32_t u32() {
    const uint32_t b = next >> 2;
    if (b != blk) {
      cache = philox4x32_10(make_uint4(c0, c1, b, c3), k0, k1);
      blk = b;
    }
    const uint32_t w = next & 3u;
    ++next;
    uint32_t v = cache.x;
    v = (w == 1u) ? cache.y : v;
    v = (w == 2u) ? cache.z : v;
    v = (w == 3u) ? cache.w : v;
    return v;
  }
};

}  // namespace rtk
