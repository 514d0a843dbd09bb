// Philox4x32-10 counter-based generator and the Gaussian start vectors of
// the null-vector setup (section "Setup procedure": inverse iteration starts
// from a random vector).  Counter-based, so every site draws its own numbers
// without state.
#pragma once
#include "common.cuh"

namespace mg {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): round
// (c0,c1,c2,c3) -> (hi(M1 c2)^c1^k0, lo(M1 c2), hi(M0 c0)^c3^k1, lo(M0 c0)),
// key bumped by (0x9E3779B9, 0xBB67AE85) between the 10 rounds.
__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; r++) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Value of component `dof` of site `lex` in start vector k of level `level`:
// counter (lex, dof, k, level), key (seed lo, seed hi); Box-Muller with
// u = (w + 1/2) 2^-32 gives Re, Im ~ N(0, 1/2).
__device__ __forceinline__ cx<double> philox_gauss(uint64_t seed, int level, int k, int lex, int dof) {
  uint4 w = philox10(make_uint4((unsigned)lex, (unsigned)dof, (unsigned)k, (unsigned)level),
                     make_uint2((unsigned)(seed & 0xffffffffu), (unsigned)(seed >> 32)));
  const double u0 = ((double)w.x + 0.5) * 2.3283064365386963e-10;
  const double u1 = ((double)w.y + 0.5) * 2.3283064365386963e-10;
  const double rad = sqrt(-log(u0));
  double sn, cs;
  sincospi(2.0 * u1, &sn, &cs);
  return mkc(rad * cs, rad * sn);
}

}  // namespace mg
