// sr_device.cuh -- device arithmetic of the n-fold-way event loop (sm_103a).
//
// Every floating-point operation on the trajectory is an explicit IEEE
// double operation with round-to-nearest (no contraction to FMA), so that the
// event times are the exact doubles the formulas define:
//   * -log U_i of Eq. 3.4 via the artanh series ln m = 2 artanh((m-1)/(m+1));
//   * the waiting time with break points of Eqs. 3.4 and 5.2-5.6;
// Random numbers are Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), keyed
// by the seed and counted by (event index, region), which makes each region's
// random sequence the "presimulated list" of §4.
#pragma once
#include <stdint.h>

namespace sr {

// ---------------------------------------------------------------- Philox
// One Philox4x32-10 block: ten rounds; in each, two 32x32->64 products of
// words 0 and 2 with the round multipliers, the high halves xored with the
// other words and the key; the key advances by the Weyl increments.
__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1, uint32_t out[4]) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// ---------------------------------------------------------------- -log U
// U = (2k+1) 2^-53 with k a 52-bit integer.  Write u = 2k+1 = 2^e m with
// m in [sqrt(1/2), sqrt(2)); then ln U = (e - 53) ln 2 + 2 s (1 + z/3 + ... +
// z^10/21), s = (m-1)/(m+1), z = s^2, the series summed by Horner from z^10
// down.  Double-precision constants below are the correctly rounded values of
// 1/(2j+1), sqrt(2) and ln 2.
__device__ __forceinline__ double neg_log_unit(uint64_t k52) {
  const uint64_t u = 2ull * k52 + 1ull;
  int e = 63 - __clzll((long long)u);                    // u in [2^e, 2^(e+1))
  const double pow2_neg_e = __longlong_as_double((long long)(1023 - e) << 52);
  double m = __dmul_rn(__ull2double_rn(u), pow2_neg_e);  // exact, in [1, 2)
  if (m >= 1.4142135623730951) {
    m = __dmul_rn(m, 0.5);
    e += 1;
  }
  const double s = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
  const double z = __dmul_rn(s, s);
  double poly = 1.0 / 21.0;
  poly = __dadd_rn(__dmul_rn(poly, z), 1.0 / 19.0);
  poly = __dadd_rn(__dmul_rn(poly, z), 1.0 / 17.0);
  poly = __dadd_rn(__dmul_rn(poly, z), 1.0 / 15.0);
  poly = __dadd_rn(__dmul_rn(poly, z), 1.0 / 13.0);
  poly = __dadd_rn(__dmul_rn(poly, z), 1.0 / 11.0);
  poly = __dadd_rn(__dmul_rn(poly, z), 1.0 / 9.0);
  poly = __dadd_rn(__dmul_rn(poly, z), 1.0 / 7.0);
  poly = __dadd_rn(__dmul_rn(poly, z), 1.0 / 5.0);
  poly = __dadd_rn(__dmul_rn(poly, z), 1.0 / 3.0);
  poly = __dadd_rn(__dmul_rn(poly, z), 1.0);
  const double ln_m = __dmul_rn(2.0, __dmul_rn(s, poly));
  const double ln_u = __dadd_rn(__dmul_rn((double)(e - 53), 0.6931471805599453), ln_m);
  return -ln_u;
}

// The pair (U_i, V_i) of event i of a region: U feeds Eq. 3.4 (returned as
// x = -log U), V feeds the class/site choice (returned as its 52-bit integer
// kV, V = (2 kV + 1) 2^-53).
// Out of line: the event loop calls it only past the presimulated ring, and
// keeping its Philox rounds and series out of the loop body shortens the
// loop's instruction footprint (measured 2-4% faster).
__device__ __noinline__ void draw_counter(uint32_t c0, uint32_t c1, uint32_t region, uint32_t tag,
                                             uint32_t key0, uint32_t key1, double& x,
                                             unsigned long long& kv) {
  uint32_t w[4];
  philox4x32_10(c0, c1, region, tag, key0, key1, w);
  const unsigned long long ku = ((((unsigned long long)w[1]) << 32) | w[0]) >> 12;
  kv = ((((unsigned long long)w[3]) << 32) | w[2]) >> 12;
  x = neg_log_unit(ku);
}
__device__ __forceinline__ void draw_event(unsigned long long i, uint32_t region, uint32_t key0,
                                           uint32_t key1, double& x, unsigned long long& kv) {
  draw_counter((uint32_t)i, (uint32_t)(i >> 32), region, 0u, key0, key1, x, kv);
}
// The alternate step rule of §5: the j-th event of window w has its own
// numbers, counter (j, w, region, 2), never used by an earlier window.
__device__ __forceinline__ void draw_event_fresh(unsigned j, unsigned w, uint32_t region,
                                                 uint32_t key0, uint32_t key1, double& x,
                                                 unsigned long long& kv) {
  draw_counter(j, w, region, 2u, key0, key1, x, kv);
}

// ---------------------------------------------------------------- time
// Lambda as a double: the exact grid value lam * 2^-F, rounded once.
__device__ __forceinline__ double lambda_of(uint64_t lam, double scale) {
  return __dmul_rn(__ull2double_rn(lam), scale);
}

// Next event candidate (Eqs. 3.4, 5.2-5.6 in incremental form): with
// x = -log U_i and b = integral of Lambda from the previous event up to t_last,
// the remaining hazard x - b (clamped at 0) is used up at rate Lambda(t_last).
// A result that does not exceed t_last is moved to the next double above it,
// which keeps a region's event times strictly increasing.
__device__ __forceinline__ double tau_hat(double t_last, double x, double b, uint64_t lam,
                                          double scale) {
  if (lam == 0ull) return __longlong_as_double(0x7FF0000000000000ll);   // +inf
  double d = __dsub_rn(x, b);
  if (d < 0.0) d = 0.0;
  double t = __dadd_rn(t_last, __ddiv_rn(d, lambda_of(lam, scale)));
  if (!(t > t_last)) t = __longlong_as_double(__double_as_longlong(t_last) + 1ll);
  return t;
}

// A break point at t_b (a neighbour flip, §5): the hazard accrued since
// t_last at the old rate is added to b (Eqs. 5.3-5.4).
__device__ __forceinline__ double accrue(double b, double t_b, double t_last, uint64_t lam,
                                         double scale) {
  return __dadd_rn(b, __dmul_rn(lambda_of(lam, scale), __dsub_rn(t_b, t_last)));
}

}  // namespace sr
