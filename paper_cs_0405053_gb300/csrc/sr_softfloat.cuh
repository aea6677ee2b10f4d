// sr_softfloat.cuh -- IEEE 754 binary64 arithmetic (round to nearest, ties to
// even) in integer instructions, for the time chain of the event loop.
//
// Why: on this part an FP64 warp instruction occupies the FP64 pipe for about
// 20 SM cycles whatever the number of active lanes, and an FP64 division takes
// about 8.6 such slots and ~600 cycles of latency.  A warp that simulates one
// region evaluates the time formula of Eqs. 3.4 / 5.2-5.6 on one value at a
// time, so the hardware FP64 path would make that pipe the bottleneck; the
// integer pipes are far wider.
//
// Exactness: IEEE 754 defines every result as the exact value rounded once, so
// a correct integer implementation returns the same bits as the hardware.  The
// fast paths cover finite non-negative operands whose result is a normal
// number; zeros are handled inline and everything else (subnormal operands or
// results, infinities, NaN, overflow) goes to the hardware instruction.  Tests
// compare every operation bit for bit with the hardware.
//
// Methods (textbook, e.g. Muller et al., Handbook of Floating-Point
// Arithmetic): significands carried with three extra bits (guard, round,
// sticky) and rounded once; an inexact alignment shift of the subtrahend is
// folded in as "truncated value plus one, with the sticky bit set" so that the
// difference keeps its position relative to every rounding boundary; division
// by a 64-bit reciprocal seeded from the FP32 reciprocal, refined by two
// Newton-Raphson steps in fixed point, then an exact remainder correction.
#pragma once
#include <stdint.h>

namespace sr {
namespace sf {

typedef unsigned long long u64;

__device__ __forceinline__ u64 bits(double x) { return (u64)__double_as_longlong(x); }
__device__ __forceinline__ double from_bits(u64 b) { return __longlong_as_double((long long)b); }
__device__ __forceinline__ int ef(u64 b) { return (int)((b >> 52) & 0x7FF); }          // biased exponent
__device__ __forceinline__ u64 sig(u64 b) { return (b & 0xFFFFFFFFFFFFFull) | (1ull << 52); }

// m in [2^55, 2^56) holds 53 significand bits and 3 extra bits; the value is
// m * 2^(e - 1078).  Round to nearest even and pack (positive).  The caller
// guarantees 1 <= e and that e stays <= 2046 after a carry.
__device__ __forceinline__ u64 pack_round(u64 m, int e) {
  const u64 low = m & 7ull;
  m >>= 3;
  if (low > 4ull || (low == 4ull && (m & 1ull))) m += 1ull;
  if (m >> 53) {
    m >>= 1;
    e += 1;
  }
  return ((u64)e << 52) + (m & 0xFFFFFFFFFFFFFull);
}

// m >> s, and whether a nonzero bit was shifted out.
__device__ __forceinline__ u64 shr_lost(u64 m, int s, u64& lost) {
  if (s <= 0) {
    lost = 0ull;
    return m;
  }
  if (s >= 64) {
    lost = m != 0ull ? 1ull : 0ull;
    return 0ull;
  }
  lost = (m & ((1ull << s) - 1ull)) != 0ull ? 1ull : 0ull;
  return m >> s;
}

// a + b, a and b finite and >= 0.
__device__ __forceinline__ double add_pos(double a, double b) {
  u64 ba = bits(a), bb = bits(b);
  if (ba < bb) {
    const u64 t = ba;
    ba = bb;
    bb = t;
  }
  if (bb == 0ull) return from_bits(ba);
  const int ea = ef(ba), eb = ef(bb);
  if (eb == 0 || ea >= 2046) return __dadd_rn(a, b);
  u64 lost;
  const u64 mb = shr_lost(sig(bb) << 3, ea - eb, lost);
  u64 m = ((sig(ba) << 3) + mb) | lost;        // < 2^57
  int e = ea;
  if (m >> 56) {
    m = (m >> 1) | (m & 1ull);
    e += 1;
    if (e >= 2046) return __dadd_rn(a, b);
  }
  return from_bits(pack_round(m, e));
}

// a - b, a and b finite and >= 0 (the result may be negative).
__device__ __forceinline__ double sub_pos(double a, double b) {
  u64 ba = bits(a), bb = bits(b);
  if (bb == 0ull) return a;
  if (ba == bb) return 0.0;                     // x - x = +0 in round to nearest
  if (ba == 0ull) return from_bits(bb | 0x8000000000000000ull);
  u64 neg = 0ull;
  if (ba < bb) {
    const u64 t = ba;
    ba = bb;
    bb = t;
    neg = 0x8000000000000000ull;
  }
  const int ea = ef(ba), eb = ef(bb);
  if (eb == 0 || ea >= 2047) return __dsub_rn(a, b);
  const int d = ea - eb;
  u64 m;
  int e;
  if (d <= 1) {
    // exact: the significands aligned with one extra bit
    m = (sig(ba) << 1) - (sig(bb) << (1 - d));  // > 0, < 2^54
    const int sh = __clzll((long long)m) - 8;   // bring the top bit to position 55
    m <<= sh;
    e = ea + 2 - sh;
  } else {
    // eight extra bits; an inexact shift contributes "truncated + 1" and the
    // sticky bit, which keeps the difference on the right side of every
    // rounding boundary (those lie on multiples of 2^5 here)
    u64 lost;
    const u64 mb = shr_lost(sig(bb) << 8, d, lost);
    m = ((sig(ba) << 8) - mb - lost) | lost;    // in (2^59, 2^61)
    e = ea;
    if (!(m >> 60)) {
      m <<= 1;
      e -= 1;
    }
    m = (m >> 5) | ((m & 31ull) != 0ull ? 1ull : 0ull);
  }
  if (e < 1) return __dsub_rn(a, b);
  return from_bits(pack_round(m, e) | neg);
}

__device__ __forceinline__ void mul128(u64 a, u64 b, u64& hi, u64& lo) {
  lo = a * b;
  hi = __umul64hi(a, b);
}

// a * b, a and b finite and >= 0.
__device__ __forceinline__ double mul_pos(double a, double b) {
  const u64 ba = bits(a), bb = bits(b);
  if (ba == 0ull || bb == 0ull) return 0.0;
  const int ea = ef(ba), eb = ef(bb);
  if (ea == 0 || eb == 0 || ea == 2047 || eb == 2047) return __dmul_rn(a, b);
  u64 hi, lo;
  mul128(sig(ba) << 11, sig(bb) << 10, hi, lo);   // product in [2^125, 2^127)
  int e = ea + eb - 1023;
  u64 m;
  if (hi >> 62) {
    m = (hi >> 7) | (((hi & 127ull) | lo) != 0ull ? 1ull : 0ull);
    e += 1;
  } else {
    m = (hi >> 6) | (((hi & 63ull) | lo) != 0ull ? 1ull : 0ull);
  }
  if (e < 1 || e >= 2046) return __dmul_rn(a, b);
  return from_bits(pack_round(m, e));
}

// a / b, a finite and >= 0, b finite and > 0.
__device__ __forceinline__ double div_pos(double a, double b) {
  const u64 ba = bits(a), bb = bits(b);
  if (ba == 0ull) return 0.0;
  const int ea = ef(ba), eb = ef(bb);
  if (ea == 0 || eb == 0 || ea == 2047 || eb == 2047) return __ddiv_rn(a, b);
  const u64 A = sig(ba), B = sig(bb);            // [2^52, 2^53)
  // Q = floor(A 2^s / B) lies in [2^55, 2^56) for s = 55 (A >= B) or 56 (A < B)
  int e = ea - eb + 1023;
  int s = 55;
  if (A < B) {
    s = 56;
    e -= 1;
  }
  if (e < 1 || e >= 2046) return __ddiv_rn(a, b);
  const u64 n_hi = A >> (64 - s), n_lo = A << s;   // N = A 2^s < 2^109

  // reciprocal V ~ 2^127 / D of D = B 2^11 in [2^63, 2^64)
  const u64 D = B << 11;
  const float df = __uint2float_rn((unsigned)(D >> 40));          // exact, [2^23, 2^24)
  const float rf = __fdividef(1.0f, df);                          // ~2^-22 relative
  // rf * 2^55 in [2^31, 2^32]: a 32-bit conversion (saturating), then << 32
  u64 V = (u64)__float2uint_rz(rf * 36028797018963968.0f) << 32;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    // E = 2^127 - D V (signed); V += V E / 2^127
    u64 ph, pl;
    mul128(D, V, ph, pl);
    const u64 e_lo = 0ull - pl;
    const long long e_hi = (long long)(0x8000000000000000ull - ph - (pl != 0ull ? 1ull : 0ull));
    (void)e_lo;
    const bool negative = e_hi < 0;
    const u64 mag = negative ? (u64)(-e_hi) : (u64)e_hi;       // |E| >> 64, within 1
    u64 ch, cl;
    mul128(V, mag, ch, cl);
    const u64 corr = (ch << 1) | (cl >> 63);                     // V |E| / 2^127
    V = negative ? V - corr : V + corr;
  }
  // quotient estimate floor(N V / 2^116), then the exact remainder fixes it
  u64 t_hi, t_lo, x_hi, x_lo;
  mul128(n_lo, V, t_hi, t_lo);
  mul128(n_hi, V, x_hi, x_lo);
  (void)t_lo;
  const u64 mid = x_lo + t_hi;
  const u64 top = x_hi + (mid < x_lo ? 1ull : 0ull);
  u64 Q = (top << 12) | (mid >> 52);
  u64 p_hi, p_lo;
  mul128(Q, B, p_hi, p_lo);
  u64 r_lo = n_lo - p_lo;
  long long r_hi = (long long)(n_hi - p_hi - (n_lo < p_lo ? 1ull : 0ull));
#pragma unroll
  for (int fix = 0; fix < 3; ++fix) {
    if (r_hi < 0) {                     // Q too large
      Q -= 1ull;
      const u64 nl = r_lo + B;
      r_hi += (nl < r_lo) ? 1 : 0;
      r_lo = nl;
    } else if (r_hi > 0 || r_lo >= B) {  // Q too small
      Q += 1ull;
      r_hi -= (r_lo < B) ? 1 : 0;
      r_lo = r_lo - B;
    }
  }
  Q |= (r_lo != 0ull) ? 1ull : 0ull;   // the remainder is the sticky bit
  return from_bits(pack_round(Q, e));
}

// v * 2^-F rounded to double, v >= 1 (the total rate on its fixed-point grid);
// the same value as converting v to double and scaling by the power of two.
__device__ __forceinline__ double u64_scaled(u64 v, int F) {
  const int top = 63 - __clzll((long long)v);
  const int e = top - F + 1023;
  if (e < 1 || e >= 2046)
    return __dmul_rn(__ull2double_rn(v), __longlong_as_double((long long)(1023 - F) << 52));
  u64 m;
  if (top <= 55) {
    m = v << (55 - top);
  } else {
    u64 lost;
    m = shr_lost(v, top - 55, lost) | lost;
  }
  return from_bits(pack_round(m, e));
}

}  // namespace sf
}  // namespace sr
