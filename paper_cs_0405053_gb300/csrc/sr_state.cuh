// sr_state.cuh -- device-side state of libsr: launch parameters, per-lattice
// descriptors and counters, the bounded grid barrier, a region's view in shared
// memory, and the small exact-arithmetic helpers of the region pass.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sr.h"
#include "sr_device.cuh"
#include "sr_softfloat.cuh"

namespace sr {

enum : unsigned { ST_CAPACITY = 1u, ST_NOT_CONVERGED = 2u, ST_TIMEOUT = 4u };

// Device-side status and counters.  The first block of fields is cleared by
// the host before every launch.
struct DevStats {
  unsigned long long qhead, qtail;   // task queue (asynchronous schedule): claimed / published
  unsigned long long cwork;     // regions with a commit task outstanding (asynchronous); the
                                // top bit stops new commits after an error
  unsigned work;                // next unclaimed work-list entry of the iteration (dynamic)
  unsigned wl_count[2];         // entries of the two work lists (dynamic, by iteration parity)
  unsigned status;
  unsigned bar_count;
  unsigned bar_gen;
  unsigned active;              // lattices with windows left in this launch
  // persistent across launches
  unsigned long long region_passes, region_skips;   // region iterations run / skipped
  unsigned long long run_cycles, run_cycles_max;    // cycles region slots spent on their regions
  unsigned long long slots;                         // region slots that reported
};

constexpr int kWinRing = 4096;

// Task items of the asynchronous schedule: bit 63 valid, bit 62 kind,
// bits 42-61 lattice, bits 20-41 chunk, bits 0-19 the tag of its ticket.
constexpr unsigned long long kTaskValid = 1ull << 63;
constexpr unsigned long long kTaskTag = (1ull << 20) - 1ull;
constexpr int kTaskMaxLattices = 1 << 20;
constexpr long long kTaskMaxChunks = 1ll << 22;

// One lattice of a batch, with its own region shape; its regions are numbered
// off .. off + NR - 1 in the global region index.
struct RepDesc {
  int L, NX, NY, NR;            // side, regions across, regions down, regions
  int W, H;                     // region shape (at most the launch's W, H)
  int F;                        // rate grid 2^-F of this shape (63 - bitlen(W H))
  int off;                      // global index of its first region
  int spans_x, spans_y;         // a region covers the whole periodic extent
  uint32_t key0, key1;          // seed
  int nwin;                     // windows to run in the current launch
  int init_mode;                // SR_INIT_* of sr_reset
  unsigned w0;                  // windows committed before the current launch
  double t0, Tw;                // committed time at the launch, window length
  double scale;                 // 2^-F
  unsigned long long P[10];     // p_k on the 2^-F grid
  unsigned long long Rp[10];    // floor((2^64 - 1) / P[k]) (0 when P[k] = 0)
};

// Per-lattice counters.
struct RepStats {
  unsigned long long committed, generated, breaks, windows, iterations;
  unsigned long long sum_f;     // sum over committed windows of f (§6)
  unsigned last_iters, max_iters_seen, max_f, max_win_events;
  unsigned windows_done;        // windows committed in the current launch
};

// Per-lattice progress of the asynchronous schedule (host-initialised).
struct LatState {
  unsigned pend;                // regions of the current task set not finished
  unsigned chg;                 // a region's lists changed in the current iteration
  unsigned ovf;                 // a region overflowed its history capacity
  unsigned n;                   // iteration of the current passes (1-based, per window)
  unsigned w;                   // windows committed in this launch
  unsigned pad;
  double ts;                    // start of the current window
};

struct KParams {
  int W, H, NR;                 // the largest region shape of any lattice (the layout of the
                                // per-region arrays and of shared memory), regions of all lattices
  int nrep;                     // lattices
  const RepDesc* reps;
  const uint32_t* rrep;         // [NR] lattice of each region
  RepStats* rs;                 // [nrep]
  uint32_t* rflags;             // [3][nrep] "some region's lists changed", one row per
                                // iteration slot; cleared by the host before a launch
  uint8_t* rcidx;               // [NR] committed copy of each region's state
  uint32_t* rn;                 // [NR] iteration of the region's current window
  uint32_t* rwin;               // [NR] windows the region committed in this launch
  double* rts;                  // [NR] start of the region's current window
  uint8_t* rfill;               // [NR] ring top-up pending
  uint32_t* rows;               // [2][H][NR]   spin rows, bit x = site x of the row
  uint32_t* halo;               // [4][NR]      N, S, W, E halo words at t_c
  unsigned long long* ci;       // [2][NR]      index of the pending event
  double* cx;                   // [2][NR]      -log U of the pending event
  unsigned long long* ckv;      // [2][NR]      V bits of the pending event
  double* cb;                   // [2][NR]      integral of Lambda since the last event
  double* ct;                   // [2][NR]      time up to which cb is taken
  double* cim;                  // [2][NR]      integral over time of the region's spin sum
  // path statistics of the score function (score mode): committed events by
  // the class of the flipped site before the flip, and the integral of N_k dt
  unsigned long long* sc;       // [2][10][NR]
  double* si;                   // [2][10][NR]
  double* cib;                  // [2][NR]      integral over time of the region's owned bonds
  double* ht;                   // [2][4][cap][NR] boundary history: times
  uint8_t* hp;                  // [2][4][cap][NR] boundary history: positions along the edge
  uint32_t* hl;                 // [2][4][NR]   boundary history lengths
  uint8_t* chg;                 // [2][NR]      lists of the iteration of that parity changed
  int cap;
  double* trt;                  // [NR][tcap]   committed event times (optional)
  uint32_t* trs;                // [NR][tcap]   committed event sites
  int tcap;
  double* rx;                   // [K][NR]      presimulated -log U of event i at slot i mod K
  unsigned long long* rkv;      // [K][NR]      presimulated V bits
  unsigned long long* rhi;      // [NR]         ring holds events [committed index, rhi)
  int K;                        // ring length (power of two)
  uint32_t* log;                // [NR][CB][kRecHead + H] checkpoints of consumed break points
  uint32_t* loghdr;             // [NR][4] breaks consumed, records kept, window-start sums
  int CB;                       // checkpoint records per region (0 = no incremental replay)
  int rl;                       // region slots per block (the other threads only help fill)
  int lanes;                    // lane mappings: region lanes in each warp
  DevStats* st;
  uint32_t* win_iters;          // [2][kWinRing] iterations g and f of each window of lattice 0
  uint32_t* curf;               // [2][nrep] f of the running window, by window parity
  int fresh;                    // the alternate step rule of §5
  int score;                    // accumulate the path statistics sc / si
  uint32_t* wl;                 // [2][NR] regions that need a pass (dynamic schedule)
  LatState* ls;                 // [nrep] (asynchronous schedule)
  unsigned long long* q;        // [qcap] task queue (asynchronous schedule)
  unsigned long long qcap;
  int max_iters;
  long long timeout_cycles;
  int skip_block;
};

// The lattice of region r.
struct Lat {
  const unsigned long long* P;
  const unsigned long long* Rp;
  int L, NX, NY, off, loc, rep;
  int W, H, F;                  // its region shape and rate grid
  double scale;
  bool spans_x, spans_y;
  uint32_t key0, key1;
};

__device__ __forceinline__ Lat lat_of(const KParams& p, int r) {
  Lat t;
  const int b = (int)__ldg(&p.rrep[r]);
  const RepDesc* d = p.reps + b;
  t.rep = b;
  t.L = d->L;
  t.NX = d->NX;
  t.NY = d->NY;
  t.off = d->off;
  t.loc = r - d->off;
  t.W = d->W;
  t.H = d->H;
  t.F = d->F;
  t.scale = d->scale;
  t.spans_x = d->spans_x != 0;
  t.spans_y = d->spans_y != 0;
  t.key0 = d->key0;
  t.key1 = d->key1;
  t.P = d->P;
  t.Rp = d->Rp;
  return t;
}

// Words of a checkpoint record before the spin rows (see run_region).
constexpr int kRecHead = 24;

// ---------------------------------------------------------------- barrier
// Grid-wide "synchronize" with a bounded wait (SR_TIMEOUT instead of a hang).
__device__ __noinline__ bool grid_barrier(DevStats* st, long long timeout) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* gen = &st->bar_gen;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(&st->bar_count, 1u) + 1u;
    if (arrived == gridDim.x) {
      atomicExch(&st->bar_count, 0u);
      __threadfence();
      atomicAdd(&st->bar_gen, 1u);
    } else {
      const long long start = clock64();
      while (*gen == g) {
        if (clock64() - start > timeout) {
          ok = 0;
          atomicOr(&st->status, ST_TIMEOUT);
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    if (*(volatile unsigned*)&st->status & ST_TIMEOUT) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---------------------------------------------------------------- region view
// A lane's region: rows in shared memory (stride = threads per block), halos
// in registers.  Bit x of row y is the spin (1 = up) of site (x, y).
struct Region {
  uint32_t* rows;              // rows[y * stride]
  uint32_t* C;                 // C[(k * hq + y/4) * stride]: byte y%4 = sites of class k in row y
  unsigned long long* PT;      // PT[k * pts] = P_k, PT[(10 + k) * pts] = its reciprocal
  // score mode: per class the window's event count SX[k * stride] and the
  // window's occupancy sum as a 128-bit fixed-point number,
  // SX[(10 + 2k) * stride] (low word) and SX[(11 + 2k) * stride] (high word)
  unsigned long long* SX;
  int cur_rep;                 // lattice whose table PT holds (-1: none)
  int pts;                     // stride of PT: the slot stride (a table per region slot) or 1
                               // (one table per warp, whose lanes all run one lattice)
  int hq;                      // count words per class, (H + 3) / 4
  int stride;
  int W, H;
  bool spans_x, spans_y;       // the region covers the whole periodic extent
  uint32_t wmask;
  uint32_t hN, hS, hW, hE;

  __device__ __forceinline__ uint32_t row(int y) const { return rows[y * stride]; }
  // The region shape of the lattice being run (the layout is the launch's largest).
  __device__ __forceinline__ void set_shape(int w, int h) {
    W = w;
    H = h;
    hq = (h + 3) / 4;
    wmask = (w == 32) ? 0xFFFFFFFFu : ((1u << w) - 1u);
  }
  __device__ __forceinline__ unsigned long long P(int k) const { return PT[k * pts]; }
  __device__ __forceinline__ unsigned long long Rp(int k) const { return PT[(10 + k) * pts]; }

  // Row y for y in [-2, H + 1]: periodic inside a region spanning the lattice,
  // else the halo row for y = -1 and y = H (0 beyond, never used).
  __device__ __forceinline__ uint32_t row_at(int y) const {
    if (y >= 0 && y < H) return row(y);
    if (spans_y) return row(y < 0 ? y + H : y - H);
    return y == -1 ? hN : (y == H ? hS : 0u);
  }

  // Neighbour words of row y: bit x = spin of the up/down/left/right neighbour.
  __device__ __forceinline__ void side_words(int y, uint32_t r, uint32_t& lf, uint32_t& rt) const {
    const uint32_t lbit = spans_x ? (r >> (W - 1)) & 1u : (hW >> y) & 1u;
    const uint32_t rbit = spans_x ? (r & 1u) : (hE >> y) & 1u;
    lf = ((r << 1) | lbit) & wmask;
    rt = (r >> 1) | (rbit << (W - 1));
  }
  __device__ __forceinline__ void nbr_words(int y, uint32_t r, uint32_t& up, uint32_t& dn,
                                            uint32_t& lf, uint32_t& rt) const {
    up = row_at(y - 1);
    dn = row_at(y + 1);
    side_words(y, r, lf, rt);
  }

  // Class 5*s + n_up of site (x, y) from its row rm and the rows above (ru)
  // and below (rd); left and right from rm or the side halos.
  __device__ __forceinline__ int class_in(int x, int y, uint32_t ru, uint32_t rm, uint32_t rd) const {
    const int s = (rm >> x) & 1;
    const int up = (ru >> x) & 1, dn = (rd >> x) & 1;
    const int lf = (x > 0) ? (rm >> (x - 1)) & 1 : (spans_x ? (rm >> (W - 1)) & 1 : (hW >> y) & 1);
    const int rt = (x < W - 1) ? (rm >> (x + 1)) & 1 : (spans_x ? rm & 1 : (hE >> y) & 1);
    return 5 * s + up + dn + lf + rt;
  }

  // Score mode: a site leaves class `from` and joins `to` at fixed-point time
  // tf.  The occupancy integral of class k over the window is
  // N_k(end) t_end - N_k(start) t_start + sum(times of departures from k)
  // - sum(times of arrivals in k); the sums are kept here.
  __device__ __forceinline__ void occ_add(int k, unsigned long long tf, bool minus) const {
    unsigned long long& lo = SX[(10 + 2 * k) * stride];
    unsigned long long& hi = SX[(11 + 2 * k) * stride];
    if (minus) {
      hi -= (lo < tf) ? 1ull : 0ull;
      lo -= tf;
    } else {
      const unsigned long long n = lo + tf;
      hi += (n < lo) ? 1ull : 0ull;
      lo = n;
    }
  }
  __device__ __forceinline__ void occ_move(int from, int to, unsigned long long tf) const {
    occ_add(from, tf, false);
    occ_add(to, tf, true);
  }

  // A site of row y moves from class `from` to class `to` (per-row counts).
  __device__ __forceinline__ void c_move(int from, int to, int y) const {
    const uint32_t one = 1u << (8 * (y & 3));
    atomicAdd(&C[(from * hq + (y >> 2)) * stride], 0u - one);
    atomicAdd(&C[(to * hq + (y >> 2)) * stride], one);
  }
};

// The ten class counts N_k in two registers: 12-bit fields, classes 0-4 in lo
// and 5-9 in hi (a region has at most 1024 sites).
struct Counts {
  unsigned long long lo = 0ull, hi = 0ull;
  __device__ __forceinline__ unsigned get(int k) const {
    return (unsigned)(((k < 5 ? lo : hi) >> (12 * (k < 5 ? k : k - 5))) & 0xFFFull);
  }
  __device__ __forceinline__ unsigned get_dyn(int k) const { return get(k); }
  __device__ __forceinline__ void add(int k, unsigned v) {
    const unsigned long long d = (unsigned long long)v << (12 * (k < 5 ? k : k - 5));
    if (k < 5) lo += d; else hi += d;
  }
  __device__ __forceinline__ void move(int from, int to) {
    const unsigned long long df = 1ull << (12 * (from < 5 ? from : from - 5));
    const unsigned long long dt = 1ull << (12 * (to < 5 ? to : to - 5));
    if (from < 5) lo -= df; else hi -= df;
    if (to < 5) lo += dt; else hi += dt;
  }
};

// A 4-byte asynchronous copy from global to shared memory (cp.async): the
// copies of a loop are in flight together.
__device__ __forceinline__ void cp_async4(uint32_t* dst_shared, const uint32_t* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::
               "r"((unsigned)__cvta_generic_to_shared(dst_shared)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Per-position sum of four bits as a 3-bit number (b0, b1, b2).
__device__ __forceinline__ void add4(uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t& s0,
                                     uint32_t& s1, uint32_t& s2) {
  const uint32_t x0 = a ^ b, c0 = a & b;
  const uint32_t x1 = c ^ d, c1 = c & d;
  s0 = x0 ^ x1;
  const uint32_t c2 = x0 & x1;
  s1 = c0 ^ c1 ^ c2;
  s2 = (c0 & c1) | (c0 & c2) | (c1 & c2);
}

// Position of the j-th (0-based) set bit of m, j < popc(m): binary search on
// the population counts of the low halves.
__device__ __forceinline__ int nth_set_bit(uint32_t m, unsigned j) {
  int pos = 0;
#pragma unroll
  for (int w = 16; w > 0; w >>= 1) {
    const uint32_t low = m & ((1u << w) - 1u);
    const unsigned c = __popc(low);
    if (j >= c) {
      j -= c;
      m >>= w;
      pos += w;
    } else {
      m = low;
    }
  }
  return pos;
}

__device__ __forceinline__ uint32_t eq_count(uint32_t s0, uint32_t s1, uint32_t s2, int n) {
  return ((n & 1) ? s0 : ~s0) & ((n & 2) ? s1 : ~s1) & ((n & 4) ? s2 : ~s2);
}

// tau of Eq. 3.4 / 5.6 in integer-emulated doubles (same bits as tau_hat).
__device__ __forceinline__ double tau_soft(double t_last, double x, double b, unsigned long long lam,
                                           int F) {
  if (lam == 0ull) return __longlong_as_double(0x7FF0000000000000ll);
  double d = sf::sub_pos(x, b);
  if (__double_as_longlong(d) < 0ll) d = 0.0;      // sign bit: the remaining hazard is used up
  const double t = sf::add_pos(t_last, sf::div_pos(d, sf::u64_scaled(lam, F)));
  if (__double_as_longlong(t) <= __double_as_longlong(t_last))
    return __longlong_as_double(__double_as_longlong(t_last) + 1ll);
  return t;
}

// 128-bit signed accumulator of fixed-point times (observables).
struct Acc128 {
  unsigned long long lo;
  long long hi;
  __device__ __forceinline__ void add(long long k, unsigned long long v) {   // += k * v, |k| <= 2
    unsigned long long a = v;
    if (k == 2 || k == -2) a = v << 1;
    const long long ahi = (k == 2 || k == -2) ? (long long)(v >> 63) : 0;
    if (k > 0) {
      const unsigned long long n = lo + a;
      hi += ahi + (n < lo ? 1 : 0);
      lo = n;
    } else if (k < 0) {
      const unsigned long long n = lo - a;
      hi -= ahi + (lo < a ? 1 : 0);
      lo = n;
    }
  }
  __device__ __forceinline__ double value(int frac) const {   // as a double times 2^-frac
    return __dadd_rn(__dmul_rn((double)hi, __longlong_as_double((long long)(1023 + 64 - frac) << 52)),
                     __dmul_rn(__ull2double_rn(lo), __longlong_as_double((long long)(1023 - frac) << 52)));
  }
};

// t >= 0 as an integer multiple of 2^-frac (truncated), t * 2^frac < 2^63.
__device__ __forceinline__ unsigned long long to_fixed(double t, int frac) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(t);
  if (b == 0ull) return 0ull;
  const int e = (int)(b >> 52) - 1075 + frac;       // t = m 2^(ebits - 1075)
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  if (e >= 0) return m << e;
  if (e <= -64) return 0ull;
  return m >> (-e);
}

// K t_end - S as a 128-bit fixed-point number (the window term of a time integral).
__device__ __forceinline__ Acc128 window_moment(int k, double t_end, int frac, const Acc128& sum) {
  Acc128 out;
  const unsigned long long tend_fix = to_fixed(t_end, frac);
  const unsigned long long ak = (unsigned long long)(k < 0 ? -k : k);
  const unsigned long long plo = ak * tend_fix, phi = __umul64hi(ak, tend_fix);
  if (k >= 0) {
    out.lo = plo;
    out.hi = (long long)phi;
  } else {
    out.lo = 0ull - plo;
    out.hi = -(long long)phi - (plo != 0ull ? 1 : 0);
  }
  const unsigned long long n = out.lo - sum.lo;
  out.hi = out.hi - sum.hi - (out.lo < sum.lo ? 1 : 0);
  out.lo = n;
  return out;
}

// floor(D / P_k) for the position within class k (Eqs. 3.7-3.8): a multiply by
// the reciprocal floor((2^64-1)/P_k) undershoots by at most one.
__device__ __forceinline__ unsigned long long class_pos(unsigned long long D, unsigned long long Pk,
                                                        unsigned long long Rk) {
  unsigned long long j = __umul64hi(D, Rk);
  if ((j + 1ull) * Pk <= D) ++j;
  return j;
}

// Score mode: an event of class cv and the class moves of its in-region
// neighbours (class -1: no such neighbour).  Out of line: it keeps the event
// loop's instruction footprint small when score mode is off (measured 3%).
__device__ __noinline__ void score_event(const Region& g, int cv, int s_old, int dnb,
                                        unsigned long long tfix, int cE, int cW, int cS, int cN) {
  g.SX[cv * g.stride] += 1ull;
  g.occ_move(cv, cv + (s_old ? -5 : 5), tfix);
  if (cE >= 0) g.occ_move(cE, cE + dnb, tfix);
  if (cW >= 0) g.occ_move(cW, cW + dnb, tfix);
  if (cS >= 0) g.occ_move(cS, cS + dnb, tfix);
  if (cN >= 0) g.occ_move(cN, cN + dnb, tfix);
}

}  // namespace sr
