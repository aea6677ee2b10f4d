// sr_lib.cu -- libsr: synchronous relaxation of the continuous-time n-fold-way
// Ising simulation on one GPU (sm_103a).  C ABI in include/sr.h.
//
// Mapping (Lubachevsky & Weiss, §4-§5):
//   * A region G_i is one lane ("PE").  Its spins live bit-packed in shared
//     memory, one 32-bit word per row; its ten class counts N_k (§3) in
//     shared memory; the total rate Lambda = sum_k N_k p_k (Eq. 3.3) as an
//     exact integer on the 2^-F grid.  One lane per region keeps every FP64
//     instruction 32 regions wide, the only way to use the FP64 pipe well on
//     this part: a warp-wide FP64 instruction costs the same whatever the
//     number of active lanes.
//   * "Synchronize" (§4 boxed procedure) is a grid-wide barrier of a persistent
//     cooperative kernel; "all PEs detect no difference" is a grid flag set by
//     atomics.  Every wait is bounded and ends in SR_TIMEOUT, never a hang.
//   * Boundary histories (§5, "the single layer of atoms that border its
//     region") are per-edge lists of (time, position) in HBM, double-buffered by
//     iteration parity: iteration n reads the neighbours' lists of iteration
//     n-1 (§4: "uses that history generated in the last iteration") and
//     compares its own new lists with its own previous ones.
#include <cuda_runtime.h>

#include <climits>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>

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

// One lattice of a batch.  Every lattice of a launch shares the region shape;
// its regions are numbered off .. off + NR - 1 in the global region index.
struct RepDesc {
  int L, NX, NY, NR;            // side, regions across, regions down, regions
  int off;                      // global index of its first region
  int spans_x, spans_y;         // a region covers the whole periodic extent
  uint32_t key0, key1;          // seed
  int nwin;                     // windows to run in the current launch
  int init_mode;                // SR_INIT_* of sr_reset
  unsigned w0;                  // windows committed before the current launch
  double t0, Tw;                // committed time at the launch, window length
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
  int W, H, NR;                 // region shape, regions of all lattices
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
  double scale;                 // 2^-F
  int F;
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
  unsigned long long* PT;      // PT[k * stride] = P_k, PT[(10 + k) * stride] = its reciprocal
  // score mode: per class the window's event count SX[k * stride] and the
  // window's occupancy sum as a 128-bit fixed-point number,
  // SX[(10 + 2k) * stride] (low word) and SX[(11 + 2k) * stride] (high word)
  unsigned long long* SX;
  int cur_rep;                 // lattice whose table PT holds (-1: none)
  int hq;                      // count words per class, (H + 3) / 4
  int stride;
  int W, H;
  bool spans_x, spans_y;       // the region covers the whole periodic extent
  uint32_t wmask;
  uint32_t hN, hS, hW, hE;

  __device__ __forceinline__ uint32_t row(int y) const { return rows[y * stride]; }
  __device__ __forceinline__ unsigned long long P(int k) const { return PT[k * stride]; }
  __device__ __forceinline__ unsigned long long Rp(int k) const { return PT[(10 + k) * stride]; }

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

// ---------------------------------------------------------------- region pass
struct Acc {
  unsigned events, breaks, passes, skips;   // per slot and iteration: well below 2^32
  unsigned fmax, emax;
  bool changed, overflow;
};

// One iteration of one region over [t_s, t_end): statement (a) of the §4
// procedure, specialised in §5.  Starts from the committed state (copy cidx),
// merges the neighbours' previous-iteration boundary lists as break points,
// writes the tentative end state to copy cidx ^ 1 and its own boundary lists to
// parity wp, comparing them with its lists of the previous iteration.
// SOFT = 1: the waiting-time chain in integer-emulated doubles; 0: FP64
// instructions.  Both round every operation once (IEEE), so the bits agree.
template <int SOFT>
__device__ __forceinline__ double tau_any(double t_last, double x, double b, unsigned long long lam,
                                          const KParams& p) {
  return SOFT ? tau_soft(t_last, x, b, lam, p.F) : tau_hat(t_last, x, b, lam, p.scale);
}
template <int SOFT>
__device__ __forceinline__ double accrue_any(double b, double tb, double tl, unsigned long long lam,
                                             const KParams& p) {
  return SOFT ? sf::add_pos(b, sf::mul_pos(sf::u64_scaled(lam, p.F), sf::sub_pos(tb, tl)))
              : accrue(b, tb, tl, lam, p.scale);
}

template <int SOFT>
__device__ void run_region(const KParams& p, const Lat& lt, int r, int n_iter, unsigned cidx,
                           double t_s, double t_end, unsigned wg, Region& g, Acc& acc) {
  const int W = p.W, H = p.H, NR = p.NR;
  const int wp = n_iter & 1;
  const int rp = wp ^ 1;
  const int rx = lt.loc % lt.NX, ry = lt.loc / lt.NX;
  const size_t nr = (size_t)NR;
  const size_t cap = (size_t)p.cap;
  g.spans_x = lt.spans_x;
  g.spans_y = lt.spans_y;

  // ---- neighbours (global region indices): d = 0 N, 1 S, 2 W, 3 E.  Every
  // small per-direction array below is indexed by compile-time constants only
  // (unrolled loops, selects), so it stays in registers.
  const int q[4] = {lt.off + ((ry + lt.NY - 1) % lt.NY) * lt.NX + rx,
                    lt.off + ((ry + 1) % lt.NY) * lt.NX + rx,
                    lt.off + ry * lt.NX + (rx + lt.NX - 1) % lt.NX,
                    lt.off + ry * lt.NX + (rx + 1) % lt.NX};
  const bool has[4] = {!g.spans_y, !g.spans_y, !g.spans_x, !g.spans_x};

  // ---- a region whose neighbours' lists did not change in the last iteration
  // sees the same input as then, so its output is the same: keep the
  // tentative state and carry the lists over instead of replaying the window
  auto carry_over = [&]() {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (!has[e]) continue;
      const unsigned n = __ldcg(&p.hl[((size_t)rp * 4 + e) * nr + r]);
      for (unsigned j = 0; j < n; ++j) {
        const size_t src = (((size_t)rp * 4 + e) * cap + j) * nr + r;
        const size_t dst = (((size_t)wp * 4 + e) * cap + j) * nr + r;
        p.ht[dst] = __ldcg(&p.ht[src]);
        p.hp[dst] = __ldcg(&p.hp[src]);
      }
      p.hl[((size_t)wp * 4 + e) * nr + r] = n;
    }
    p.chg[(size_t)wp * nr + r] = 0;
    acc.skips += 1;
  };
  if (n_iter >= 2) {
    bool dirty = false;
#pragma unroll
    for (int d = 0; d < 4; ++d)
      if (has[d] && __ldcg(&p.chg[(size_t)rp * nr + q[d]])) dirty = true;
    if (!dirty) {
      carry_over();
      return;
    }
  }

  // ---- incoming boundary lists: the neighbours' lists of the previous iteration;
  // my N halo is fed by the N neighbour's S list, etc.
  // per direction: the time of the next entry, and a cursor word holding the
  // list length (high 16 bits) and the index of the next entry (low 16 bits);
  // the four positions share one word, a byte each
  const double INF = __longlong_as_double(0x7FF0000000000000ll);
  unsigned cur[4], npos = 0u;
  double nt[4];
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    const int ein = d ^ 1;                 // the neighbour's edge facing me
    // iteration 1: the canonical assumption, no neighbour flips (§5)
    const unsigned len = (has[d] && n_iter >= 2) ? __ldcg(&p.hl[((size_t)rp * 4 + ein) * nr + q[d]]) : 0u;
    cur[d] = len << 16;
    nt[d] = INF;
    if (len > 0) {
      const size_t a = (((size_t)rp * 4 + ein) * cap) * nr + q[d];
      nt[d] = __ldcg(&p.ht[a]);
      npos |= (unsigned)__ldcg(&p.hp[a]) << (8 * d);
    }
  }
  // earliest pending break point; ties go to the lower direction
  auto next_break = [&](long long& tbb, int& db, unsigned& pos) {
    tbb = __double_as_longlong(nt[0]);
    db = 0;
#pragma unroll
    for (int d = 1; d < 4; ++d) {
      const long long v = __double_as_longlong(nt[d]);
      if (v < tbb) {
        tbb = v;
        db = d;
      }
    }
    pos = (npos >> (8 * db)) & 0xFFu;
  };
  auto advance = [&](int db) {
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      if (d == db) {
        const unsigned c = cur[d] + 1u;
        cur[d] = c;
        nt[d] = INF;
        if ((c & 0xFFFFu) < (c >> 16)) {
          const size_t a = (((size_t)rp * 4 + (d ^ 1)) * cap + (c & 0xFFFFu)) * nr + q[d];
          nt[d] = __ldcg(&p.ht[a]);
          npos = (npos & ~(0xFFu << (8 * d))) | ((unsigned)__ldcg(&p.hp[a]) << (8 * d));
        }
      }
    }
  };

  // ---- incremental replay: the state of this region after its m-th consumed
  // break point depends only on the committed state and on its first m inputs.
  // Walk the new inputs against the inputs logged by the last pass; resume from
  // the checkpoint before the first difference.
  const size_t rwords = (size_t)kRecHead + H;
  uint32_t* rec0 = p.log + (size_t)r * p.CB * rwords;
  uint32_t* hdr = p.loghdr + (size_t)r * 4;     // breaks consumed, records kept, M0, bonds0
  unsigned m = 0;
  if (n_iter >= 2 && p.CB > 0) {
    const unsigned nb_total = hdr[0], nb_log = hdr[1];
    long long tbb;
    int db;
    unsigned pos;
    while (m < nb_log) {
      next_break(tbb, db, pos);
      const uint32_t* rec = rec0 + (size_t)m * rwords;
      const long long rt = (long long)(((unsigned long long)rec[1] << 32) | rec[0]);
      if (tbb != rt || rec[2] != (pos | ((unsigned)db << 8))) break;
      advance(db);
      ++m;
    }
    next_break(tbb, db, pos);
    if (m == nb_total && m == nb_log && tbb == 0x7FF0000000000000ll) {
      carry_over();          // every input is the one the last pass consumed
      return;
    }
  }
  const bool resume = m > 0;
  acc.passes += 1;

  // the lattice's rate table and reciprocals, staged in this slot's shared
  // memory when the slot moves to another lattice
  if (g.cur_rep != lt.rep) {
#pragma unroll
    for (int k = 0; k < 10; ++k) {
      g.PT[k * g.stride] = lt.P[k];
      g.PT[(10 + k) * g.stride] = lt.Rp[k];
    }
    g.cur_rep = lt.rep;
  }

  unsigned long long i;
  double x, b, tl;
  unsigned long long kv;
  unsigned olen[4] = {0u, 0u, 0u, 0u};
  unsigned bevents = 0;
  int ksig = 0, kbeta = 0;
  Acc128 ssig = {0ull, 0}, sbeta = {0ull, 0};
  if (resume) {
    // ---- state after the m-th consumed break of the last pass
    const uint32_t* rec = rec0 + (size_t)(m - 1) * rwords;
    tl = __longlong_as_double((long long)(((unsigned long long)rec[1] << 32) | rec[0]));
    i = ((unsigned long long)rec[4] << 32) | rec[3];
    b = __longlong_as_double((long long)(((unsigned long long)rec[6] << 32) | rec[5]));
    olen[0] = rec[7] & 0xFFFFu;
    olen[1] = rec[7] >> 16;
    olen[2] = rec[8] & 0xFFFFu;
    olen[3] = rec[8] >> 16;
    bevents = rec[9];
    ksig = (int)rec[10];
    kbeta = (int)rec[11];
    ssig.lo = ((unsigned long long)rec[13] << 32) | rec[12];
    ssig.hi = (long long)(((unsigned long long)rec[15] << 32) | rec[14]);
    sbeta.lo = ((unsigned long long)rec[17] << 32) | rec[16];
    sbeta.hi = (long long)(((unsigned long long)rec[19] << 32) | rec[18]);
    g.hN = rec[20];
    g.hS = rec[21];
    g.hW = rec[22];
    g.hE = rec[23];
    for (int y = 0; y < H; ++y) g.rows[y * g.stride] = rec[kRecHead + y];
  } else {
    // ---- committed state
    const uint32_t* rows_c = p.rows + (size_t)cidx * H * nr;
    for (int y = 0; y < H; ++y) g.rows[y * g.stride] = rows_c[(size_t)y * nr + r];
    g.hN = p.halo[0 * nr + r];
    g.hS = p.halo[1 * nr + r];
    g.hW = p.halo[2 * nr + r];
    g.hE = p.halo[3 * nr + r];
    i = p.ci[cidx * nr + r];        // first event of the window
    // the carry of §5 "Subsequent steps", or (alternate rule) a clock that
    // restarts at the window start with no hazard accrued
    b = p.fresh ? 0.0 : p.cb[cidx * nr + r];
    tl = p.fresh ? t_s : p.ct[cidx * nr + r];
  }
  // presimulated pairs (U, V) of the coming events (§4: the random numbers
  // as a list drawn before use); the pair of event i+1 is loaded one event ahead
  const unsigned long long hi = p.rhi[r];
  const unsigned kmask = (unsigned)p.K - 1u;     // K is a power of two <= 4096
  // events past the ring are drawn here (alternate rule: numbered from the window start)
  auto draw_at = [&](unsigned long long ii, double& xx, unsigned long long& kk) {
    if (p.fresh)
      draw_event_fresh((unsigned)(ii - p.ci[cidx * nr + r]), wg, (uint32_t)lt.loc, lt.key0,
                       lt.key1, xx, kk);
    else
      draw_event(ii, (uint32_t)lt.loc, lt.key0, lt.key1, xx, kk);
  };
  if (!resume && !p.fresh) {
    x = p.cx[cidx * nr + r];
    kv = p.ckv[cidx * nr + r];
  } else if (i < hi) {
    const size_t a = (size_t)((unsigned)i & kmask) * nr + r;
    x = p.rx[a];
    kv = p.rkv[a];
  } else {
    draw_at(i, x, kv);
  }
  double px = 0.0;
  unsigned long long pkv = 0ull;
  bool pvalid = (i + 1ull) < hi;
  if (pvalid) {
    const size_t a = (size_t)((unsigned)(i + 1ull) & kmask) * nr + r;
    px = p.rx[a];
    pkv = p.rkv[a];
  }

  // ---- class counts N_k (packed in registers, Counts), the per-row class
  // counts in shared memory, Lambda, and the region's spin / owned-bond sums
  // (recounted from the rows: measured cheaper than storing them with the
  // state and the checkpoints)
  Counts N;
  int mag0 = 0, bond0 = 0;
  uint32_t cw[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) cw[k] = 0;
  for (int y = 0; y < H; ++y) {
    const uint32_t rw = g.row(y);
    uint32_t up, dn, lf, rt, s0, s1, s2;
    g.nbr_words(y, rw, up, dn, lf, rt);
    add4(up, dn, lf, rt, s0, s1, s2);
    const int sh = 8 * (y & 3);
#pragma unroll
    for (int n = 0; n < 5; ++n) {
      const uint32_t e = eq_count(s0, s1, s2, n) & g.wmask;
      const unsigned cu = __popc(e & rw), cd = __popc(e) - cu;
      cw[5 + n] |= cu << sh;
      cw[n] |= cd << sh;
    }
    if ((y & 3) == 3 || y == H - 1) {
#pragma unroll
      for (int k = 0; k < 10; ++k) {
        g.C[(k * g.hq + (y >> 2)) * g.stride] = cw[k];
        N.add(k, __vsadu4(cw[k], 0u));     // the four rows' counts of class k
        cw[k] = 0;
      }
    }
    mag0 += 2 * __popc(rw) - W;
    bond0 += (W - 2 * __popc((rw ^ rt) & g.wmask)) + (W - 2 * __popc((rw ^ dn) & g.wmask));
  }
  unsigned long long lam = 0;
#pragma unroll
  for (int k = 0; k < 10; ++k) lam += (unsigned long long)N.get(k) * g.P(k);
  if (resume) {                      // window-start sums, kept since the first pass
    mag0 = (int)hdr[2];
    bond0 = (int)hdr[3];
  } else if (p.CB > 0) {
    hdr[2] = (uint32_t)mag0;
    hdr[3] = (uint32_t)bond0;
  }

  // own lists: on a resumed pass the entries before the checkpoint are the
  // same as last time.  The previous lengths (for the comparison of §4,
  // statement (c)) are read where they are needed.
  auto plen = [&](int e) -> unsigned {
    return n_iter >= 2 ? __ldcg(&p.hl[((size_t)rp * 4 + e) * nr + r]) : 0u;
  };
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if (resume && has[e]) {
      for (unsigned j = 0; j < olen[e]; ++j) {
        const size_t src = (((size_t)rp * 4 + e) * cap + j) * nr + r;
        const size_t dst = (((size_t)wp * 4 + e) * cap + j) * nr + r;
        p.ht[dst] = __ldcg(&p.ht[src]);
        p.hp[dst] = __ldcg(&p.hp[src]);
      }
    }
  }

  bool changed = false, overflow = false;
  unsigned events = 0, brk = 0;
  unsigned nrec = m, nbt = m;           // checkpoint records kept, breaks consumed
  // window integrals of the observables in fixed point (times as multiples of 2^-frac)
  const int frac = 62 - (int)((((unsigned long long)__double_as_longlong(t_end)) >> 52) - 1022);
  const long long tend_b = __double_as_longlong(t_end);
  if (p.score) {
    // the window's occupancy sums start at -N_k(t_s) t_s, its event counts at 0
    const unsigned long long tf0 = to_fixed(t_s, frac);
#pragma unroll
    for (int k = 0; k < 10; ++k) {
      const unsigned long long nk = N.get(k);
      const unsigned long long plo = nk * tf0, phi = __umul64hi(nk, tf0);
      g.SX[k * g.stride] = 0ull;
      g.SX[(10 + 2 * k) * g.stride] = 0ull - plo;
      g.SX[(11 + 2 * k) * g.stride] = 0ull - phi - (plo != 0ull ? 1ull : 0ull);
    }
  }

  // times are >= 0, so their bit patterns order like their values
  double tau = tau_any<SOFT>(tl, x, b, lam, p);
  for (;;) {
    long long tbb;
    int db;
    unsigned bpos;
    next_break(tbb, db, bpos);
    const double tb = __longlong_as_double(tbb);
    const long long taub = __double_as_longlong(tau);

    if (taub <= tbb) {
      // ---- own event at tau, unless it falls past the window (§5: tau_m < t_c + T_max)
      if (!(taub < tend_b)) break;
      // class k* of Eqs. 3.5-3.6, exactly: P = V*Lambda*2^(53+F) as a 128-bit
      // integer (q53, rem); class k is chosen when P <= A(k) * 2^53 (the scan
      // stops there: measured faster than a full branch-free scan)
      const unsigned long long mV = 2ull * kv + 1ull;
      const unsigned long long plo = mV * lam, phi = __umul64hi(mV, lam);
      const unsigned long long q53 = (phi << 11) | (plo >> 53);
      const bool exact = (plo & ((1ull << 53) - 1ull)) == 0ull;
      unsigned long long A = 0, Aprev = 0;
      int ks = 9;
      for (int k = 0; k < 10; ++k) {
        Aprev = A;
        A += (unsigned long long)N.get_dyn(k) * g.P(k);
        if (q53 < A || (q53 == A && exact)) {
          ks = k;
          break;
        }
      }
      // position within the class, Eqs. 3.7-3.8: floor((V*Lambda - A(k*-1)) / p_k*)
      const unsigned Nks = N.get_dyn(ks);
      unsigned long long j = class_pos(q53 - Aprev, g.P(ks), g.Rp(ks));
      if (j >= Nks) j = Nks - 1;
      // the j-th class-k* site in row-major order (linear order of §3, Phase 3):
      // the row from the per-row counts of class k*, then the site in that row
      unsigned jj = (unsigned)j;
      int fy = 0;
      {
        const uint32_t* Ck = g.C + (ks * g.hq) * g.stride;
        unsigned base = 0, jr = 0;
        uint32_t wsel = 0;
        int qsel = -1;
        for (int qd = 0; qd < g.hq; ++qd) {
          const uint32_t w = Ck[qd * g.stride];
          const unsigned s4 = __vsadu4(w, 0u);        // sites of class k* in these 4 rows
          if (jj < base + s4) {
            qsel = qd;
            wsel = w;
            jr = jj - base;
            break;
          }
          base += s4;
        }
        const unsigned c0 = wsel & 0xFFu, c1 = (wsel >> 8) & 0xFFu, c2 = (wsel >> 16) & 0xFFu;
        const unsigned u1 = jr >= c0, u2 = jr >= c0 + c1, u3 = jr >= c0 + c1 + c2;
        jj = jr - (u1 ? c0 : 0u) - (u2 ? c1 : 0u) - (u3 ? c2 : 0u);
        fy = 4 * qsel + (int)(u1 + u2 + u3);
      }
      // ---- the rows around fy (periodic, or the halo rows at the region edge)
      const uint32_t rM = g.row(fy);
      const uint32_t rU = g.row_at(fy - 1), rD = g.row_at(fy + 1);
      const int sp = ks >= 5;
      const int nn = ks - 5 * sp;
      int fx;
      {
        uint32_t lf, rt, s0, s1, s2;
        g.side_words(fy, rM, lf, rt);
        add4(rU, rD, lf, rt, s0, s1, s2);
        fx = nth_set_bit(eq_count(s0, s1, s2, nn) & (sp ? rM : ~rM) & g.wmask, jj);
      }
      // ---- flip (fx, fy); classes of the site and its in-region neighbours
      // (taken before the flip); E, W, S, N neighbours
      const bool vE = fx < W - 1 || g.spans_x, vW = fx > 0 || g.spans_x;
      const bool vS = fy < H - 1 || g.spans_y, vN = fy > 0 || g.spans_y;
      const int xE = (fx + 1 == W) ? 0 : fx + 1, xW = (fx == 0) ? W - 1 : fx - 1;
      const int yS = (fy + 1 == H) ? 0 : fy + 1, yN = (fy == 0) ? H - 1 : fy - 1;
      const int cv = g.class_in(fx, fy, rU, rM, rD);
      const int cE = g.class_in(xE, fy, rU, rM, rD);
      const int cW = g.class_in(xW, fy, rU, rM, rD);
      const int cS = g.class_in(fx, yS, rM, rD, g.row_at(fy + 2));
      const int cN = g.class_in(fx, yN, g.row_at(fy - 2), rU, rM);
      const int s_old = cv >= 5;
      const int nup = cv - 5 * s_old;
      const int dnb = s_old ? -1 : 1;          // change of the neighbours' up count
      g.rows[fy * g.stride] = rM ^ (1u << fx);
      // Lambda's change, in wrap-around unsigned arithmetic (exact at the end)
      unsigned long long dl = g.P(cv + (s_old ? -5 : 5)) - g.P(cv);
      N.move(cv, cv + (s_old ? -5 : 5));
      g.c_move(cv, cv + (s_old ? -5 : 5), fy);
      if (vE) {
        dl += g.P(cE + dnb) - g.P(cE);
        N.move(cE, cE + dnb);
        g.c_move(cE, cE + dnb, fy);
      }
      if (vW) {
        dl += g.P(cW + dnb) - g.P(cW);
        N.move(cW, cW + dnb);
        g.c_move(cW, cW + dnb, fy);
      }
      if (vS) {
        dl += g.P(cS + dnb) - g.P(cS);
        N.move(cS, cS + dnb);
        g.c_move(cS, cS + dnb, yS);
      }
      if (vN) {
        dl += g.P(cN + dnb) - g.P(cN);
        N.move(cN, cN + dnb);
        g.c_move(cN, cN + dnb, yN);
      }
      lam += dl;

      // observables: dM = 2 sig, dBonds = 4 beta (Eq. 2.1 book-keeping)
      const int sig = s_old ? -1 : 1;
      const int beta = sig * (nup - 2);
      {
        const unsigned long long tfix = to_fixed(tau, frac);
        if (p.score)                   // score statistics of the event and its class moves
          score_event(g, cv, s_old, dnb, tfix, vE ? cE : -1, vW ? cW : -1, vS ? cS : -1,
                      vN ? cN : -1);
        ksig += sig;
        ssig.add(sig, tfix);
        kbeta += beta;
        sbeta.add(beta, tfix);
      }

      // ---- boundary history (§5: the single layer of border atoms)
      bool boundary = false;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        bool on;
        unsigned pos;
        if (e == 0) { on = !g.spans_y && fy == 0; pos = fx; }
        else if (e == 1) { on = !g.spans_y && fy == H - 1; pos = fx; }
        else if (e == 2) { on = !g.spans_x && fx == 0; pos = fy; }
        else { on = !g.spans_x && fx == W - 1; pos = fy; }
        if (on) {
          boundary = true;
          const unsigned n = olen[e];
          if (n >= (unsigned)p.cap) {
            overflow = true;
          } else {
            const size_t a = (((size_t)wp * 4 + e) * cap + n) * nr + r;
            p.ht[a] = tau;
            p.hp[a] = (uint8_t)pos;
            if (n < plen(e)) {
              const size_t pa = (((size_t)rp * 4 + e) * cap + n) * nr + r;
              if (__double_as_longlong(__ldcg(&p.ht[pa])) != __double_as_longlong(tau) ||
                  __ldcg(&p.hp[pa]) != (uint8_t)pos)
                changed = true;
            } else {
              changed = true;
            }
            olen[e] = n + 1;
          }
        }
      }
      if (boundary) ++bevents;
      if (p.tcap > 0 && i < (unsigned long long)p.tcap) {
        p.trt[(size_t)r * p.tcap + i] = tau;
        p.trs[(size_t)r * p.tcap + i] =
            ((uint32_t)(ry * H) + fy) * (uint32_t)lt.L + (uint32_t)(rx * W) + fx;
      }
      ++events;
      if (overflow) break;
      // ---- next event: clock restarts at tau with U_{i+1} (§5, "Subsequent iterations")
      tl = tau;
      b = 0.0;
      ++i;
      if (pvalid) {
        x = px;
        kv = pkv;
      } else {
        draw_at(i, x, kv);
      }
      pvalid = (i + 1ull) < hi;
      if (pvalid) {
        const size_t a = (size_t)((unsigned)(i + 1ull) & kmask) * nr + r;
        px = p.rx[a];
        pkv = p.rkv[a];
      }
    } else {
      // ---- break point: a neighbour flip at tb < tau (§5, Eqs. 5.2-5.6)
      b = accrue_any<SOFT>(b, tb, tl, lam, p);
      tl = tb;
      const unsigned pos = bpos;
      int ux, uy, up_now;
      if (db == 0) { g.hN ^= 1u << pos; up_now = (g.hN >> pos) & 1; ux = pos; uy = 0; }
      else if (db == 1) { g.hS ^= 1u << pos; up_now = (g.hS >> pos) & 1; ux = pos; uy = H - 1; }
      else if (db == 2) { g.hW ^= 1u << pos; up_now = (g.hW >> pos) & 1; ux = 0; uy = pos; }
      else { g.hE ^= 1u << pos; up_now = (g.hE >> pos) & 1; ux = W - 1; uy = pos; }
      // class of the adjacent site after the change; before it, its up count
      // differed by one
      const int cu_new = g.class_in(ux, uy, g.row_at(uy - 1), g.row(uy), g.row_at(uy + 1));
      const int cu_old = cu_new + (up_now ? -1 : 1);
      lam += g.P(cu_new) - g.P(cu_old);
      N.move(cu_old, cu_new);
      g.c_move(cu_old, cu_new, uy);
      if (p.score) g.occ_move(cu_old, cu_new, to_fixed(tb, frac));
      // checkpoint after this break point, for the next pass's replay
      if (nrec < (unsigned)p.CB) {
        uint32_t* rec = rec0 + (size_t)nrec * rwords;
        rec[0] = (uint32_t)tbb;
        rec[1] = (uint32_t)((unsigned long long)tbb >> 32);
        rec[2] = pos | ((unsigned)db << 8);
        rec[3] = (uint32_t)i;
        rec[4] = (uint32_t)(i >> 32);
        const unsigned long long bb = (unsigned long long)__double_as_longlong(b);
        rec[5] = (uint32_t)bb;
        rec[6] = (uint32_t)(bb >> 32);
        rec[7] = olen[0] | (olen[1] << 16);
        rec[8] = olen[2] | (olen[3] << 16);
        rec[9] = bevents;
        rec[10] = (uint32_t)ksig;
        rec[11] = (uint32_t)kbeta;
        rec[12] = (uint32_t)ssig.lo;
        rec[13] = (uint32_t)(ssig.lo >> 32);
        rec[14] = (uint32_t)ssig.hi;
        rec[15] = (uint32_t)((unsigned long long)ssig.hi >> 32);
        rec[16] = (uint32_t)sbeta.lo;
        rec[17] = (uint32_t)(sbeta.lo >> 32);
        rec[18] = (uint32_t)sbeta.hi;
        rec[19] = (uint32_t)((unsigned long long)sbeta.hi >> 32);
        rec[20] = g.hN;
        rec[21] = g.hS;
        rec[22] = g.hW;
        rec[23] = g.hE;
        for (int y = 0; y < H; ++y) rec[kRecHead + y] = g.row(y);
        ++nrec;
      }
      ++nbt;
      advance(db);
      ++brk;
    }
    tau = tau_any<SOFT>(tl, x, b, lam, p);
  }

#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if (has[e]) {
      if (olen[e] != plen(e)) changed = true;
      p.hl[((size_t)wp * 4 + e) * nr + r] = olen[e];
    }
  }
  p.chg[(size_t)wp * nr + r] = (changed || overflow) ? 1 : 0;
  if (p.CB > 0) {
    hdr[0] = nbt;
    hdr[1] = nrec;
  }
  // ---- tentative end state
  const unsigned tc = cidx ^ 1u;
  uint32_t* rows_t = p.rows + (size_t)tc * H * nr;
  for (int y = 0; y < H; ++y) rows_t[(size_t)y * nr + r] = g.row(y);
  p.ci[tc * nr + r] = i;
  p.cx[tc * nr + r] = x;
  p.ckv[tc * nr + r] = kv;
  p.cb[tc * nr + r] = b;
  p.ct[tc * nr + r] = tl;
  {
    const double span = __dsub_rn(t_end, t_s);
    const Acc128 um = window_moment(ksig, t_end, frac, ssig);
    const Acc128 ub = window_moment(kbeta, t_end, frac, sbeta);
    const double im = __dadd_rn(__dmul_rn((double)mag0, span), __dmul_rn(2.0, um.value(frac)));
    const double ib = __dadd_rn(__dmul_rn((double)bond0, span), __dmul_rn(4.0, ub.value(frac)));
    p.cim[tc * nr + r] = __dadd_rn(p.cim[cidx * nr + r], im);
    p.cib[tc * nr + r] = __dadd_rn(p.cib[cidx * nr + r], ib);
  }
  if (p.score) {
    // close the window's occupancy sums with N_k(t_end) t_end; add to the totals
    const unsigned long long tfe = to_fixed(t_end, frac);
    for (int k = 0; k < 10; ++k) {
      const unsigned long long nk = N.get_dyn(k);
      const unsigned long long plo = nk * tfe, phi = __umul64hi(nk, tfe);
      const unsigned long long lo = g.SX[(10 + 2 * k) * g.stride];
      const unsigned long long hi = g.SX[(11 + 2 * k) * g.stride];
      Acc128 a;
      a.lo = lo + plo;
      a.hi = (long long)(hi + phi + (a.lo < lo ? 1ull : 0ull));
      const size_t o = ((size_t)k) * nr + r;
      p.si[(size_t)tc * 10 * nr + o] = __dadd_rn(p.si[(size_t)cidx * 10 * nr + o], a.value(frac));
      p.sc[(size_t)tc * 10 * nr + o] = p.sc[(size_t)cidx * 10 * nr + o] + g.SX[k * g.stride];
    }
  }

  acc.events += events;
  acc.breaks += brk;
  {
    const unsigned long long i_win = p.ci[cidx * nr + r];   // first event of the window
    if ((unsigned)(i - i_win) > acc.emax) acc.emax = (unsigned)(i - i_win);
  }
  if (bevents > acc.fmax) acc.fmax = bevents;
  acc.changed |= changed || overflow;
  acc.overflow |= overflow;
}

// ---------------------------------------------------------------- warp per region
// The same region pass with one warp per region: lane y holds row y in a
// register, the ten class counts sit in lanes 0..9, the four incoming-list
// cursors in lanes 0..3.  Class choice (Eqs. 3.5-3.6) is a warp prefix scan of
// N_k p_k and a ballot; site choice (Eqs. 3.7-3.8) a prefix scan of the rows'
// class-k* counts and a ballot; the waiting time (Eqs. 3.4, 5.2-5.6) runs in
// integer-emulated IEEE doubles (sr_softfloat.cuh), identical bits to the
// lane version.  Control flow is uniform across the warp.

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ unsigned long long shfl_u64(unsigned long long v, int src) {
  const unsigned lo = __shfl_sync(kFull, (unsigned)v, src);
  const unsigned hi = __shfl_sync(kFull, (unsigned)(v >> 32), src);
  return ((unsigned long long)hi << 32) | lo;
}
__device__ __forceinline__ unsigned long long shfl_up_u64(unsigned long long v, int d) {
  const unsigned lo = __shfl_up_sync(kFull, (unsigned)v, d);
  const unsigned hi = __shfl_up_sync(kFull, (unsigned)(v >> 32), d);
  return ((unsigned long long)hi << 32) | lo;
}
__device__ __forceinline__ long long shfl_xor_s64(long long v, int m) {
  const unsigned lo = __shfl_xor_sync(kFull, (unsigned)v, m);
  const unsigned hi = __shfl_xor_sync(kFull, (unsigned)((unsigned long long)v >> 32), m);
  return (long long)(((unsigned long long)hi << 32) | lo);
}

__device__ void run_region_warp(const KParams& p, const Lat& lt, int r, int n_iter, unsigned cidx,
                                double t_s, double t_end, Acc& acc) {
  const int lane = threadIdx.x & 31;
  const int W = p.W, H = p.H;
  const size_t nr = (size_t)p.NR;
  const size_t cap = (size_t)p.cap;
  const int wp = n_iter & 1, rp = wp ^ 1;
  const int rx = lt.loc % lt.NX, ry = lt.loc / lt.NX;
  const bool spx = lt.spans_x, spy = lt.spans_y;
  const uint32_t wmask = (W == 32) ? 0xFFFFFFFFu : ((1u << W) - 1u);
  const bool vlane = lane < H;
  const bool has_y = !spy, has_x = !spx;
  const double INF = __longlong_as_double(0x7FF0000000000000ll);

  // lane d < 4 serves direction d (0 N, 1 S, 2 W, 3 E)
  int qd = 0;
  if (lane == 0) qd = lt.off + ((ry + lt.NY - 1) % lt.NY) * lt.NX + rx;
  else if (lane == 1) qd = lt.off + ((ry + 1) % lt.NY) * lt.NX + rx;
  else if (lane == 2) qd = lt.off + ry * lt.NX + (rx + lt.NX - 1) % lt.NX;
  else if (lane == 3) qd = lt.off + ry * lt.NX + (rx + 1) % lt.NX;
  const bool hasd = (lane < 2 && has_y) || (lane >= 2 && lane < 4 && has_x);

  // ---- skip when no neighbour's lists changed in the last iteration
  if (n_iter >= 2) {
    const bool dirty = hasd && __ldcg(&p.chg[(size_t)rp * nr + qd]) != 0;
    if (!__any_sync(kFull, dirty)) {
      for (int e = 0; e < 4; ++e) {
        if (!((e < 2) ? has_y : has_x)) continue;
        const unsigned n = __ldcg(&p.hl[((size_t)rp * 4 + e) * nr + r]);
        for (unsigned j = lane; j < n; j += 32) {
          const size_t src = (((size_t)rp * 4 + e) * cap + j) * nr + r;
          const size_t dst = (((size_t)wp * 4 + e) * cap + j) * nr + r;
          p.ht[dst] = __ldcg(&p.ht[src]);
          p.hp[dst] = __ldcg(&p.hp[src]);
        }
        if (lane == 0) p.hl[((size_t)wp * 4 + e) * nr + r] = n;
      }
      if (lane == 0) {
        p.chg[(size_t)wp * nr + r] = 0;
        acc.skips += 1;
      }
      return;
    }
  }
  if (lane == 0) acc.passes += 1;

  // ---- committed state
  uint32_t row = vlane ? __ldcg(&p.rows[((size_t)cidx * H + lane) * nr + r]) : 0u;
  uint32_t hN = __ldcg(&p.halo[0 * nr + r]), hS = __ldcg(&p.halo[1 * nr + r]);
  uint32_t hW = __ldcg(&p.halo[2 * nr + r]), hE = __ldcg(&p.halo[3 * nr + r]);
  unsigned long long i = __ldcg(&p.ci[cidx * nr + r]);
  double x = __ldcg(&p.cx[cidx * nr + r]);
  unsigned long long kv = __ldcg(&p.ckv[cidx * nr + r]);
  double b = __ldcg(&p.cb[cidx * nr + r]);
  double tl = __ldcg(&p.ct[cidx * nr + r]);
  const unsigned long long hi_ring = __ldcg(&p.rhi[r]);
  const unsigned long long kmask = (unsigned long long)p.K - 1ull;
  double px = 0.0;
  unsigned long long pkv = 0ull;
  bool pvalid = (i + 1ull) < hi_ring;
  if (pvalid) {
    const size_t a = (size_t)((i + 1ull) & kmask) * nr + r;
    px = __ldcg(&p.rx[a]);
    pkv = __ldcg(&p.rkv[a]);
  }
  const int F = p.F;

  // neighbour words and per-position up counts of my row
  uint32_t s0, s1, s2;
  auto refresh = [&]() {
    const uint32_t vu = __shfl_sync(kFull, row, lane > 0 ? lane - 1 : H - 1);
    const uint32_t vd = __shfl_sync(kFull, row, lane < H - 1 ? lane + 1 : 0);
    const uint32_t up = (lane > 0 || spy) ? vu : hN;
    const uint32_t dn = (lane < H - 1 || spy) ? vd : hS;
    const uint32_t lb = spx ? (row >> (W - 1)) & 1u : (hW >> lane) & 1u;
    const uint32_t rb = spx ? (row & 1u) : (hE >> lane) & 1u;
    const uint32_t lf = ((row << 1) | lb) & wmask;
    const uint32_t rt = (row >> 1) | (rb << (W - 1));
    add4(up, dn, lf, rt, s0, s1, s2);
  };
  refresh();

  // ---- class counts (lane k holds N_k) and Lambda
  unsigned myN = 0;
  unsigned long long lam = 0ull;
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    const uint32_t e = vlane ? (eq_count(s0, s1, s2, k % 5) & (k >= 5 ? row : ~row) & wmask) : 0u;
    const unsigned tot = __reduce_add_sync(kFull, (unsigned)__popc(e));
    if (lane == k) myN = tot;
    lam += (unsigned long long)tot * lt.P[k];
  }
  int mag0 = 0, bond0 = 0;
  {
    const uint32_t vd = __shfl_sync(kFull, row, lane < H - 1 ? lane + 1 : 0);
    const uint32_t dn = (lane < H - 1 || spy) ? vd : hS;
    const uint32_t rb = spx ? (row & 1u) : (hE >> lane) & 1u;
    const uint32_t rt = (row >> 1) | (rb << (W - 1));
    const int m = vlane ? 2 * __popc(row) - W : 0;
    const int bd = vlane ? (W - 2 * __popc((row ^ rt) & wmask)) + (W - 2 * __popc((row ^ dn) & wmask)) : 0;
    mag0 = __reduce_add_sync(kFull, m);
    bond0 = __reduce_add_sync(kFull, bd);
  }

  // ---- incoming cursors (lane d), two entries buffered
  const int ein = (lane == 0) ? 1 : (lane == 1) ? 0 : (lane == 2) ? 3 : 2;
  unsigned len = 0, idx = 0, npos = 0, npos2 = 0;
  double nt = INF, nt2 = INF;
  if (hasd && n_iter >= 2) {     // iteration 1: the canonical assumption (§5)
    len = __ldcg(&p.hl[((size_t)rp * 4 + ein) * nr + qd]);
    if (len > 0) {
      const size_t a = (((size_t)rp * 4 + ein) * cap) * nr + qd;
      nt = __ldcg(&p.ht[a]);
      npos = __ldcg(&p.hp[a]);
    }
    if (len > 1) {
      const size_t a = (((size_t)rp * 4 + ein) * cap + 1) * nr + qd;
      nt2 = __ldcg(&p.ht[a]);
      npos2 = __ldcg(&p.hp[a]);
    }
  }

  unsigned olen0 = 0, olen1 = 0, olen2 = 0, olen3 = 0;
  bool overflow = false;
  unsigned long long events = 0, brk = 0;
  unsigned bevents = 0;
  int ksig = 0, kbeta = 0;
  const int frac = 62 - (int)((((unsigned long long)__double_as_longlong(t_end)) >> 52) - 1022);
  Acc128 ssig = {0ull, 0}, sbeta = {0ull, 0};
  const uint32_t gx0 = (uint32_t)(rx * W), gy0 = (uint32_t)(ry * H);

  double tau = tau_soft(tl, x, b, lam, F);
  for (;;) {
    // earliest pending break point over the four cursor lanes
    long long key = (lane < 4) ? __double_as_longlong(nt) : 0x7FF0000000000000ll;
    int who = lane;
#pragma unroll
    for (int m = 1; m <= 2; m <<= 1) {
      const long long ok = shfl_xor_s64(key, m);
      const int ow = __shfl_xor_sync(kFull, who, m);
      if (ok < key || (ok == key && ow < who)) {
        key = ok;
        who = ow;
      }
    }
    key = (long long)shfl_u64((unsigned long long)key, 0);
    who = __shfl_sync(kFull, who, 0);
    const long long tau_b = __double_as_longlong(tau);

    if (tau_b <= key) {
      if (!(tau_b < __double_as_longlong(t_end))) break;
      // ---- class k*: prefix sums A(k) of N_k p_k over lanes 0..9 (Eqs. 3.5-3.6)
      const unsigned long long mV = 2ull * kv + 1ull;
      const unsigned long long plo = mV * lam, phi = __umul64hi(mV, lam);
      const unsigned long long q53 = (phi << 11) | (plo >> 53);
      const bool exact = (plo & ((1ull << 53) - 1ull)) == 0ull;
      const unsigned long long term = (lane < 10) ? (unsigned long long)myN * lt.P[lane < 10 ? lane : 0] : 0ull;
      unsigned long long A = term;
#pragma unroll
      for (int d = 1; d < 16; d <<= 1) {
        const unsigned long long o = shfl_up_u64(A, d);
        if (lane >= d) A += o;
      }
      const bool hit = lane < 10 && (q53 < A || (q53 == A && exact));
      const int ks = __ffs(__ballot_sync(kFull, hit)) - 1;
      const unsigned long long Aprev = shfl_u64(A - term, ks);
      const unsigned Nks = __shfl_sync(kFull, myN, ks);
      const unsigned long long Pk = lt.P[ks];
      // position in the class (Eqs. 3.7-3.8): floor((V Lambda - A(k*-1)) / p_k*)
      unsigned long long jl = class_pos(q53 - Aprev, Pk, lt.Rp[ks]);
      if (jl >= Nks) jl = Nks - 1;
      const unsigned j = (unsigned)jl;
      // the j-th class-k* site in row-major order
      const int sp = ks >= 5;
      const int nn = ks - 5 * sp;
      const uint32_t mrow = vlane ? (eq_count(s0, s1, s2, nn) & (sp ? row : ~row) & wmask) : 0u;
      const unsigned cnt = __popc(mrow);
      unsigned cum = cnt;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned o = __shfl_up_sync(kFull, cum, d);
        if (lane >= d) cum += o;
      }
      const int fy = __ffs(__ballot_sync(kFull, vlane && j < cum)) - 1;
      const unsigned before = __shfl_sync(kFull, cum - cnt, fy);
      const int fxl = nth_set_bit(mrow, j - before);
      const int fx = __shfl_sync(kFull, fxl, fy);
      const int s_old = (__shfl_sync(kFull, row, fy) >> fx) & 1;

      // ---- classes before the flip of the site and its in-region neighbours
      auto nup_at = [&](int xx) -> int {
        return (int)(((s0 >> xx) & 1u) + 2u * ((s1 >> xx) & 1u) + 4u * ((s2 >> xx) & 1u));
      };
      // lane fy packs (v, left, right); its row neighbours pack (x*)
      unsigned pk_mid = 0u, pk_vert = 0u;
      if (lane == fy) {
        const int cv = 5 * s_old + nup_at(fx);
        pk_mid = (unsigned)cv | 0x10u;
        if (fx > 0 || spx) {
          const int xl = fx > 0 ? fx - 1 : W - 1;
          pk_mid |= ((unsigned)(5 * ((row >> xl) & 1u) + nup_at(xl)) | 0x10u) << 5;
        }
        if (fx < W - 1 || spx) {
          const int xr = fx < W - 1 ? fx + 1 : 0;
          pk_mid |= ((unsigned)(5 * ((row >> xr) & 1u) + nup_at(xr)) | 0x10u) << 10;
        }
      }
      const int yu = fy > 0 ? fy - 1 : H - 1;
      const int yd = fy < H - 1 ? fy + 1 : 0;
      const bool hu = fy > 0 || spy, hd = fy < H - 1 || spy;
      if ((lane == yu && hu) || (lane == yd && hd))
        pk_vert = ((unsigned)(5 * ((row >> fx) & 1u) + nup_at(fx))) | 0x10u;
      const unsigned m_mid = __shfl_sync(kFull, pk_mid, fy);
      const unsigned m_up = hu ? __shfl_sync(kFull, pk_vert, yu) : 0u;
      const unsigned m_dn = hd ? __shfl_sync(kFull, pk_vert, yd) : 0u;
      const int dnb = s_old ? -1 : 1;
      int dN = 0;
      long long dlam = 0;
      auto apply = [&](unsigned code, int delta) {
        if (!(code & 0x10u)) return;
        const int from = (int)(code & 0xFu), to = from + delta;
        dN += (lane == to) - (lane == from);
        dlam += (long long)(lt.P[to] - lt.P[from]);
      };
      apply(m_mid & 0x1Fu, s_old ? -5 : 5);
      apply((m_mid >> 5) & 0x1Fu, dnb);
      apply((m_mid >> 10) & 0x1Fu, dnb);
      apply(m_up, dnb);
      apply(m_dn, dnb);
      myN = (unsigned)((int)myN + dN);
      lam = lam + (unsigned long long)dlam;
      if (lane == fy) row ^= (1u << fx);

      // ---- observables: dM = 2 sig, dBonds = 4 beta
      const int sig = s_old ? -1 : 1;
      const int nup_v = (int)(m_mid & 0xFu) - 5 * s_old;
      const int beta = sig * (nup_v - 2);
      const unsigned long long tfix = to_fixed(tau, frac);
      ksig += sig;
      ssig.add(sig, tfix);
      kbeta += beta;
      sbeta.add(beta, tfix);

      // ---- boundary history (lane 0 writes; compared at the end)
      bool boundary = false;
      if (has_y && fy == 0) {
        if (olen0 >= cap) overflow = true;
        else if (lane == 0) {
          const size_t a = (((size_t)wp * 4 + 0) * cap + olen0) * nr + r;
          p.ht[a] = tau;
          p.hp[a] = (uint8_t)fx;
        }
        ++olen0;
        boundary = true;
      }
      if (has_y && fy == H - 1) {
        if (olen1 >= cap) overflow = true;
        else if (lane == 0) {
          const size_t a = (((size_t)wp * 4 + 1) * cap + olen1) * nr + r;
          p.ht[a] = tau;
          p.hp[a] = (uint8_t)fx;
        }
        ++olen1;
        boundary = true;
      }
      if (has_x && fx == 0) {
        if (olen2 >= cap) overflow = true;
        else if (lane == 0) {
          const size_t a = (((size_t)wp * 4 + 2) * cap + olen2) * nr + r;
          p.ht[a] = tau;
          p.hp[a] = (uint8_t)fy;
        }
        ++olen2;
        boundary = true;
      }
      if (has_x && fx == W - 1) {
        if (olen3 >= cap) overflow = true;
        else if (lane == 0) {
          const size_t a = (((size_t)wp * 4 + 3) * cap + olen3) * nr + r;
          p.ht[a] = tau;
          p.hp[a] = (uint8_t)fy;
        }
        ++olen3;
        boundary = true;
      }
      if (boundary) ++bevents;
      if (lane == 0 && p.tcap > 0 && i < (unsigned long long)p.tcap) {
        p.trt[(size_t)r * p.tcap + i] = tau;
        p.trs[(size_t)r * p.tcap + i] = (gy0 + fy) * (uint32_t)lt.L + gx0 + fx;
      }
      ++events;
      if (overflow) break;
      // ---- next event: clock restarts at tau with the next presimulated pair
      tl = tau;
      b = 0.0;
      ++i;
      if (pvalid) {
        x = px;
        kv = pkv;
      } else {
        draw_event(i, (uint32_t)lt.loc, lt.key0, lt.key1, x, kv);
      }
      pvalid = (i + 1ull) < hi_ring;
      if (pvalid) {
        const size_t a = (size_t)((i + 1ull) & kmask) * nr + r;
        px = __ldcg(&p.rx[a]);
        pkv = __ldcg(&p.rkv[a]);
      }
      refresh();
    } else {
      // ---- break point at tb from direction `who` (§5, Eqs. 5.2-5.6)
      const double tb = __longlong_as_double(key);
      b = sf::add_pos(b, sf::mul_pos(sf::u64_scaled(lam, F), sf::sub_pos(tb, tl)));
      tl = tb;
      const int pos = (int)__shfl_sync(kFull, npos, who);
      int ux, uy, up_now;
      if (who == 0) { hN ^= 1u << pos; up_now = (hN >> pos) & 1u; ux = pos; uy = 0; }
      else if (who == 1) { hS ^= 1u << pos; up_now = (hS >> pos) & 1u; ux = pos; uy = H - 1; }
      else if (who == 2) { hW ^= 1u << pos; up_now = (hW >> pos) & 1u; ux = 0; uy = pos; }
      else { hE ^= 1u << pos; up_now = (hE >> pos) & 1u; ux = W - 1; uy = pos; }
      refresh();
      // class of the adjacent site after the change (owner lane uy), before it one less/more
      const int cnew_l = 5 * (int)((row >> ux) & 1u) +
                         (int)(((s0 >> ux) & 1u) + 2u * ((s1 >> ux) & 1u) + 4u * ((s2 >> ux) & 1u));
      const int cnew = __shfl_sync(kFull, cnew_l, uy);
      const int cold = cnew + (up_now ? -1 : 1);
      myN = (unsigned)((int)myN + (lane == cnew) - (lane == cold));
      lam = lam - lt.P[cold] + lt.P[cnew];
      if (lane == who) {                     // advance the cursor
        ++idx;
        nt = nt2;
        npos = npos2;
        if (idx + 1 < len) {
          const size_t a = (((size_t)rp * 4 + ein) * cap + idx + 1) * nr + qd;
          nt2 = __ldcg(&p.ht[a]);
          npos2 = __ldcg(&p.hp[a]);
        } else {
          nt2 = INF;
        }
      }
      ++brk;
    }
    tau = tau_soft(tl, x, b, lam, F);
  }

  // ---- compare the new lists with the previous ones (§4 statement (c))
  __syncwarp();
  bool changed = overflow;
  for (int e = 0; e < 4; ++e) {
    if (!((e < 2) ? has_y : has_x)) continue;
    const unsigned nn = (e == 0) ? olen0 : (e == 1) ? olen1 : (e == 2) ? olen2 : olen3;
    const unsigned n_new = nn < (unsigned)cap ? nn : (unsigned)cap;
    const unsigned n_old = n_iter >= 2 ? __ldcg(&p.hl[((size_t)rp * 4 + e) * nr + r]) : 0u;
    bool diff = n_new != n_old;
    const unsigned n_min = n_new < n_old ? n_new : n_old;
    for (unsigned j = lane; j < n_min; j += 32) {
      const size_t an = (((size_t)wp * 4 + e) * cap + j) * nr + r;
      const size_t ao = (((size_t)rp * 4 + e) * cap + j) * nr + r;
      if (__double_as_longlong(__ldcg(&p.ht[an])) != __double_as_longlong(__ldcg(&p.ht[ao])) ||
          __ldcg(&p.hp[an]) != __ldcg(&p.hp[ao]))
        diff = true;
    }
    changed |= __any_sync(kFull, diff);
    if (lane == 0) p.hl[((size_t)wp * 4 + e) * nr + r] = n_new;
  }
  if (lane == 0) p.chg[(size_t)wp * nr + r] = changed ? 1 : 0;

  // ---- tentative end state
  const unsigned tc = cidx ^ 1u;
  if (vlane) p.rows[((size_t)tc * H + lane) * nr + r] = row;
  if (lane == 0) {
    p.ci[tc * nr + r] = i;
    p.cx[tc * nr + r] = x;
    p.ckv[tc * nr + r] = kv;
    p.cb[tc * nr + r] = b;
    p.ct[tc * nr + r] = tl;
    // window integrals: M0 span + 2 (t_end K - S), bonds likewise with 4
    const double span = __dsub_rn(t_end, t_s);
    const Acc128 um = window_moment(ksig, t_end, frac, ssig);
    const Acc128 ub = window_moment(kbeta, t_end, frac, sbeta);
    const double im = __dadd_rn(__dmul_rn((double)mag0, span), __dmul_rn(2.0, um.value(frac)));
    const double ib = __dadd_rn(__dmul_rn((double)bond0, span), __dmul_rn(4.0, ub.value(frac)));
    p.cim[tc * nr + r] = __dadd_rn(__ldcg(&p.cim[cidx * nr + r]), im);
    p.cib[tc * nr + r] = __dadd_rn(__ldcg(&p.cib[cidx * nr + r]), ib);
    acc.events += events;
    acc.breaks += brk;
    if (bevents > acc.fmax) acc.fmax = bevents;
    if ((unsigned)events > acc.emax) acc.emax = (unsigned)events;
    acc.changed |= changed;
    acc.overflow |= overflow;
  }
}

// Halo words of region r from copy `cidx` of the rows of its four neighbours.
__device__ void compute_halo(const KParams& p, const Lat& lt, int r, unsigned cidx) {
  const size_t nr = (size_t)p.NR;
  const int rx = lt.loc % lt.NX, ry = lt.loc / lt.NX;
  const uint32_t* rows_c = p.rows + (size_t)cidx * p.H * nr;
  uint32_t hN = 0, hS = 0, hW = 0, hE = 0;
  if (!lt.spans_y) {
    const int qN = lt.off + ((ry + lt.NY - 1) % lt.NY) * lt.NX + rx;
    const int qS = lt.off + ((ry + 1) % lt.NY) * lt.NX + rx;
    hN = __ldcg(&rows_c[(size_t)(p.H - 1) * nr + qN]);
    hS = __ldcg(&rows_c[qS]);
  }
  if (!lt.spans_x) {
    const int qW = lt.off + ry * lt.NX + (rx + lt.NX - 1) % lt.NX;
    const int qE = lt.off + ry * lt.NX + (rx + 1) % lt.NX;
    for (int y = 0; y < p.H; ++y) {
      hW |= ((__ldcg(&rows_c[(size_t)y * nr + qW]) >> (p.W - 1)) & 1u) << y;
      hE |= (__ldcg(&rows_c[(size_t)y * nr + qE]) & 1u) << y;
    }
  }
  p.halo[0 * nr + r] = hN;
  p.halo[1 * nr + r] = hS;
  p.halo[2 * nr + r] = hW;
  p.halo[3 * nr + r] = hE;
}

// A region whose inputs for the coming iteration equal those of the last one
// keeps its tentative state; its lists are carried to the new parity wp.
__device__ void carry_lists(const KParams& p, int r, int wp, bool spans_x, bool spans_y) {
  const size_t nr = (size_t)p.NR, cap = (size_t)p.cap;
  const int rp = wp ^ 1;
  for (int e = 0; e < 4; ++e) {
    if ((e < 2 && spans_y) || (e >= 2 && spans_x)) continue;
    const unsigned n = __ldcg(&p.hl[((size_t)rp * 4 + e) * nr + r]);
    for (unsigned j = 0; j < n; ++j) {
      const size_t src = (((size_t)rp * 4 + e) * cap + j) * nr + r;
      const size_t dst = (((size_t)wp * 4 + e) * cap + j) * nr + r;
      p.ht[dst] = __ldcg(&p.ht[src]);
      p.hp[dst] = __ldcg(&p.hp[src]);
    }
    p.hl[((size_t)wp * 4 + e) * nr + r] = n;
  }
  p.chg[(size_t)wp * nr + r] = 0;
}

// Append region r to work list `buf` when `want`; the lanes that reach this
// point together share one atomic.
__device__ __forceinline__ void wl_append(const KParams& p, unsigned buf, int r, bool want) {
  const unsigned mask = __activemask();
  const unsigned bal = __ballot_sync(mask, want);
  const int leader = __ffs(mask) - 1;
  const int lane = threadIdx.x & 31;
  unsigned base = 0u;
  if (lane == leader && bal) base = atomicAdd(&p.st->wl_count[buf], (unsigned)__popc(bal));
  base = __shfl_sync(mask, base, leader);
  if (want) p.wl[(size_t)buf * p.NR + base + __popc(bal & ((1u << lane) - 1u))] = (uint32_t)r;
}

// ---------------------------------------------------------------- persistent kernel
// The DO(step) / DO(iteration) loops of the §4 procedure for nwin windows.
// Ring top-up at a window start: the block's threads together draw the pairs of
// events [max(rhi, i_c), i_c + K) for each region of the block that has a
// top-up pending (the regions of its slots: b*rl + l + k*gridDim.x*rl).
__device__ void fill_ring(const KParams& p) {
  const size_t nr = (size_t)p.NR;
  const unsigned long long kmask = (unsigned long long)p.K - 1ull;
  const int lstride = gridDim.x * p.rl;
  for (int l = 0; l < p.rl; ++l) {
    for (int r = blockIdx.x * p.rl + l; r < p.NR; r += lstride) {
      if (!p.rfill[r]) continue;
      const Lat lt = lat_of(p, r);
      const unsigned long long lo = __ldcg(&p.ci[(size_t)p.rcidx[r] * nr + r]);
      const unsigned long long hi_old = p.rhi[r];
      // the alternate step rule starts every window on new numbers: refill all
      const unsigned long long from = (hi_old > lo && !p.fresh) ? hi_old : lo;
      const unsigned long long to = lo + (unsigned long long)p.K;
      const unsigned wg = p.reps[lt.rep].w0 + p.rwin[r];
      for (unsigned long long i = from + threadIdx.x; i < to; i += blockDim.x) {
        double x;
        unsigned long long kv;
        if (p.fresh)
          draw_event_fresh((unsigned)(i - lo), wg, (uint32_t)lt.loc, lt.key0, lt.key1, x, kv);
        else
          draw_event(i, (uint32_t)lt.loc, lt.key0, lt.key1, x, kv);
        const size_t a = (size_t)(i & kmask) * nr + r;
        p.rx[a] = x;
        p.rkv[a] = kv;
      }
    }
  }
  __syncthreads();
  for (int l = threadIdx.x; l < p.rl; l += blockDim.x)
    for (int r = blockIdx.x * p.rl + l; r < p.NR; r += lstride)
      if (p.rfill[r]) {
        p.rhi[r] = __ldcg(&p.ci[(size_t)p.rcidx[r] * nr + r]) + (unsigned long long)p.K;
        p.rfill[r] = 0;
      }
  __syncthreads();
}

// Ring top-up of one region by one lane (asynchronous schedule): the pairs of
// events [max(rhi, i_c), i_c + K) (all K under the alternate step rule, whose
// window wg starts on new numbers).
__device__ void fill_own(const KParams& p, int r, const Lat& lt, unsigned wg) {
  const size_t nr = (size_t)p.NR;
  const unsigned long long kmask = (unsigned long long)p.K - 1ull;
  const unsigned long long lo = __ldcg(&p.ci[(size_t)p.rcidx[r] * nr + r]);
  const unsigned long long hi_old = p.rhi[r];
  const unsigned long long from = (hi_old > lo && !p.fresh) ? hi_old : lo;
  const unsigned long long to = lo + (unsigned long long)p.K;
  for (unsigned long long i = from; i < to; ++i) {
    double x;
    unsigned long long kv;
    if (p.fresh)
      draw_event_fresh((unsigned)(i - lo), wg, (uint32_t)lt.loc, lt.key0, lt.key1, x, kv);
    else
      draw_event(i, (uint32_t)lt.loc, lt.key0, lt.key1, x, kv);
    const size_t a = (size_t)(i & kmask) * nr + r;
    p.rx[a] = x;
    p.rkv[a] = kv;
  }
  p.rhi[r] = to;
}

// Task queue of the asynchronous schedule: a task is (kind, lattice, chunk of
// `chunk` consecutive regions); kinds 0 = pass, 1 = commit.  The publishing
// thread has made the lattice's state visible first (fence).
constexpr unsigned long long kTaskValid = 1ull << 62;
__device__ void enqueue_lattice(const KParams& p, int b, unsigned kind, int chunk) {
  const int nreg = p.reps[b].NR;
  const unsigned long long nch = (unsigned long long)((nreg + chunk - 1) / chunk);
  __threadfence();
  const unsigned long long base = atomicAdd(&p.st->qtail, nch);
  for (unsigned long long c = 0; c < nch; ++c) {
    const unsigned long long item = kTaskValid | ((unsigned long long)kind << 60) |
                                    ((unsigned long long)b << 32) | c;
    atomicExch(&p.q[(base + c) % p.qcap], item);
  }
}

#ifndef SR_WARP_MIN_BLOCKS
#define SR_WARP_MIN_BLOCKS 7
#endif
#ifndef SR_LANE_MAX_THREADS
#define SR_LANE_MAX_THREADS 256
#endif
#ifndef SR_LANE_MIN_BLOCKS
#define SR_LANE_MIN_BLOCKS 2
#endif
// MODE 0 / 2: one lane per region with FP64 / integer-emulated time
// arithmetic; the first `lanes` lanes of every warp are region lanes.  MODE 1:
// one warp per region.  Region slot j of block b owns regions
// b*rl + j + k*(gridDim.x*rl).
template <int MODE, int DYN>
__global__ void __launch_bounds__(MODE == 1 ? 128 : SR_LANE_MAX_THREADS,
                                   MODE == 1 ? SR_WARP_MIN_BLOCKS : SR_LANE_MIN_BLOCKS)
    relax_kernel(KParams p) {
  extern __shared__ uint32_t smem[];
  if ((int)blockIdx.x == p.skip_block) return;   // test hook: never reaches a barrier
  constexpr bool LANES = MODE != 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int slot = LANES ? warp * p.lanes + lane : warp;
  const bool is_slot = (LANES ? lane < p.lanes : true) && slot < p.rl;
  const int sstride = gridDim.x * p.rl;
  const int sfirst = is_slot ? (int)(blockIdx.x * p.rl + slot) : p.NR;
  Region g;
  const int stride = p.rl;
  g.hq = (p.H + 3) / 4;
  g.rows = smem + (LANES && is_slot ? slot : 0);
  g.C = smem + p.H * stride + (LANES && is_slot ? slot : 0);
  {
    const int pt_words = ((p.H + 10 * g.hq) * stride + 1) & ~1;   // 8-byte aligned table
    g.PT = reinterpret_cast<unsigned long long*>(smem + pt_words) + (LANES && is_slot ? slot : 0);
    g.SX = g.PT + 20 * stride;                                       // score mode only
  }
  g.cur_rep = -1;
  g.stride = stride;
  g.W = p.W;
  g.H = p.H;
  g.wmask = (p.W == 32) ? 0xFFFFFFFFu : ((1u << p.W) - 1u);
  DevStats* st = p.st;
  const size_t nr = (size_t)p.NR;
  const bool reporter = LANES ? true : (threadIdx.x & 31) == 0;
  unsigned long long run_cyc = 0ull;
  // per-slot busy cycles, reported when the launch ends normally
  struct Report {
    DevStats* st;
    const unsigned long long* cyc;
    bool on;
    __device__ ~Report() {
      if (on) {
        atomicAdd(&st->run_cycles, *cyc);
        atomicMax(&st->run_cycles_max, *cyc);
        atomicAdd(&st->slots, 1ull);
      }
    }
  } report{st, &run_cyc, reporter && is_slot};

  // ---- launch start: every region begins iteration 1 of its lattice's first window
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    unsigned active = 0;
    for (int b = 0; b < p.nrep; ++b) active += p.reps[b].nwin > 0 ? 1u : 0u;
    st->active = active;
  }
  if (blockIdx.x == 0)
    for (int b = threadIdx.x; b < p.nrep; b += blockDim.x) p.rs[b].windows_done = 0u;
  if (is_slot && (LANES || (threadIdx.x & 31) == 0)) {
    for (int r = sfirst; r < p.NR; r += sstride) {
      const RepDesc* d = p.reps + __ldg(&p.rrep[r]);
      p.rn[r] = 1u;
      p.rwin[r] = 0u;
      p.rts[r] = d->t0;
      p.rfill[r] = d->nwin > 0 ? 1 : 0;
      if (DYN == 1) wl_append(p, 0u, r, d->nwin > 0);  // every region runs iteration 1
    }
  }
  __syncthreads();
  fill_ring(p);
  if (DYN) {
    // a region's first pass may run on another block: its state and ring first
    if (!grid_barrier(st, p.timeout_cycles)) return;
  }

  if constexpr (DYN == 2) {
    // ---- asynchronous schedule (lane mapping): every lattice advances on its
    // own.  A warp takes a task (a chunk of one lattice's regions) from the
    // queue; the warp that finishes the last task of a lattice's iteration
    // decides for that lattice alone -- iterate again (pass tasks) or commit
    // (commit tasks, then the next window's pass tasks).  No grid-wide
    // synchronize; every wait is bounded.
    if (!LANES) return;
    constexpr unsigned kStop = ST_CAPACITY | ST_NOT_CONVERGED | ST_TIMEOUT;
    constexpr unsigned long long kCworkStop = 1ull << 63;
    // an error stops new work; the commits already published still run, so no
    // lattice is left half committed (a decision that meets the stop bit
    // withdraws its commit before publishing it)
    auto stop_all = [&](unsigned bit) {
      atomicOr(&st->status, bit);
      atomicOr(&st->cwork, kCworkStop);
    };
    const int CH = p.lanes;
    for (;;) {
      unsigned long long item = 0ull;
      if (lane == 0) {
        const unsigned long long slot = atomicAdd(&st->qhead, 1ull) % p.qcap;
        const long long tw0 = clock64();
        for (;;) {
          item = *(volatile unsigned long long*)&p.q[slot];
          if (item) break;
          if (*(volatile unsigned*)&st->active == 0u) break;           // all lattices done
          if (*(volatile unsigned*)&st->status & ST_TIMEOUT) break;
          if (*(volatile unsigned long long*)&st->cwork == kCworkStop) break;  // stopped, drained
          if (clock64() - tw0 > p.timeout_cycles) {
            stop_all(ST_TIMEOUT);
            break;
          }
          __nanosleep(128);
        }
        if (item) atomicExch(&p.q[slot], 0ull);
        __threadfence();
      }
      item = __shfl_sync(0xFFFFFFFFu, item, 0);
      if (!item) break;
      __syncwarp();          // every lane's reads come after lane 0's acquire
      const unsigned kind = (unsigned)((item >> 60) & 3ull);
      const int b = (int)((item >> 32) & 0x0FFFFFFFull);
      const int c = (int)(item & 0xFFFFFFFFull);
      const RepDesc* d = p.reps + b;
      LatState* Ls = p.ls + b;
      const int loc = c * CH + lane;
      const bool mine = is_slot && lane < CH && loc < d->NR;
      const int r = d->off + loc;
      const unsigned cnt = (unsigned)__popc(__ballot_sync(0xFFFFFFFFu, mine));
      const unsigned w = *(volatile unsigned*)&Ls->w;
      RepStats* rs = p.rs + b;
      if (kind == 1u) {
        // ---- commit of window w (statement 3 of §4): the tentative state of
        // the converged iteration becomes the committed one
        if (mine) {
          const unsigned cnew = p.rcidx[r] ^ 1u;
          const unsigned long long dc = __ldcg(&p.ci[(size_t)cnew * nr + r]) -
                                        __ldcg(&p.ci[(size_t)(cnew ^ 1u) * nr + r]);
          if (dc) atomicAdd(&rs->committed, dc);
          p.rcidx[r] = (uint8_t)cnew;
          const Lat lt = lat_of(p, r);
          compute_halo(p, lt, r, cnew);
          if (w + 1u < (unsigned)d->nwin) fill_own(p, r, lt, d->w0 + w + 1u);
        }
        __syncwarp();        // every lane's writes come before lane 0's release
        if (lane == 0) {
          __threadfence();
          const unsigned old = atomicSub(&Ls->pend, cnt);
          if (old == cnt) {
            const unsigned wn = w + 1u;
            const unsigned n = Ls->n;                 // iterations of window w
            rs->windows += 1ull;
            rs->iterations += (unsigned long long)n;
            rs->last_iters = n;
            if (n > rs->max_iters_seen) rs->max_iters_seen = n;
            const unsigned fw = p.curf[(w & 1u) * p.nrep + b];
            p.curf[(w & 1u) * p.nrep + b] = 0u;
            rs->sum_f += fw;
            if (b == 0) {
              p.win_iters[w % kWinRing] = n;
              p.win_iters[kWinRing + w % kWinRing] = fw;
            }
            Ls->w = wn;
            rs->windows_done = wn;
            if (wn < (unsigned)d->nwin && !(*(volatile unsigned*)&st->status & kStop)) {
              Ls->n = 1u;
              Ls->chg = 0u;
              Ls->ovf = 0u;
              Ls->pend = (unsigned)d->NR;
              Ls->ts = __dadd_rn(Ls->ts, d->Tw);
              enqueue_lattice(p, b, 0u, CH);
            }
            __threadfence();
            if (wn == (unsigned)d->nwin) atomicSub(&st->active, 1u);
          }
          atomicAdd(&st->cwork, 0ull - (unsigned long long)cnt);
        }
      } else {
        // ---- iteration n of window w; after an error no new passes run
        if (*(volatile unsigned*)&st->status & kStop) continue;
        const unsigned n = *(volatile unsigned*)&Ls->n;
        const double t_s = *(volatile double*)&Ls->ts;
        const double t_end = __dadd_rn(t_s, d->Tw);
        Acc ra = {0u, 0u, 0u, 0u, 0u, 0u, false, false};
        if (mine) {
          const Lat lt = lat_of(p, r);
          const unsigned cidx = p.rcidx[r];
          if (MODE == 2)
            run_region<1>(p, lt, r, (int)n, cidx, t_s, t_end, d->w0 + w, g, ra);
          else
            run_region<0>(p, lt, r, (int)n, cidx, t_s, t_end, d->w0 + w, g, ra);
          if (ra.fmax) atomicMax(&p.curf[(w & 1u) * p.nrep + b], ra.fmax);
          if (ra.events) atomicAdd(&rs->generated, (unsigned long long)ra.events);
          if (ra.breaks) atomicAdd(&rs->breaks, (unsigned long long)ra.breaks);
          if (ra.fmax) atomicMax(&rs->max_f, ra.fmax);
          if (ra.emax) atomicMax(&rs->max_win_events, ra.emax);
          if (ra.passes) atomicAdd(&st->region_passes, (unsigned long long)ra.passes);
          if (ra.skips) atomicAdd(&st->region_skips, (unsigned long long)ra.skips);
        }
        const bool anych = __any_sync(0xFFFFFFFFu, mine && ra.changed);
        const bool anyov = __any_sync(0xFFFFFFFFu, mine && ra.overflow);
        __syncwarp();        // every lane's writes come before lane 0's release
        if (lane == 0) {
          if (anych) atomicOr(&Ls->chg, 1u);
          if (anyov) atomicOr(&Ls->ovf, 1u);
          __threadfence();
          const unsigned old = atomicSub(&Ls->pend, cnt);
          if (old == cnt) {
            __threadfence();
            const unsigned ch = *(volatile unsigned*)&Ls->chg;
            const unsigned ov = *(volatile unsigned*)&Ls->ovf;
            if (ov) {
              stop_all(ST_CAPACITY);
            } else if (!ch) {
              // no region of this lattice changed its lists: the fixed point;
              // commit tasks follow (the window's statistics count at their end)
              Ls->pend = (unsigned)d->NR;
              const unsigned long long before = atomicAdd(&st->cwork, (unsigned long long)d->NR);
              if (before & kCworkStop)
                atomicAdd(&st->cwork, 0ull - (unsigned long long)d->NR);   // stopped: no commit
              else
                enqueue_lattice(p, b, 1u, CH);
            } else if ((int)n >= p.max_iters) {
              stop_all(ST_NOT_CONVERGED);
            } else if (!(*(volatile unsigned*)&st->status & kStop)) {
              Ls->n = n + 1u;
              Ls->chg = 0u;
              Ls->pend = (unsigned)d->NR;
              enqueue_lattice(p, b, 0u, CH);
            }
          }
        }
      }
    }
    return;
  }

  // ---- the DO(step) / DO(iteration) loops of the §4 procedure, every lattice
  // of the launch in lockstep: one grid-wide synchronize per iteration, after
  // which each region reads its own lattice's "no difference" flag and either
  // iterates again or commits and starts its next window
  unsigned giter = 0;
  for (;;) {
    const unsigned fslot = giter % 3u;
    ++giter;
    Acc acc = {0u, 0u, 0u, 0u, 0u, 0u, false, false};
    const long long c0 = clock64();
    // regions of this slot in this iteration: its own (static schedule), or
    // consecutive regions claimed a warp at a time from a shared counter, so
    // that slots whose regions are idle take work from busy lattices
    int r_dyn = -1;
    const unsigned wlb = (giter - 1u) & 1u;          // this iteration's work list
    const unsigned wln = DYN ? *(volatile unsigned*)&st->wl_count[wlb] : 0u;
    auto next_region = [&](int r) -> int {
      if constexpr (!DYN) {
        return r < 0 ? sfirst : r + sstride;
      } else {
        const int per_warp = LANES ? p.lanes : 1;
        unsigned base = 0u;
        if ((threadIdx.x & 31) == 0) base = atomicAdd(&st->work, (unsigned)per_warp);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (base >= wln) return INT_MAX;
        const unsigned cand = base + (LANES ? (unsigned)lane : 0u);
        return (is_slot && (!LANES || lane < p.lanes) && cand < wln)
                   ? (int)__ldcg(&p.wl[(size_t)wlb * p.NR + cand]) : -2;
      }
    };
    for (int r = next_region(r_dyn); r != INT_MAX && (DYN || r < p.NR); r = next_region(r)) {
      if (r < 0 || r >= p.NR) continue;     // dynamic: no region for this lane in this round
      const int b = (int)__ldg(&p.rrep[r]);
      const RepDesc* d = p.reps + b;
      if (p.rwin[r] >= (unsigned)d->nwin) continue;
      const Lat lt = lat_of(p, r);
      const double t_s = p.rts[r];
      const double t_end = __dadd_rn(t_s, d->Tw);
      const unsigned cidx = p.rcidx[r];
      const int n = (int)p.rn[r];
      Acc ra = {0u, 0u, 0u, 0u, 0u, 0u, false, false};
      const unsigned wg = d->w0 + p.rwin[r];
      if (MODE == 0)
        run_region<0>(p, lt, r, n, cidx, t_s, t_end, wg, g, ra);
      else if (MODE == 2)
        run_region<1>(p, lt, r, n, cidx, t_s, t_end, wg, g, ra);
      else
        run_region_warp(p, lt, r, n, cidx, t_s, t_end, ra);
      if (reporter) {
        RepStats* rs = p.rs + b;
        // f of §6: the most boundary events of a region in an iteration
        if (ra.fmax) atomicMax(&p.curf[(p.rwin[r] & 1u) * p.nrep + b], ra.fmax);
        if (ra.changed) atomicOr(&p.rflags[fslot * p.nrep + b], 1u);
        if (ra.overflow) atomicOr(&st->status, ST_CAPACITY);
        if (ra.events) atomicAdd(&rs->generated, (unsigned long long)ra.events);
        if (ra.breaks) atomicAdd(&rs->breaks, (unsigned long long)ra.breaks);
        if (ra.fmax) atomicMax(&rs->max_f, ra.fmax);
        if (ra.emax) atomicMax(&rs->max_win_events, ra.emax);
        acc.passes += ra.passes;
        acc.skips += ra.skips;
      }
    }
    run_cyc += (unsigned long long)(clock64() - c0);
    if (reporter) {
      if (acc.passes) atomicAdd(&st->region_passes, (unsigned long long)acc.passes);
      if (acc.skips) atomicAdd(&st->region_skips, (unsigned long long)acc.skips);
    }
    if (!grid_barrier(st, p.timeout_cycles)) return;
    if (*(volatile unsigned*)&st->status & (ST_CAPACITY | ST_NOT_CONVERGED)) return;
    if (*(volatile unsigned*)&st->active == 0u) return;     // every lattice is done
    // the flag slot of the next-but-one iteration starts clear
    for (int b = (int)(blockIdx.x * blockDim.x + threadIdx.x); b < p.nrep; b += gridDim.x * blockDim.x)
      p.rflags[((fslot + 2u) % 3u) * p.nrep + b] = 0u;

    // ---- per region: commit or iterate again (statement 3 of §4); with the
    // dynamic schedule, also the work list of the next iteration: regions
    // whose inputs did not change are carried over here instead
    const unsigned wlnext = giter & 1u;
    if (DYN && blockIdx.x == 0 && threadIdx.x == 0) st->wl_count[wlb] = 0u;   // list after next
    if (is_slot && (LANES || (threadIdx.x & 31) == 0)) {
      for (int r = sfirst; r < p.NR; r += sstride) {
        const int b = (int)__ldg(&p.rrep[r]);
        const RepDesc* d = p.reps + b;
        const unsigned w = p.rwin[r];
        bool want = false;
        if (w < (unsigned)d->nwin) {
        RepStats* rs = p.rs + b;
        const unsigned n = p.rn[r];
        if (*(volatile unsigned*)&p.rflags[fslot * p.nrep + b] == 0u) {
          // no region of this lattice changed its lists: its histories are the
          // fixed point; the tentative state becomes the committed one
          const unsigned cnew = p.rcidx[r] ^ 1u;
          const unsigned long long dc = __ldcg(&p.ci[(size_t)cnew * nr + r]) -
                                        __ldcg(&p.ci[(size_t)(cnew ^ 1u) * nr + r]);
          if (dc) atomicAdd(&rs->committed, dc);
          p.rcidx[r] = (uint8_t)cnew;
          const Lat lt = lat_of(p, r);
          compute_halo(p, lt, r, cnew);     // neighbours commit in this same step
          p.rts[r] = __dadd_rn(p.rts[r], d->Tw);
          p.rwin[r] = w + 1u;
          p.rn[r] = 1u;
          p.rfill[r] = (w + 1u < (unsigned)d->nwin) ? 1 : 0;
          if (lt.loc == 0) {
            rs->windows += 1ull;
            rs->iterations += (unsigned long long)n;
            rs->last_iters = n;
            if (n > rs->max_iters_seen) rs->max_iters_seen = n;
            rs->windows_done = w + 1u;
            // f of this window; its parity slot is next written in window w + 2
            const unsigned fw = p.curf[(w & 1u) * p.nrep + b];
            p.curf[(w & 1u) * p.nrep + b] = 0u;
            rs->sum_f += fw;
            if (b == 0) {
              p.win_iters[w % kWinRing] = n;
              p.win_iters[kWinRing + w % kWinRing] = fw;
            }
            if (w + 1u == (unsigned)d->nwin) atomicSub(&st->active, 1u);
          }
          want = w + 1u < (unsigned)d->nwin;      // iteration 1 of its next window
        } else if ((int)n >= p.max_iters) {
          atomicOr(&st->status, ST_NOT_CONVERGED);
        } else {
          p.rn[r] = n + 1u;
          if (DYN) {
            // iteration n + 1 reads the neighbours' lists of iteration n
            const Lat lt = lat_of(p, r);
            const int rx = lt.loc % lt.NX, ry = lt.loc / lt.NX;
            const size_t cp = (size_t)(n & 1u) * nr;
            bool dirty = false;
            if (!lt.spans_y)
              dirty = __ldcg(&p.chg[cp + lt.off + ((ry + lt.NY - 1) % lt.NY) * lt.NX + rx]) ||
                      __ldcg(&p.chg[cp + lt.off + ((ry + 1) % lt.NY) * lt.NX + rx]);
            if (!lt.spans_x)
              dirty = dirty || __ldcg(&p.chg[cp + lt.off + ry * lt.NX + (rx + lt.NX - 1) % lt.NX]) ||
                      __ldcg(&p.chg[cp + lt.off + ry * lt.NX + (rx + 1) % lt.NX]);
            if (dirty) {
              want = true;
            } else {
              carry_lists(p, r, (int)((n + 1u) & 1u), lt.spans_x, lt.spans_y);
              atomicAdd(&st->region_skips, 1ull);
            }
          }
        }
        }
        if (DYN) wl_append(p, wlnext, r, want);
      }
    }
    __syncthreads();
    fill_ring(p);
    if (DYN) {
      // another warp may run any region next: its commit and ring top-up
      // must be complete first
      if (blockIdx.x == 0 && threadIdx.x == 0) st->work = 0u;
      if (!grid_barrier(st, p.timeout_cycles)) return;
    }
  }
}

// ---------------------------------------------------------------- helpers
__global__ void halo_kernel(KParams p) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < p.NR) compute_halo(p, lat_of(p, r), r, p.rcidx[r]);
}

// Rows (copy 0) of every region of lattice `rep` (of every lattice when
// rep < 0) from the lattice's init mode: fair coin / all up / all down.
__global__ void init_rows_kernel(KParams p, int rep) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)p.NR * p.H) return;
  const int r = (int)(t % p.NR), y = (int)(t / p.NR);
  const Lat lt = lat_of(p, r);
  if (rep >= 0 && lt.rep != rep) return;
  const int mode = p.reps[lt.rep].init_mode;
  const int rx = lt.loc % lt.NX, ry = lt.loc / lt.NX;
  uint32_t word = 0;
  if (mode == SR_INIT_ALL_UP) {
    word = (p.W == 32) ? 0xFFFFFFFFu : ((1u << p.W) - 1u);
  } else if (mode == SR_INIT_FAIR_COIN) {
    const uint32_t gy = (uint32_t)(ry * p.H + y);
    for (int x = 0; x < p.W; ++x) {
      const uint32_t site = gy * (uint32_t)lt.L + (uint32_t)(rx * p.W + x);
      uint32_t w[4];
      philox4x32_10(site, 0u, 0u, 1u, lt.key0, lt.key1, w);
      word |= (w[0] & 1u) << x;
    }
  }
  p.rows[(size_t)y * p.NR + r] = word;
}

// Rows (copy 0) of lattice b from an int8 L x L array in device memory.
__global__ void pack_rows_kernel(KParams p, int b, const int8_t* spins) {
  const RepDesc& d = p.reps[b];
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)d.NR * p.H) return;
  const int loc = (int)(t % d.NR), y = (int)(t / d.NR);
  const int r = d.off + loc;
  const int rx = loc % d.NX, ry = loc / d.NX;
  const size_t base = (size_t)(ry * p.H + y) * d.L + (size_t)rx * p.W;
  uint32_t word = 0;
  for (int x = 0; x < p.W; ++x) word |= (uint32_t)(spins[base + x] > 0) << x;
  p.rows[(size_t)y * p.NR + r] = word;
}

// Committed spins of lattice b as an int8 L x L array.
__global__ void unpack_rows_kernel(KParams p, int b, int8_t* spins) {
  const RepDesc& d = p.reps[b];
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)d.L * d.L) return;
  const int gx = (int)(t % d.L), gy = (int)(t / d.L);
  const int r = d.off + (gy / p.H) * d.NX + gx / p.W;
  const uint32_t word = p.rows[((size_t)p.rcidx[r] * p.H + gy % p.H) * p.NR + r];
  spins[t] = ((word >> (gx % p.W)) & 1u) ? 1 : -1;
}

// Clock state at t = 0 of every region of lattice `rep` (every lattice when
// rep < 0): tau_0 = 0, first pair (U_1, V_1), committed copy 0, empty ring.
__global__ void init_carry_kernel(KParams p, int rep) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= p.NR) return;
  const Lat lt = lat_of(p, r);
  if (rep >= 0 && lt.rep != rep) return;
  double x;
  unsigned long long kv;
  draw_event(0ull, (uint32_t)lt.loc, lt.key0, lt.key1, x, kv);
  p.ci[r] = 0ull;
  p.cx[r] = x;
  p.ckv[r] = kv;
  p.cb[r] = 0.0;
  p.ct[r] = 0.0;
  p.cim[r] = 0.0;
  if (p.score)
    for (int k = 0; k < 10; ++k) {
      p.sc[(size_t)k * p.NR + r] = 0ull;
      p.si[(size_t)k * p.NR + r] = 0.0;
    }
  p.cib[r] = 0.0;
  p.rhi[r] = 0ull;    // ring empty
  p.rcidx[r] = 0;
}

// Spin sum and owned-bond sum (right and down bonds of every site) of lattice b, exact.
__global__ void observe_ints_kernel(KParams p, int b, long long* out2) {
  const RepDesc& d = p.reps[b];
  const int loc = blockIdx.x * blockDim.x + threadIdx.x;
  long long mag = 0, bonds = 0;
  if (loc < d.NR) {
    const int r = d.off + loc;
    const size_t nr = (size_t)p.NR;
    const uint32_t wmask = (p.W == 32) ? 0xFFFFFFFFu : ((1u << p.W) - 1u);
    const uint32_t* rows_c = p.rows + (size_t)p.rcidx[r] * p.H * nr;
    const uint32_t hS = p.halo[1 * nr + r], hE = p.halo[3 * nr + r];
    for (int y = 0; y < p.H; ++y) {
      const uint32_t rw = rows_c[(size_t)y * nr + r];
      const uint32_t dn = (y < p.H - 1) ? rows_c[(size_t)(y + 1) * nr + r]
                                        : (d.spans_y ? rows_c[r] : hS);
      const uint32_t rbit = d.spans_x ? (rw & 1u) : (hE >> y) & 1u;
      const uint32_t rt = (rw >> 1) | (rbit << (p.W - 1));
      mag += 2 * __popc(rw) - p.W;
      bonds += (p.W - 2 * __popc((rw ^ rt) & wmask)) + (p.W - 2 * __popc((rw ^ dn) & wmask));
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    mag += __shfl_down_sync(0xFFFFFFFFu, mag, o);
    bonds += __shfl_down_sync(0xFFFFFFFFu, bonds, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd((unsigned long long*)&out2[0], (unsigned long long)mag);
    atomicAdd((unsigned long long*)&out2[1], (unsigned long long)bonds);
  }
}

// Fixed-order FP64 sums of the per-region time integrals of lattice b (one block).
__global__ void observe_integrals_kernel(KParams p, int b, double* out2) {
  __shared__ double sm[2][1024];
  const RepDesc& d = p.reps[b];
  const size_t nr = (size_t)p.NR;
  double a = 0.0, c = 0.0;
  for (int loc = threadIdx.x; loc < d.NR; loc += blockDim.x) {
    const int r = d.off + loc;
    const size_t ci = (size_t)p.rcidx[r];
    a = __dadd_rn(a, p.cim[ci * nr + r]);
    c = __dadd_rn(c, p.cib[ci * nr + r]);
  }
  sm[0][threadIdx.x] = a;
  sm[1][threadIdx.x] = c;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) {
      sm[0][threadIdx.x] = __dadd_rn(sm[0][threadIdx.x], sm[0][threadIdx.x + k]);
      sm[1][threadIdx.x] = __dadd_rn(sm[1][threadIdx.x], sm[1][threadIdx.x + k]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out2[0] = sm[0][0];
    out2[1] = sm[1][0];
  }
}

// Committed clock state of lattice b (per region: index, x, b, t_last), and
// the committed copy of every region's event index.
__global__ void gather_carry_kernel(KParams p, int b, unsigned long long* i_out, double* x_out,
                                    double* b_out, double* t_out) {
  const RepDesc& d = p.reps[b];
  const int loc = blockIdx.x * blockDim.x + threadIdx.x;
  if (loc >= d.NR) return;
  const int r = d.off + loc;
  const size_t c = (size_t)p.rcidx[r] * p.NR + r;
  if (i_out) i_out[loc] = p.ci[c];
  if (x_out) x_out[loc] = p.cx[c];
  if (b_out) b_out[loc] = p.cb[c];
  if (t_out) t_out[loc] = p.ct[c];
}

// ---------------------------------------------------------------- score
// Per lattice b (one block each): the path statistics summed over its regions
// (committed copies) in a fixed order -- C_k exactly, I_k by a fixed
// tree -- then the score dlog L / d(beta, h, J) = sum_k C_k dlog p_k - sum_k dp_k I_k
// with the lattice's tables tab[b] = {dlog p [3][10], dp [3][10]}.
// out[b] = {S[3], C[10] (as doubles), I[10]}.
__global__ void score_kernel(KParams p, const double* tab, double* out) {
  __shared__ double sd[256];
  __shared__ unsigned long long su[256];
  __shared__ double cI[20];
  const int b = blockIdx.x;
  const RepDesc& d = p.reps[b];
  const size_t nr = (size_t)p.NR;
  for (int k = 0; k < 10; ++k) {
    double a = 0.0;
    unsigned long long c = 0ull;
    for (int loc = threadIdx.x; loc < d.NR; loc += blockDim.x) {
      const int r = d.off + loc;
      const size_t o = ((size_t)p.rcidx[r] * 10 + k) * nr + r;
      a = __dadd_rn(a, p.si[o]);
      c += p.sc[o];
    }
    sd[threadIdx.x] = a;
    su[threadIdx.x] = c;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) {
        sd[threadIdx.x] = __dadd_rn(sd[threadIdx.x], sd[threadIdx.x + w]);
        su[threadIdx.x] += su[threadIdx.x + w];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      cI[k] = (double)su[0];
      cI[10 + k] = sd[0];
    }
    __syncthreads();
  }
  if (threadIdx.x < 3) {
    const int q = threadIdx.x;
    const double* dlogp = tab + (size_t)b * 60 + q * 10;
    const double* dp = tab + (size_t)b * 60 + 30 + q * 10;
    double sa = 0.0, sb = 0.0;
    for (int k = 0; k < 10; ++k) {
      sa = __dadd_rn(sa, __dmul_rn(cI[k], dlogp[k]));
      sb = __dadd_rn(sb, __dmul_rn(dp[k], cI[10 + k]));
    }
    out[(size_t)b * 23 + q] = __dsub_rn(sa, sb);
  }
  if (threadIdx.x < 20) out[(size_t)b * 23 + 3 + threadIdx.x] = cI[threadIdx.x];
}

// Column sums of A [n][m] in a fixed order (one block per column).
__global__ void colsum_kernel(int n, int m, const double* A, double* sums) {
  __shared__ double sd[256];
  const int j = blockIdx.x;
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a = __dadd_rn(a, A[(size_t)i * m + j]);
  sd[threadIdx.x] = a;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sd[threadIdx.x] = __dadd_rn(sd[threadIdx.x], sd[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[j] = sd[0];
}

// The backward of time averages A [n][m] through the score: for replica i and
// parameter q, G[i][q] = sum_j gA[i][j] ((A[i][j] - base_ij) S[i][q] + E[i][j][q]),
// base_ij the mean of column j over the other replicas (0 when n = 1).
__global__ void score_grad_kernel(int n, int m, int nq, const double* A, const double* gA,
                                  const double* S, const double* E, const double* sums, double* G) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * nq) return;
  const int i = t / nq, q = t % nq;
  double g = 0.0;
  for (int j = 0; j < m; ++j) {
    const double a = A[(size_t)i * m + j];
    const double base = n > 1 ? __ddiv_rn(__dsub_rn(sums[j], a), (double)(n - 1)) : 0.0;
    double term = __dmul_rn(__dsub_rn(a, base), S[(size_t)i * nq + q]);
    if (E) term = __dadd_rn(term, E[((size_t)i * m + j) * nq + q]);
    g = __dadd_rn(g, __dmul_rn(gA[(size_t)i * m + j], term));
  }
  G[t] = g;
}

__global__ void eval_draws_kernel(uint32_t key0, uint32_t key1, uint32_t region,
                                  unsigned long long i0, size_t n, double* x,
                                  unsigned long long* kv) {
  const size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double xx;
  unsigned long long k;
  draw_event(i0 + j, region, key0, key1, xx, k);
  x[j] = xx;
  kv[j] = k;
}

__global__ void eval_softfloat_kernel(int op, const double* a, const double* b, double* out,
                                      size_t n) {
  const size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double x = a[j], y = b[j];
  double r;
  switch (op) {
    case 0: r = sf::add_pos(x, y); break;
    case 1: r = sf::sub_pos(x, y); break;
    case 2: r = sf::mul_pos(x, y); break;
    case 3: r = sf::div_pos(x, y); break;
    default: r = sf::u64_scaled((unsigned long long)__double_as_longlong(x), (int)y); break;
  }
  out[j] = r;
}

}  // namespace sr

// ====================================================================== C ABI
using namespace sr;

struct sr_ctx {
  sr_params prm;                // common settings (the region shape, capacities, launch)
  int nrep;                     // lattices
  sr_replica* reps;             // [nrep] their parameters
  RepDesc* hdesc;               // [nrep] host copy of the descriptors
  double* t_c;                  // [nrep] committed time of each lattice
  unsigned* wins;               // [nrep] committed windows of each lattice
  int NR, F, Lmax;
  double scale;
  cudaStream_t stream;
  bool own_stream;
  int num_sms;
  int clock_khz;
  // device state
  RepDesc* desc;
  RepStats* rs;
  uint32_t *rrep, *rflags;
  uint8_t *rcidx, *rfill;
  uint32_t* wl;                 // [2][NR] work lists of the dynamic schedule
  LatState* ls;                 // asynchronous schedule: per-lattice progress
  unsigned long long* q;        // asynchronous schedule: task queue
  unsigned long long qcap;
  unsigned long long async_tail;  // tasks published before the launch (asynchronous schedule)
  unsigned async_active;
  uint32_t *rn, *rwin;
  double* rts;
  uint32_t *rows, *halo, *hl, *trs, *win_iters, *log, *loghdr, *curf;
  uint8_t* chg;
  int CB;
  unsigned long long *ci, *ckv, *rkv, *rhi;
  double* rx;
  int K, Kcap;
  double *cx, *cb, *ct, *cim, *cib, *ht, *trt;
  unsigned long long* sc;       // score statistics (score mode)
  double* si;
  double* score_tab;            // [nrep][2][3][10] dlog p and dp per lattice (score mode)
  double* score_out;            // [nrep][3 + 20] scores and lattice statistics
  uint8_t* hp;
  int cap;
  bool cap_auto;
  DevStats* st;
  DevStats* h_st;
  RepStats* h_rs;
  long long* obs_i;
  double* obs_f;
  long long* h_obs_i;
  double* h_obs_f;
  int8_t* stage;
  int rl, tpb, blocks, mode, lanes;
  int dynamic;                  // dynamic region schedule
  size_t smem;
  int last_nwin;
  unsigned long long launches;   // kernels launched by this context
};

namespace {

constexpr int kMaxCap = 1 << 15;   // list cursors hold lengths in 16 bits

int bitlen(long long v) {
  int b = 0;
  while ((v >> b) > 0) ++b;
  return b;
}

// p_k for the ten classes k = 5*[s=+1] + n_up (Eqs. 2.2-2.3), then the
// fixed-point grid P_k = round(p_k 2^F), F = 63 - bitlen(sites per region).
void rate_table(const sr_replica& p, int F, unsigned long long P[10]) {
  for (int k = 0; k < 10; ++k) {
    const int s = (k >= 5) ? 1 : -1;
    const int n_up = k % 5;
    const int nb_sum = 2 * n_up - 4;
    const double dE = 2.0 * (double)s * (p.J * (double)nb_sum + p.h);
    const double theta = std::exp(-dE / p.T);
    double pk;
    if (p.rates == SR_RATES_GLAUBER)
      pk = theta / (1.0 + theta);
    else
      pk = theta < 1.0 ? theta : 1.0;
    P[k] = (unsigned long long)std::nearbyint(std::ldexp(pk, F));
  }
}

// d log p_k and d p_k with respect to (beta, h, J), beta = 1/T, for the ten
// classes (Eqs. 2.1-2.3): a class-k flip changes the energy by
// dE = 2 s (J (2 n_up - 4) + h), so d(beta dE) = (dE, 2 beta s, 2 beta s nb).
// Metropolis, p = min(1, exp(-beta dE)): d log p = -d(beta dE) where dE > 0,
// 0 where p = 1.  Glauber, p = e / (1 + e) with e = exp(-beta dE):
// d log p = -(1 - p) d(beta dE).  tab = {dlog p [3][10], dp [3][10]}.
void score_tables(const sr_replica& p, double* tab) {
  const double beta = 1.0 / p.T;
  for (int k = 0; k < 10; ++k) {
    const double s = (k >= 5) ? 1.0 : -1.0;
    const double nb = 2.0 * (double)(k % 5) - 4.0;
    const double dE = 2.0 * s * (p.J * nb + p.h);
    const double e = std::exp(-dE / p.T);
    const double pk = p.rates == SR_RATES_GLAUBER ? e / (1.0 + e) : (e < 1.0 ? e : 1.0);
    const double dx[3] = {dE, 2.0 * beta * s, 2.0 * beta * s * nb};
    for (int q = 0; q < 3; ++q) {
      double dl;
      if (p.rates == SR_RATES_GLAUBER)
        dl = -(1.0 - pk) * dx[q];
      else
        dl = dE > 0.0 ? -dx[q] : 0.0;
      tab[q * 10 + k] = dl;
      tab[30 + q * 10 + k] = pk * dl;
    }
  }
}

KParams make_params(const sr_ctx* c) {
  KParams k;
  std::memset(&k, 0, sizeof k);
  k.W = c->prm.region_w;
  k.H = c->prm.region_h;
  k.NR = c->NR;
  k.nrep = c->nrep;
  k.reps = c->desc;
  k.rrep = c->rrep;
  k.rs = c->rs;
  k.rflags = c->rflags;
  k.rcidx = c->rcidx;
  k.rn = c->rn;
  k.rwin = c->rwin;
  k.rts = c->rts;
  k.rfill = c->rfill;
  k.wl = c->wl;
  k.ls = c->ls;
  k.q = c->q;
  k.qcap = c->qcap;
  k.scale = c->scale;
  k.F = c->F;
  k.rows = c->rows;
  k.halo = c->halo;
  k.ci = c->ci;
  k.cx = c->cx;
  k.ckv = c->ckv;
  k.cb = c->cb;
  k.ct = c->ct;
  k.cim = c->cim;
  k.sc = c->sc;
  k.si = c->si;
  k.score = c->prm.score ? 1 : 0;
  k.cib = c->cib;
  k.ht = c->ht;
  k.hp = c->hp;
  k.hl = c->hl;
  k.chg = c->chg;
  k.cap = c->cap;
  k.trt = c->trt;
  k.trs = c->trs;
  k.tcap = c->prm.trace_capacity;
  k.log = c->log;
  k.loghdr = c->loghdr;
  k.CB = c->CB;
  k.rx = c->rx;
  k.rkv = c->rkv;
  k.rhi = c->rhi;
  k.K = c->K;
  k.rl = c->rl;
  k.lanes = c->lanes;
  k.st = c->st;
  k.win_iters = c->win_iters;
  k.fresh = c->prm.fresh_steps ? 1 : 0;
  k.curf = c->curf;
  k.max_iters = c->prm.max_iters;
  k.timeout_cycles = (long long)c->prm.barrier_timeout_ms * (long long)c->clock_khz;
  k.skip_block = c->prm.test_barrier_skip_block;
  return k;
}

template <class T>
int dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc((void**)p, count * sizeof(T)) == cudaSuccess ? SR_OK : SR_ENOMEM;
}

int alloc_history(sr_ctx* c, int cap) {
  if (c->ht) cudaFree(c->ht);
  if (c->hp) cudaFree(c->hp);
  c->ht = nullptr;
  c->hp = nullptr;
  const size_t n = (size_t)2 * 4 * (size_t)cap * (size_t)c->NR;
  if (dalloc(&c->ht, n) || dalloc(&c->hp, n)) return SR_ENOMEM;
  c->cap = cap;
  return SR_OK;
}

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? SR_OK : SR_ECUDA; }

// The kernel instance of a mapping (0 lane/FP64, 1 warp, 2 lane/integer time)
// and schedule (static or dynamic).
const void* relax_fn(int mode, int dynamic) {
  if (dynamic == 2)
    return mode == 2 ? (const void*)relax_kernel<2, 2> : (const void*)relax_kernel<0, 2>;
  if (dynamic)
    return mode == 1 ? (const void*)relax_kernel<1, 1>
                     : (mode == 2 ? (const void*)relax_kernel<2, 1> : (const void*)relax_kernel<0, 1>);
  return mode == 1 ? (const void*)relax_kernel<1, 0>
                   : (mode == 2 ? (const void*)relax_kernel<2, 0> : (const void*)relax_kernel<0, 0>);
}

// Shared memory of a lane-mapping block: per region slot, H spin rows, ten
// class-by-row count groups of ceil(H/4) words, the rate table (20 words of
// 8 bytes) and, in score mode, 30 more 8-byte words of path statistics.
size_t lane_smem_bytes(int H, int slots, bool score) {
  const size_t words = ((size_t)(H + 10 * ((H + 3) / 4)) * (size_t)slots + 1) & ~(size_t)1;
  return (words + (score ? 100 : 40) * (size_t)slots) * sizeof(uint32_t);
}

// Allow a kernel `bytes` of dynamic shared memory (beyond the default 48 KB,
// which also counts the kernel's static shared memory, an opt-in is needed).
bool allow_smem(const void* fn, size_t bytes) {
  if (bytes <= 32 * 1024) return true;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess;
}

int upload_desc(sr_ctx* c) {
  return cuda_rc(cudaMemcpyAsync(c->desc, c->hdesc, (size_t)c->nrep * sizeof(RepDesc),
                                 cudaMemcpyHostToDevice, c->stream));
}

// Initial state of lattice `rep` (every lattice when rep < 0): rows (copy 0)
// from dev_spins (one lattice) or the lattice's init mode, clocks at t = 0,
// counters cleared; then the halos of every region.
int init_state(sr_ctx* c, int rep, const int8_t* dev_spins) {
  KParams k = make_params(c);
  int rc = upload_desc(c);
  if (rc != SR_OK) return rc;
  const unsigned gr = (unsigned)((c->NR + 255) / 256);
  init_carry_kernel<<<gr, 256, 0, c->stream>>>(k, rep);
  if (dev_spins) {
    const RepDesc& d = c->hdesc[rep];
    pack_rows_kernel<<<(unsigned)(((size_t)d.NR * k.H + 255) / 256), 256, 0, c->stream>>>(k, rep,
                                                                                          dev_spins);
  } else {
    init_rows_kernel<<<(unsigned)(((size_t)c->NR * k.H + 255) / 256), 256, 0, c->stream>>>(k, rep);
  }
  halo_kernel<<<gr, 256, 0, c->stream>>>(k);
  c->launches += 3;
  for (int b = 0; b < c->nrep; ++b) {
    if (rep >= 0 && b != rep) continue;
    if (cudaMemsetAsync(c->rs + b, 0, sizeof(RepStats), c->stream) != cudaSuccess) return SR_ECUDA;
    c->t_c[b] = 0.0;
    c->wins[b] = 0u;
  }
  if (rep < 0 && cudaMemsetAsync(c->st, 0, sizeof(DevStats), c->stream) != cudaSuccess) return SR_ECUDA;
  c->last_nwin = 0;
  return cuda_rc(cudaGetLastError());
}

// One persistent launch running, for each lattice b, nwin[b] windows of
// length Tw[b] from its committed time.
int launch_relax(sr_ctx* c, const double* Tw, const int* nwin) {
  for (int b = 0; b < c->nrep; ++b) {
    c->hdesc[b].t0 = c->t_c[b];
    c->hdesc[b].Tw = Tw[b];
    c->hdesc[b].nwin = nwin[b];
    c->hdesc[b].w0 = c->wins[b];
  }
  int rc = upload_desc(c);
  if (rc != SR_OK) return rc;
  KParams k = make_params(c);
  if (c->dynamic == 2) {
    // per-lattice progress and the first pass tasks of every lattice with windows
    LatState* hls = (LatState*)std::calloc((size_t)c->nrep, sizeof(LatState));
    unsigned long long total = 0ull;
    unsigned active = 0u;
    for (int b = 0; b < c->nrep; ++b)
      if (nwin[b] > 0) {
        total += (unsigned long long)((c->hdesc[b].NR + c->lanes - 1) / c->lanes);
        ++active;
      }
    unsigned long long* items = (unsigned long long*)std::malloc((size_t)(total + 1) * 8);
    if (!hls || !items) {
      std::free(hls);
      std::free(items);
      return SR_ENOMEM;
    }
    unsigned long long t = 0ull;
    for (int b = 0; b < c->nrep; ++b) {
      hls[b].pend = (unsigned)c->hdesc[b].NR;
      hls[b].n = 1u;
      hls[b].ts = c->t_c[b];
      if (nwin[b] <= 0) continue;
      const int nch = (c->hdesc[b].NR + c->lanes - 1) / c->lanes;
      for (int ch = 0; ch < nch; ++ch)
        items[t++] = kTaskValid | ((unsigned long long)b << 32) | (unsigned long long)ch;
    }
    int rca = cuda_rc(cudaMemcpyAsync(c->ls, hls, (size_t)c->nrep * sizeof(LatState),
                                      cudaMemcpyHostToDevice, c->stream));
    if (rca == SR_OK)
      rca = cuda_rc(cudaMemsetAsync(c->q, 0, (size_t)c->qcap * 8, c->stream));
    if (rca == SR_OK && total)
      rca = cuda_rc(cudaMemcpyAsync(c->q, items, (size_t)total * 8, cudaMemcpyHostToDevice, c->stream));
    if (rca == SR_OK) rca = cuda_rc(cudaStreamSynchronize(c->stream));
    std::free(hls);
    std::free(items);
    if (rca != SR_OK) return rca;
    c->async_tail = total;
    c->async_active = active;
  }
  if (cudaMemsetAsync(c->st, 0, offsetof(DevStats, region_passes), c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->rflags, 0, 3 * (size_t)c->nrep * sizeof(uint32_t), c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->curf, 0, 2 * (size_t)c->nrep * sizeof(uint32_t), c->stream) != cudaSuccess)
    return SR_ECUDA;
  if (c->dynamic == 2) {
    if (cudaMemcpyAsync((char*)c->st + offsetof(DevStats, qtail), &c->async_tail, 8,
                        cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync((char*)c->st + offsetof(DevStats, active), &c->async_active, 4,
                        cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      return SR_ECUDA;
  }
  void* args[] = {&k};
  const void* fn = relax_fn(c->mode, c->dynamic);
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(c->blocks), dim3(c->tpb), args, c->smem,
                                              c->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();   // a refused launch leaves no error behind for later calls
    return SR_ECUDA;
  }
  c->launches += 1;
  if (cudaMemcpyAsync(c->h_st, c->st, sizeof(DevStats), cudaMemcpyDeviceToHost, c->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(c->h_rs, c->rs, (size_t)c->nrep * sizeof(RepStats), cudaMemcpyDeviceToHost,
                      c->stream) != cudaSuccess)
    return SR_ECUDA;
  return cuda_rc(cudaStreamSynchronize(c->stream));
}

// Ring length for windows of length Tw: at most sites * Tw events are expected
// per region (every p_k <= 1), with a margin; events past the ring are drawn on
// the fly, so the cap only bounds memory.
int ring_length(const sr_ctx* c, double Tw) {
  const double want = 1.25 * (double)c->prm.region_w * c->prm.region_h * Tw + 16.0;
  int K = 16;
  while (K < want && K < 4096) K *= 2;
  return K;
}

int set_ring(sr_ctx* c, int K) {
  if (K == c->K) return SR_OK;
  if (K > c->Kcap) {
    if (c->rx) cudaFree(c->rx);
    if (c->rkv) cudaFree(c->rkv);
    c->rx = nullptr;
    c->rkv = nullptr;
    c->Kcap = 0;
    c->K = 0;
    const size_t n = (size_t)K * c->NR;
    if (dalloc(&c->rx, n) || dalloc(&c->rkv, n)) return SR_ENOMEM;
    c->Kcap = K;
  }
  c->K = K;
  // slots are indexed modulo K: a new K invalidates every ring
  return cuda_rc(cudaMemsetAsync(c->rhi, 0, (size_t)c->NR * sizeof(unsigned long long), c->stream));
}

void free_all(sr_ctx* c) {
  void* dev[] = {c->sc, c->si, c->score_tab, c->score_out,
                 c->rows, c->halo, c->hl, c->trs, c->win_iters, c->curf, c->ci, c->ckv, c->cx, c->cb,
                 c->ct, c->cim, c->cib, c->ht, c->trt, c->hp, c->st, c->obs_i, c->obs_f, c->stage,
                 c->rx, c->rkv, c->rhi, c->chg, c->log, c->loghdr, c->desc, c->rs, c->rrep,
                 c->rflags, c->rcidx, c->rfill, c->rn, c->rwin, c->rts, c->wl, c->ls, c->q};
  for (void* d : dev)
    if (d) cudaFree(d);
  if (c->h_st) cudaFreeHost(c->h_st);
  if (c->h_rs) cudaFreeHost(c->h_rs);
  if (c->h_obs_i) cudaFreeHost(c->h_obs_i);
  if (c->h_obs_f) cudaFreeHost(c->h_obs_f);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  std::free(c->reps);
  std::free(c->hdesc);
  std::free(c->t_c);
  std::free(c->wins);
}

int check_replica(const sr_replica& r, int W, int H) {
  if (r.L < 3 || r.L % W || r.L % H) return SR_EINVAL;
  if (!(r.T > 0.0) || !std::isfinite(r.J) || !std::isfinite(r.h) || std::isnan(r.T)) return SR_EINVAL;
  if (r.init_mode < SR_INIT_FAIR_COIN || r.init_mode > SR_INIT_ALL_DOWN) return SR_EINVAL;
  if (r.rates != SR_RATES_METROPOLIS && r.rates != SR_RATES_GLAUBER) return SR_EINVAL;
  if ((long long)r.L * r.L > (1ll << 32)) return SR_EUNSUPPORTED;
  return SR_OK;
}

// A context for n lattices sharing the region shape and settings of `p`.
int create_common(sr_ctx** out, const sr_replica* reps, int n, const sr_params& p) {
  *out = nullptr;
  if (n < 1 || !reps) return SR_EINVAL;
  if (p.region_w < 1 || p.region_h < 1) return SR_EINVAL;
  if (p.capacity < 0 || p.max_iters < 0 || p.trace_capacity < 0 || p.threads_per_block < 0 ||
      p.blocks < 0 || p.barrier_timeout_ms < 0)
    return SR_EINVAL;
  if (p.lanes_per_region != 0 && p.lanes_per_region != 1 && p.lanes_per_region != 32) return SR_EINVAL;
  if (p.lanes_per_warp < 0 || p.lanes_per_warp > 32 || p.time_arith < 0 || p.time_arith > 2)
    return SR_EINVAL;
  if (p.fresh_steps != 0 && p.fresh_steps != 1) return SR_EINVAL;
  if (p.fresh_steps && p.lanes_per_region == 32) return SR_EUNSUPPORTED;
  if (p.score != 0 && p.score != 1) return SR_EINVAL;
  if (p.schedule < 0 || p.schedule > 3) return SR_EINVAL;
  if (p.schedule == 3 && p.lanes_per_region == 32) return SR_EUNSUPPORTED;
  if (p.score && p.lanes_per_region == 32) return SR_EUNSUPPORTED;
  if (p.region_w > 32 || p.region_h > 32) return SR_EUNSUPPORTED;
  for (int b = 0; b < n; ++b) {
    const int rc = check_replica(reps[b], p.region_w, p.region_h);
    if (rc != SR_OK) return rc;
  }
  sr_ctx* c = (sr_ctx*)std::calloc(1, sizeof(sr_ctx));
  if (!c) return SR_ENOMEM;
  c->prm = p;
  if (c->prm.max_iters == 0) c->prm.max_iters = 1 << 16;
  if (c->prm.barrier_timeout_ms == 0) c->prm.barrier_timeout_ms = 2000;
  c->nrep = n;
  c->reps = (sr_replica*)std::calloc((size_t)n, sizeof(sr_replica));
  c->hdesc = (RepDesc*)std::calloc((size_t)n, sizeof(RepDesc));
  c->t_c = (double*)std::calloc((size_t)n, sizeof(double));
  c->wins = (unsigned*)std::calloc((size_t)n, sizeof(unsigned));
  if (!c->reps || !c->hdesc || !c->t_c || !c->wins) {
    free_all(c);
    std::free(c);
    return SR_ENOMEM;
  }
  const int W = p.region_w, H = p.region_h;
  c->F = 63 - bitlen((long long)W * H);
  c->scale = std::ldexp(1.0, -c->F);
  long long total = 0;
  for (int b = 0; b < n; ++b) {
    c->reps[b] = reps[b];
    RepDesc& d = c->hdesc[b];
    d.L = reps[b].L;
    d.NX = d.L / W;
    d.NY = d.L / H;
    d.NR = d.NX * d.NY;
    d.off = (int)total;
    d.spans_x = d.NX == 1;
    d.spans_y = d.NY == 1;
    d.key0 = (uint32_t)reps[b].seed;
    d.key1 = (uint32_t)(reps[b].seed >> 32);
    d.init_mode = reps[b].init_mode;
    rate_table(reps[b], c->F, d.P);
    for (int k = 0; k < 10; ++k) d.Rp[k] = d.P[k] ? ~0ull / d.P[k] : 0ull;
    total += d.NR;
    if (d.L > c->Lmax) c->Lmax = d.L;
  }
  if (total > (1ll << 30)) {
    free_all(c);
    std::free(c);
    return SR_EUNSUPPORTED;
  }
  c->NR = (int)total;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->clock_khz, cudaDevAttrClockRate, dev) != cudaSuccess) {
    free_all(c);
    std::free(c);
    return SR_ECUDA;
  }
  if (p.stream) {
    c->stream = (cudaStream_t)p.stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      free_all(c);
      std::free(c);
      return SR_ECUDA;
    }
    c->own_stream = true;
  }

  // launch shape: one warp per region on request; otherwise one lane per
  // region, with few region lanes per warp when the regions are few (less
  // divergence, more warps to hide latency), and FP64 time arithmetic while the
  // FP64 pipe is not the limit
  if (p.lanes_per_region == 32) {
    c->mode = 1;
    int wpb = p.threads_per_block ? p.threads_per_block : 4;   // warps per block
    if (wpb > 4) wpb = 4;                                     // the kernel's block limit
    c->lanes = 1;
    c->rl = wpb;
    c->tpb = 32 * wpb;
    c->smem = 0;
  } else {
    int lanes = p.lanes_per_warp;
    if (lanes == 0) {
      lanes = (c->NR + 16 * c->num_sms - 1) / (16 * c->num_sms);  // about 16 warps per SM
      if (lanes < 1) lanes = 1;
      if (lanes > 32) lanes = 32;
    }
    // FP64 unless asked: measured faster than the emulation at every lane count
    const int soft = p.time_arith == 2;
    c->mode = soft ? 2 : 0;
    c->lanes = lanes;
    int wpb = p.threads_per_block ? (p.threads_per_block + lanes - 1) / lanes : 0;
    if (wpb == 0) {
      const int warps = (c->NR + lanes - 1) / lanes;
      const int per_sm = (warps + c->num_sms - 1) / c->num_sms;
      wpb = per_sm < 4 ? per_sm : 4;
      if (wpb < 1) wpb = 1;
    }
    if (wpb > SR_LANE_MAX_THREADS / 32) wpb = SR_LANE_MAX_THREADS / 32;
    c->rl = wpb * lanes;
    c->tpb = 32 * wpb;
    c->smem = lane_smem_bytes(H, c->rl, p.score != 0);
  }
  {
    const void* fn = relax_fn(c->mode, 0);
    cudaFuncAttributes fa;
    int per_sm_blocks = 0;
    if (!allow_smem(fn, c->smem) || cudaFuncGetAttributes(&fa, fn) != cudaSuccess ||
        c->tpb > fa.maxThreadsPerBlock ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_blocks, fn, c->tpb, c->smem) != cudaSuccess ||
        per_sm_blocks < 1) {
      cudaGetLastError();
      free_all(c);
      std::free(c);
      return SR_EUNSUPPORTED;
    }
    int blocks = p.blocks ? p.blocks : (c->NR + c->rl - 1) / c->rl;
    if (blocks > per_sm_blocks * c->num_sms) blocks = per_sm_blocks * c->num_sms;
    c->blocks = blocks;
    // dynamic schedule when regions outnumber the slots or several lattices
    // share the launch
    // automatic: batches in the lane mapping run asynchronously (measured
    // 19-28% faster than the dynamic lockstep); the warp mapping and single
    // lattices with more regions than slots use the dynamic lockstep
    c->dynamic = p.schedule == 3 ? 2
                 : (p.schedule == 0 && n > 1 && c->mode != 1)
                       ? 2
                       : (p.schedule == 2 ||
                          (p.schedule == 0 && (n > 1 || (long long)c->NR > (long long)blocks * c->rl)))
                             ? 1 : 0;
    if (c->dynamic) {
      // the dynamic instance: same launch bounds; check it fits the same grid
      const void* fd = relax_fn(c->mode, c->dynamic);
      int bd = 0;
      if (!allow_smem(fd, c->smem) ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bd, fd, c->tpb, c->smem) != cudaSuccess ||
          bd * c->num_sms < c->blocks) {
        cudaGetLastError();
        free_all(c);
        std::free(c);
        return SR_EUNSUPPORTED;
      }
    }
  }

  int rc = SR_OK;
  const size_t nr = (size_t)c->NR;
  rc |= dalloc(&c->rows, 2 * (size_t)H * nr);
  rc |= dalloc(&c->halo, 4 * nr);
  rc |= dalloc(&c->ci, 2 * nr);
  rc |= dalloc(&c->cx, 2 * nr);
  rc |= dalloc(&c->ckv, 2 * nr);
  rc |= dalloc(&c->cb, 2 * nr);
  rc |= dalloc(&c->ct, 2 * nr);
  rc |= dalloc(&c->cim, 2 * nr);
  if (p.score) {
    rc |= dalloc(&c->sc, 2 * 10 * nr);
    rc |= dalloc(&c->si, 2 * 10 * nr);
    rc |= dalloc(&c->score_tab, (size_t)n * 60);
    rc |= dalloc(&c->score_out, (size_t)n * 23);
  }
  rc |= dalloc(&c->cib, 2 * nr);
  rc |= dalloc(&c->hl, 2 * 4 * nr);
  rc |= dalloc(&c->st, 1);
  rc |= dalloc(&c->win_iters, 2 * (size_t)kWinRing);
  rc |= dalloc(&c->curf, 2 * (size_t)n);
  rc |= dalloc(&c->obs_i, 2);
  rc |= dalloc(&c->obs_f, 2);
  rc |= dalloc(&c->stage, (size_t)c->Lmax * c->Lmax);
  rc |= dalloc(&c->rhi, nr);
  rc |= dalloc(&c->chg, 2 * nr);
  rc |= dalloc(&c->desc, (size_t)n);
  rc |= dalloc(&c->rs, (size_t)n);
  rc |= dalloc(&c->rflags, 3 * (size_t)n);
  rc |= dalloc(&c->rrep, nr);
  rc |= dalloc(&c->rcidx, nr);
  rc |= dalloc(&c->rfill, nr);
  rc |= dalloc(&c->wl, 2 * nr);
  if (c->dynamic == 2) {
    // at most one task set per lattice is in the queue, plus one claimed slot per warp
    unsigned long long chunks = 0ull;
    for (int b = 0; b < n; ++b)
      chunks += (unsigned long long)((c->hdesc[b].NR + c->lanes - 1) / c->lanes);
    c->qcap = chunks + (unsigned long long)c->blocks * (unsigned long long)(c->tpb / 32) + 64ull;
    rc |= dalloc(&c->ls, (size_t)n);
    rc |= dalloc(&c->q, (size_t)c->qcap);
  }
  rc |= dalloc(&c->rn, nr);
  rc |= dalloc(&c->rwin, nr);
  rc |= dalloc(&c->rts, nr);
  // incremental replay log: lane mappings only
  // (score mode keeps no checkpoints: a resumed pass would need the statistics
  // accumulated before its checkpoint)
  c->CB = (c->mode == 1 || p.replay_records < 0 || p.score) ? 0
                                                           : (p.replay_records ? p.replay_records : 64);
  if (c->CB > 0) {
    rc |= dalloc(&c->log, nr * (size_t)c->CB * (size_t)(kRecHead + H));
    rc |= dalloc(&c->loghdr, nr * 4);
  }
  if (p.trace_capacity > 0) {
    rc |= dalloc(&c->trt, nr * (size_t)p.trace_capacity);
    rc |= dalloc(&c->trs, nr * (size_t)p.trace_capacity);
  }
  c->cap_auto = p.capacity == 0;
  if (rc == SR_OK) rc = alloc_history(c, p.capacity ? p.capacity : 64);
  if (rc == SR_OK &&
      (cudaMallocHost((void**)&c->h_st, sizeof(DevStats)) != cudaSuccess ||
       cudaMallocHost((void**)&c->h_rs, (size_t)n * sizeof(RepStats)) != cudaSuccess ||
       cudaMallocHost((void**)&c->h_obs_i, 2 * sizeof(long long)) != cudaSuccess ||
       cudaMallocHost((void**)&c->h_obs_f, 2 * sizeof(double)) != cudaSuccess))
    rc = SR_ENOMEM;
  if (rc == SR_OK) {
    uint32_t* map = (uint32_t*)std::malloc(nr * sizeof(uint32_t));
    if (!map) {
      rc = SR_ENOMEM;
    } else {
      for (int b = 0; b < n; ++b)
        for (int j = 0; j < c->hdesc[b].NR; ++j) map[c->hdesc[b].off + j] = (uint32_t)b;
      rc = cuda_rc(cudaMemcpyAsync(c->rrep, map, nr * sizeof(uint32_t), cudaMemcpyHostToDevice,
                                   c->stream));
      if (rc == SR_OK) rc = cuda_rc(cudaStreamSynchronize(c->stream));
      std::free(map);
    }
  }
  if (rc == SR_OK && cudaMemsetAsync(c->hl, 0, 2 * 4 * nr * sizeof(uint32_t), c->stream) != cudaSuccess)
    rc = SR_ECUDA;
  if (rc == SR_OK && p.score) {
    double* tab = (double*)std::malloc((size_t)n * 60 * sizeof(double));
    if (!tab) {
      rc = SR_ENOMEM;
    } else {
      for (int b = 0; b < n; ++b) score_tables(reps[b], tab + (size_t)b * 60);
      rc = cuda_rc(cudaMemcpyAsync(c->score_tab, tab, (size_t)n * 60 * sizeof(double),
                                   cudaMemcpyHostToDevice, c->stream));
      if (rc == SR_OK) rc = cuda_rc(cudaStreamSynchronize(c->stream));
      std::free(tab);
    }
  }
  if (rc == SR_OK) rc = init_state(c, -1, nullptr);
  if (rc == SR_OK) rc = cuda_rc(cudaStreamSynchronize(c->stream));
  if (rc != SR_OK) {
    free_all(c);
    std::free(c);
    return rc == SR_ENOMEM ? SR_ENOMEM : (rc < 0 ? rc : SR_ECUDA);
  }
  *out = c;
  return SR_OK;
}

// Run nwin[b] windows of length Tw[b] for every lattice b from its committed
// time; capacity overflows grow the history and re-run what did not commit.
int run_all(sr_ctx* c, const double* Tw, const int* nwin) {
  for (int b = 0; b < c->nrep; ++b)
    if (nwin[b] < 0 || (nwin[b] > 0 && (!(Tw[b] > 0.0) || !std::isfinite(Tw[b])))) return SR_EINVAL;
  double twmax = 0.0;
  for (int b = 0; b < c->nrep; ++b)
    if (nwin[b] > 0 && Tw[b] > twmax) twmax = Tw[b];
  int rc = set_ring(c, ring_length(c, twmax));
  if (rc != SR_OK) return rc;
  int* left = (int*)std::malloc((size_t)c->nrep * sizeof(int));
  if (!left) return SR_ENOMEM;
  int total_left = 0;
  for (int b = 0; b < c->nrep; ++b) {
    left[b] = nwin[b];
    total_left += nwin[b];
  }
  c->last_nwin = 0;
  rc = SR_OK;
  while (total_left > 0) {
    rc = launch_relax(c, Tw, left);
    if (rc != SR_OK) break;
    total_left = 0;
    for (int b = 0; b < c->nrep; ++b) {
      const int done = (int)c->h_rs[b].windows_done;
      for (int w = 0; w < done; ++w) c->t_c[b] = c->t_c[b] + Tw[b];
      c->wins[b] += (unsigned)done;
      left[b] -= done;
      total_left += left[b];
      if (b == 0) c->last_nwin += done;
    }
    const unsigned status = c->h_st->status;
    if (status == 0u) {
      if (total_left != 0) rc = SR_ECUDA;   // the kernel ended early without a reason
      break;
    }
    if (status & ST_TIMEOUT) { rc = SR_TIMEOUT; break; }
    if (status & ST_NOT_CONVERGED) { rc = SR_NOT_CONVERGED; break; }
    if (status & ST_CAPACITY) {
      if (!c->cap_auto || c->cap >= kMaxCap) { rc = SR_CAPACITY; break; }
      if (cudaStreamSynchronize(c->stream) != cudaSuccess) { rc = SR_ECUDA; break; }
      rc = alloc_history(c, c->cap * 2);
      if (rc != SR_OK) break;
      continue;
    }
    rc = SR_ECUDA;
    break;
  }
  std::free(left);
  return rc;
}

int observables_of(sr_ctx* c, int b, sr_obs* out) {
  KParams k = make_params(c);
  if (cudaMemcpyAsync(c->h_st, c->st, sizeof(DevStats), cudaMemcpyDeviceToHost, c->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(c->h_rs + b, c->rs + b, sizeof(RepStats), cudaMemcpyDeviceToHost, c->stream) !=
          cudaSuccess ||
      cudaMemsetAsync(c->obs_i, 0, 2 * sizeof(long long), c->stream) != cudaSuccess)
    return SR_ECUDA;
  const RepDesc& d = c->hdesc[b];
  observe_ints_kernel<<<(d.NR + 255) / 256, 256, 0, c->stream>>>(k, b, c->obs_i);
  observe_integrals_kernel<<<1, 1024, 0, c->stream>>>(k, b, c->obs_f);
  if (cudaGetLastError() != cudaSuccess) return SR_ECUDA;
  c->launches += 2;
  cudaMemcpyAsync(c->h_obs_i, c->obs_i, 2 * sizeof(long long), cudaMemcpyDeviceToHost, c->stream);
  cudaMemcpyAsync(c->h_obs_f, c->obs_f, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return SR_ECUDA;
  const DevStats& h = *c->h_st;
  const RepStats& rs = c->h_rs[b];
  std::memset(out, 0, sizeof *out);
  out->t_c = c->t_c[b];
  out->mag = c->h_obs_i[0];
  out->bonds = c->h_obs_i[1];
  const double sites = (double)d.L * (double)d.L;
  out->m = (double)out->mag / sites;
  out->E = -c->reps[b].J * (double)out->bonds - c->reps[b].h * (double)out->mag;
  out->int_mag = c->h_obs_f[0];
  out->int_bonds = c->h_obs_f[1];
  out->committed = rs.committed;
  out->generated = rs.generated;
  out->breaks = rs.breaks;
  out->windows = rs.windows;
  out->iterations = rs.iterations;
  out->sum_f = rs.sum_f;
  out->last_iters = rs.last_iters;
  out->max_iters_seen = rs.max_iters_seen;
  out->max_f = rs.max_f;
  out->capacity = (uint32_t)c->cap;
  out->launches = c->launches;
  out->region_passes = h.region_passes;
  out->region_skips = h.region_skips;
  out->run_cycles = h.run_cycles;
  out->run_cycles_max = h.run_cycles_max;
  out->slots = h.slots;
  return SR_OK;
}

int spins_device_of(sr_ctx* c, int b, int8_t* dev_out, size_t n) {
  const RepDesc& d = c->hdesc[b];
  if (!dev_out || n != (size_t)d.L * d.L) return SR_EINVAL;
  KParams k = make_params(c);
  unpack_rows_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(k, b, dev_out);
  c->launches += 1;
  return cuda_rc(cudaGetLastError());
}

int spins_host_of(sr_ctx* c, int b, int8_t* host_out, size_t n) {
  if (!host_out) return SR_EINVAL;
  int rc = spins_device_of(c, b, c->stage, n);
  if (rc) return rc;
  if (cudaMemcpyAsync(host_out, c->stage, n, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    return SR_ECUDA;
  return cuda_rc(cudaStreamSynchronize(c->stream));
}

// Committed clock state of lattice b into caller device buffers (scratch: obs).
int carry_of(sr_ctx* c, int b, uint64_t* index, double* x, double* bb, double* t_last, size_t n) {
  const RepDesc& d = c->hdesc[b];
  if (n != (size_t)d.NR) return SR_EINVAL;
  unsigned long long* di = nullptr;
  double *dx = nullptr, *db = nullptr, *dt = nullptr;
  int rc = SR_OK;
  if (dalloc(&di, n) || dalloc(&dx, n) || dalloc(&db, n) || dalloc(&dt, n)) rc = SR_ENOMEM;
  if (rc == SR_OK) {
    KParams k = make_params(c);
    gather_carry_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(k, b, di, dx, db, dt);
    rc = cuda_rc(cudaGetLastError());
  }
  if (rc == SR_OK && index) cudaMemcpyAsync(index, di, n * 8, cudaMemcpyDeviceToHost, c->stream);
  if (rc == SR_OK && x) cudaMemcpyAsync(x, dx, n * 8, cudaMemcpyDeviceToHost, c->stream);
  if (rc == SR_OK && bb) cudaMemcpyAsync(bb, db, n * 8, cudaMemcpyDeviceToHost, c->stream);
  if (rc == SR_OK && t_last) cudaMemcpyAsync(t_last, dt, n * 8, cudaMemcpyDeviceToHost, c->stream);
  if (rc == SR_OK) rc = cuda_rc(cudaStreamSynchronize(c->stream));
  if (di) cudaFree(di);
  if (dx) cudaFree(dx);
  if (db) cudaFree(db);
  if (dt) cudaFree(dt);
  return rc;
}

// The last n entries of row `which` (0 iterations, 1 f) of the per-window ring.
int window_ring(sr_ctx* c, int which, uint32_t* out, size_t n) {
  if (!c || !out) return SR_EINVAL;
  const int have = c->last_nwin < kWinRing ? c->last_nwin : kWinRing;
  const int m = (int)n < have ? (int)n : have;
  if (m <= 0) return 0;
  uint32_t* tmp = (uint32_t*)std::malloc(kWinRing * sizeof(uint32_t));
  if (!tmp) return SR_ENOMEM;
  if (cudaMemcpyAsync(tmp, c->win_iters + (size_t)which * kWinRing, kWinRing * sizeof(uint32_t),
                      cudaMemcpyDeviceToHost,
                      c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    std::free(tmp);
    return SR_ECUDA;
  }
  // window w of the last launch is at w; a retried call (capacity growth)
  // restarts at 0, so the last m entries of the final launch are the last windows
  const int last_launch = (int)c->h_rs[0].windows_done;
  for (int i = 0; i < m; ++i) {
    const int w = last_launch - m + i;
    out[i] = tmp[((w % kWinRing) + kWinRing) % kWinRing];
  }
  std::free(tmp);
  return m;
}

}  // namespace

extern "C" {

const char* sr_strerror(int code) {
  switch (code) {
    case SR_OK: return "ok";
    case SR_EINVAL: return "invalid argument";
    case SR_ENOMEM: return "out of memory";
    case SR_ECUDA: return "CUDA error";
    case SR_NOT_CONVERGED: return "relaxation did not converge within the iteration cap";
    case SR_CAPACITY: return "boundary history exceeded the largest capacity";
    case SR_TIMEOUT: return "grid-wide synchronize timed out";
    case SR_EUNSUPPORTED: return "unsupported configuration";
    case SR_ETOOLARGE: return "problem does not fit the fixed no-allocation scratch";
    default: return "unknown status";
  }
}

int sr_create_ex(sr_ctx** out, const sr_params* prm) {
  if (!out || !prm) return SR_EINVAL;
  *out = nullptr;
  sr_replica r;
  std::memset(&r, 0, sizeof r);
  r.L = prm->L;
  r.J = prm->J;
  r.h = prm->h;
  r.T = prm->T;
  r.seed = prm->seed;
  r.init_mode = prm->init_mode;
  r.rates = prm->rates;
  return create_common(out, &r, 1, *prm);
}

int sr_create_batch(sr_ctx** out, const sr_replica* reps, int n, const sr_params* common) {
  if (!out || !common) return SR_EINVAL;
  *out = nullptr;
  return create_common(out, reps, n, *common);
}

int sr_create(sr_ctx** out, int L, double J, double h, double T, int region_w, int region_h,
              uint64_t seed) {
  sr_params p;
  std::memset(&p, 0, sizeof p);
  p.L = L;
  p.J = J;
  p.h = h;
  p.T = T;
  p.region_w = region_w;
  p.region_h = region_h;
  p.seed = seed;
  p.init_mode = SR_INIT_FAIR_COIN;
  p.rates = SR_RATES_METROPOLIS;
  p.test_barrier_skip_block = -1;
  return sr_create_ex(out, &p);
}

void sr_destroy(sr_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_all(c);
  std::free(c);
}

int sr_run_windows(sr_ctx* c, double t0, double Tw, int n) {
  if (!c || n < 1 || !(Tw > 0.0) || !std::isfinite(Tw)) return SR_EINVAL;
  for (int b = 0; b < c->nrep; ++b)
    if (t0 != c->t_c[b]) return SR_EINVAL;
  double* tw = (double*)std::malloc((size_t)c->nrep * sizeof(double));
  int* nw = (int*)std::malloc((size_t)c->nrep * sizeof(int));
  int rc = SR_ENOMEM;
  if (tw && nw) {
    for (int b = 0; b < c->nrep; ++b) {
      tw[b] = Tw;
      nw[b] = n;
    }
    rc = run_all(c, tw, nw);
  }
  std::free(tw);
  std::free(nw);
  return rc;
}

int sr_run_window(sr_ctx* c, double t0, double Tw) { return sr_run_windows(c, t0, Tw, 1); }

int sr_run_batch(sr_ctx* c, const double* Tw, const int* n_windows) {
  if (!c || !Tw || !n_windows) return SR_EINVAL;
  return run_all(c, Tw, n_windows);
}

int sr_observables(sr_ctx* c, sr_obs* out) {
  if (!c || !out) return SR_EINVAL;
  return observables_of(c, 0, out);
}

int sr_observables_replica(sr_ctx* c, int replica, sr_obs* out) {
  if (!c || !out || replica < 0 || replica >= c->nrep) return SR_EINVAL;
  return observables_of(c, replica, out);
}

int sr_get_spins_device(sr_ctx* c, int8_t* dev_out, size_t n) {
  if (!c) return SR_EINVAL;
  return spins_device_of(c, 0, dev_out, n);
}

int sr_get_spins(sr_ctx* c, int8_t* host_out, size_t n) {
  if (!c) return SR_EINVAL;
  return spins_host_of(c, 0, host_out, n);
}

int sr_get_spins_replica(sr_ctx* c, int replica, int8_t* host_out, size_t n) {
  if (!c || replica < 0 || replica >= c->nrep) return SR_EINVAL;
  return spins_host_of(c, replica, host_out, n);
}

int sr_set_spins_device(sr_ctx* c, const int8_t* dev_in, size_t n) {
  if (!c || !dev_in || n != (size_t)c->hdesc[0].L * c->hdesc[0].L) return SR_EINVAL;
  return init_state(c, 0, dev_in);
}

int sr_set_spins(sr_ctx* c, const int8_t* host_in, size_t n) {
  if (!c || !host_in || n != (size_t)c->hdesc[0].L * c->hdesc[0].L) return SR_EINVAL;
  if (cudaMemcpyAsync(c->stage, host_in, n, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
    return SR_ECUDA;
  int rc = init_state(c, 0, c->stage);
  if (rc) return rc;
  return cuda_rc(cudaStreamSynchronize(c->stream));
}

int sr_reset(sr_ctx* c) {
  if (!c) return SR_EINVAL;
  int rc = init_state(c, -1, nullptr);
  if (rc) return rc;
  return cuda_rc(cudaStreamSynchronize(c->stream));
}

int sr_get_carry(sr_ctx* c, uint64_t* index, double* x, double* b, double* t_last, size_t n) {
  if (!c) return SR_EINVAL;
  return carry_of(c, 0, index, x, b, t_last, n);
}

int sr_get_carry_replica(sr_ctx* c, int replica, uint64_t* index, double* x, double* b,
                         double* t_last, size_t n) {
  if (!c || replica < 0 || replica >= c->nrep) return SR_EINVAL;
  return carry_of(c, replica, index, x, b, t_last, n);
}

int sr_get_trace(sr_ctx* c, uint64_t* lens, double* times, uint32_t* sites, size_t n_regions,
                 size_t cap) {
  if (!c || n_regions != (size_t)c->hdesc[0].NR) return SR_EINVAL;
  if ((times || sites) && (c->prm.trace_capacity == 0 || cap != (size_t)c->prm.trace_capacity))
    return SR_EINVAL;
  int rc = SR_OK;
  if (lens) rc = carry_of(c, 0, lens, nullptr, nullptr, nullptr, n_regions);
  if (rc) return rc;
  const size_t total = n_regions * cap;     // lattice 0 holds regions 0 .. NR0 - 1
  if (times) cudaMemcpyAsync(times, c->trt, total * 8, cudaMemcpyDeviceToHost, c->stream);
  if (sites) cudaMemcpyAsync(sites, c->trs, total * 4, cudaMemcpyDeviceToHost, c->stream);
  return cuda_rc(cudaStreamSynchronize(c->stream));
}

int sr_get_window_iters(sr_ctx* c, uint32_t* out, size_t n) { return window_ring(c, 0, out, n); }

int sr_get_window_f(sr_ctx* c, uint32_t* out, size_t n) { return window_ring(c, 1, out, n); }

int sr_eval_draws(uint64_t seed, uint32_t region, uint64_t i0, size_t n, double* x, uint64_t* kV) {
  if (n == 0) return SR_OK;
  double* dx = nullptr;
  unsigned long long* dk = nullptr;
  if (dalloc(&dx, n) || dalloc(&dk, n)) {
    if (dx) cudaFree(dx);
    if (dk) cudaFree(dk);
    return SR_ENOMEM;
  }
  eval_draws_kernel<<<(unsigned)((n + 255) / 256), 256>>>((uint32_t)seed, (uint32_t)(seed >> 32),
                                                          region, i0, n, dx, dk);
  int rc = cuda_rc(cudaGetLastError());
  if (rc == SR_OK && x) rc = cuda_rc(cudaMemcpy(x, dx, n * 8, cudaMemcpyDeviceToHost));
  if (rc == SR_OK && kV) rc = cuda_rc(cudaMemcpy(kV, dk, n * 8, cudaMemcpyDeviceToHost));
  cudaFree(dx);
  cudaFree(dk);
  return rc;
}

int sr_eval_softfloat(int op, const double* a, const double* b, double* out, size_t n) {
  if (op < 0 || op > 4 || !a || !b || !out) return SR_EINVAL;
  if (n == 0) return SR_OK;
  double *da = nullptr, *db = nullptr, *dout = nullptr;
  int rc = SR_OK;
  if (dalloc(&da, n) || dalloc(&db, n) || dalloc(&dout, n)) rc = SR_ENOMEM;
  if (rc == SR_OK) rc = cuda_rc(cudaMemcpy(da, a, n * 8, cudaMemcpyHostToDevice));
  if (rc == SR_OK) rc = cuda_rc(cudaMemcpy(db, b, n * 8, cudaMemcpyHostToDevice));
  if (rc == SR_OK) {
    eval_softfloat_kernel<<<(unsigned)((n + 255) / 256), 256>>>(op, da, db, dout, n);
    rc = cuda_rc(cudaGetLastError());
  }
  if (rc == SR_OK) rc = cuda_rc(cudaMemcpy(out, dout, n * 8, cudaMemcpyDeviceToHost));
  if (da) cudaFree(da);
  if (db) cudaFree(db);
  if (dout) cudaFree(dout);
  return rc;
}

int sr_run_batch_adaptive(sr_ctx* c, const double* t_end, const sr_adapt* opts, double* last_tw) {
  if (!c || !t_end) return SR_EINVAL;
  sr_adapt o;
  std::memset(&o, 0, sizeof o);
  if (opts) o = *opts;
  if (o.kappa == 0.0) o.kappa = 8.0;
  if (o.chunk == 0.0) o.chunk = 1.0;
  if (o.tw_first == 0.0) o.tw_first = 1.0 / 16.0;
  if (o.tw_min == 0.0) o.tw_min = std::ldexp(1.0, -10);
  if (o.tw_max == 0.0) o.tw_max = o.chunk;
  const double vals[5] = {o.kappa, o.chunk, o.tw_first, o.tw_min, o.tw_max};
  for (double v : vals)
    if (!(v > 0.0) || !std::isfinite(v)) return SR_EINVAL;
  if (o.tw_min > o.tw_max) return SR_EINVAL;
  const int n = c->nrep;
  for (int b = 0; b < n; ++b)
    if (!(t_end[b] >= c->t_c[b]) || !std::isfinite(t_end[b])) return SR_EINVAL;
  // window length to the nearest power of two, clamped
  auto pow2 = [&](double v) {
    double w = std::ldexp(1.0, (int)std::lround(std::log2(v)));
    if (w < o.tw_min) w = o.tw_min;
    if (w > o.tw_max) w = o.tw_max;
    return w;
  };
  double* tw = (double*)std::malloc((size_t)n * sizeof(double));
  double* Tw = (double*)std::malloc((size_t)n * sizeof(double));
  double* span = (double*)std::malloc((size_t)n * sizeof(double));
  unsigned long long* c0 = (unsigned long long*)std::malloc((size_t)n * sizeof(unsigned long long));
  int* nw = (int*)std::malloc((size_t)n * sizeof(int));
  int rc = SR_OK;
  if (!tw || !Tw || !span || !c0 || !nw) rc = SR_ENOMEM;
  if (rc == SR_OK) {
    for (int b = 0; b < n; ++b) tw[b] = pow2(o.tw_first);
    // the per-lattice committed counts before the first chunk
    if (cudaMemcpyAsync(c->h_rs, c->rs, (size_t)n * sizeof(RepStats), cudaMemcpyDeviceToHost,
                        c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      rc = SR_ECUDA;
  }
  while (rc == SR_OK) {
    bool any = false;
    for (int b = 0; b < n; ++b) {
      const double rem = t_end[b] - c->t_c[b];
      nw[b] = 0;
      Tw[b] = 1.0;
      span[b] = 0.0;
      c0[b] = c->h_rs[b].committed;
      if (!(rem > 0.0)) continue;
      const double sp = rem < o.chunk ? rem : o.chunk;
      double w = tw[b] < sp ? tw[b] : sp;
      double k = std::floor(sp / w);
      if (k < 1.0) k = 1.0;
      if (k > 1e6) k = 1e6;
      nw[b] = (int)k;
      Tw[b] = w;
      span[b] = k * w;
      any = true;
    }
    if (!any) break;
    rc = run_all(c, Tw, nw);
    if (rc != SR_OK) break;
    for (int b = 0; b < n; ++b) {
      if (nw[b] == 0) continue;
      const double dc = (double)(c->h_rs[b].committed - c0[b]);
      const double rho = dc / ((double)c->hdesc[b].NR * span[b]);
      tw[b] = rho > 0.0 ? pow2(o.kappa / rho) : o.tw_max;
      if (last_tw) last_tw[b] = Tw[b];
    }
  }
  std::free(tw);
  std::free(Tw);
  std::free(span);
  std::free(c0);
  std::free(nw);
  return rc;
}

int sr_autotune(const sr_replica* reps, int n, const sr_params* common, double t_trial,
                sr_tune* out) {
  if (!reps || n < 1 || !common || !out) return SR_EINVAL;
  if (t_trial == 0.0) t_trial = 1.0;
  if (!(t_trial > 0.0) || !std::isfinite(t_trial)) return SR_EINVAL;
  std::memset(out, 0, sizeof *out);
  const int shapes[5][2] = {{16, 16}, {8, 8}, {32, 32}, {16, 8}, {32, 16}};
  bool ok[5];
  int n_ok = 0;
  for (int s = 0; s < 5; ++s) {
    ok[s] = true;
    for (int b = 0; b < n; ++b)
      if (reps[b].L % shapes[s][0] || reps[b].L % shapes[s][1]) ok[s] = false;
    n_ok += ok[s];
  }
  if (n_ok == 0) return SR_EUNSUPPORTED;
  double* te = (double*)std::malloc((size_t)n * sizeof(double));
  if (!te) return SR_ENOMEM;
  // one trial: committed flips per second over [t_trial / 2, t_trial]
  auto trial = [&](int w, int h, int lpw, double kappa, double* score) -> int {
    sr_params p = *common;
    p.region_w = w;
    p.region_h = h;
    p.lanes_per_warp = lpw;
    sr_ctx* c = nullptr;
    int rc = create_common(&c, reps, n, p);
    if (rc != SR_OK) return rc;
    sr_adapt o;
    std::memset(&o, 0, sizeof o);
    o.kappa = kappa;
    o.chunk = t_trial / 4.0;
    for (int b = 0; b < n; ++b) te[b] = 0.5 * t_trial;
    rc = sr_run_batch_adaptive(c, te, &o, nullptr);
    unsigned long long before = 0, after = 0;
    for (int b = 0; b < n && rc == SR_OK; ++b) before += c->h_rs[b].committed;
    const auto t0 = std::chrono::steady_clock::now();
    for (int b = 0; b < n; ++b) te[b] = t_trial;
    if (rc == SR_OK) rc = sr_run_batch_adaptive(c, te, &o, nullptr);
    const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int b = 0; b < n && rc == SR_OK; ++b) after += c->h_rs[b].committed;
    sr_destroy(c);
    *score = dt > 0.0 ? (double)(after - before) / dt : 0.0;
    out->trials += 1;
    return rc;
  };
  int rc = SR_OK;
  int bw = 0, bh = 0, blpw = 0;
  double bk = 8.0, best = -1.0;
  for (int s = 0; s < 5 && rc == SR_OK; ++s) {
    if (!ok[s]) continue;
    double sc = 0.0;
    rc = trial(shapes[s][0], shapes[s][1], 0, bk, &sc);
    if (rc == SR_OK && sc > best) {
      best = sc;
      bw = shapes[s][0];
      bh = shapes[s][1];
    }
  }
  const double kappas[3] = {4.0, 16.0, 32.0};
  for (int i = 0; i < 3 && rc == SR_OK; ++i) {
    double sc = 0.0;
    rc = trial(bw, bh, 0, kappas[i], &sc);
    if (rc == SR_OK && sc > best) {
      best = sc;
      bk = kappas[i];
    }
  }
  const int lpws[3] = {8, 16, 32};
  for (int i = 0; i < 3 && rc == SR_OK; ++i) {
    double sc = 0.0;
    rc = trial(bw, bh, lpws[i], bk, &sc);
    if (rc == SR_OK && sc > best) {
      best = sc;
      blpw = lpws[i];
    }
  }
  std::free(te);
  if (rc != SR_OK) return rc;
  out->region_w = bw;
  out->region_h = bh;
  out->lanes_per_warp = blpw;
  out->kappa = bk;
  out->flips_per_s = best;
  return SR_OK;
}

int sr_score(sr_ctx* c, double* out) {
  if (!c || !out) return SR_EINVAL;
  if (!c->prm.score) return SR_EUNSUPPORTED;
  KParams k = make_params(c);
  score_kernel<<<c->nrep, 256, 0, c->stream>>>(k, c->score_tab, c->score_out);
  if (cudaGetLastError() != cudaSuccess) return SR_ECUDA;
  c->launches += 1;
  double* h = (double*)std::malloc((size_t)c->nrep * 23 * sizeof(double));
  if (!h) return SR_ENOMEM;
  int rc = cuda_rc(cudaMemcpyAsync(h, c->score_out, (size_t)c->nrep * 23 * sizeof(double),
                                   cudaMemcpyDeviceToHost, c->stream));
  if (rc == SR_OK) rc = cuda_rc(cudaStreamSynchronize(c->stream));
  if (rc == SR_OK)
    for (int b = 0; b < c->nrep; ++b)
      for (int q = 0; q < 3; ++q) out[b * 3 + q] = h[(size_t)b * 23 + q];
  std::free(h);
  return rc;
}

int sr_score_stats(sr_ctx* c, int replica, uint64_t* counts, double* occupancy) {
  if (!c || replica < 0 || replica >= c->nrep) return SR_EINVAL;
  if (!c->prm.score) return SR_EUNSUPPORTED;
  KParams k = make_params(c);
  score_kernel<<<c->nrep, 256, 0, c->stream>>>(k, c->score_tab, c->score_out);
  if (cudaGetLastError() != cudaSuccess) return SR_ECUDA;
  c->launches += 1;
  double h[23];
  int rc = cuda_rc(cudaMemcpyAsync(h, c->score_out + (size_t)replica * 23, sizeof h,
                                   cudaMemcpyDeviceToHost, c->stream));
  if (rc == SR_OK) rc = cuda_rc(cudaStreamSynchronize(c->stream));
  if (rc != SR_OK) return rc;
  for (int q = 0; q < 10; ++q) {
    if (counts) counts[q] = (uint64_t)h[3 + q];
    if (occupancy) occupancy[q] = h[13 + q];
  }
  return SR_OK;
}

int sr_score_grad(int n, int m, int nq, const double* A, const double* gA, const double* S,
                  const double* E, double* G, void* stream) {
  if (n < 1 || m < 1 || nq < 1 || m > 1024 || !A || !gA || !S || !G) return SR_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  double* sums = nullptr;
  if (dalloc(&sums, (size_t)m)) return SR_ENOMEM;
  colsum_kernel<<<m, 256, 0, st>>>(n, m, A, sums);
  score_grad_kernel<<<(n * nq + 255) / 256, 256, 0, st>>>(n, m, nq, A, gA, S, E, sums, G);
  int rc = cuda_rc(cudaGetLastError());
  if (rc == SR_OK) rc = cuda_rc(cudaStreamSynchronize(st));
  cudaFree(sums);
  return rc;
}

int sr_get_info(sr_ctx* c, int* n_regions, int* frac_bits, uint64_t* P, int* threads_per_block,
                int* blocks) {
  if (!c) return SR_EINVAL;
  if (n_regions) *n_regions = c->hdesc[0].NR;
  if (frac_bits) *frac_bits = c->F;
  if (P)
    for (int k = 0; k < 10; ++k) P[k] = c->hdesc[0].P[k];
  if (threads_per_block) *threads_per_block = c->rl;
  if (blocks) *blocks = c->blocks;
  return SR_OK;
}

}  // extern "C"

// ====================================================================== no-allocation entry
// For callers that must not allocate GPU memory when they simulate.  All
// working state of sr_run_noalloc lives in this fixed array, which every GPU
// that loads the library holds until the process exits.  Host code never uses
// the symbol itself as an address: it asks the runtime for the device address
// once per device (see noalloc_scratch).
static __device__ __align__(256) unsigned char g_noalloc_scratch[SR_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kNoallocCap = 64;       // boundary events per region edge per iteration
constexpr int kNoallocRing = 64;      // presimulated pairs per region
constexpr int kMaxDevices = 64;
void* g_noalloc_ptr[kMaxDevices];     // device address of the scratch, per device

// Device address of the scratch on the current device, looked up on first use.
int noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SR_ECUDA;
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return SR_ECUDA;
    g_noalloc_ptr[dev] = ptr;
  }
  *out = g_noalloc_ptr[dev];
  return SR_OK;
}

// Carve a 256-byte-aligned piece of `bytes` out of the scratch.
struct Carver {
  unsigned char* base;
  size_t used;
  template <class T>
  T* take(size_t count) {
    used = (used + 255) & ~(size_t)255;
    T* p = reinterpret_cast<T*>(base + used);
    used += count * sizeof(T);
    return p;
  }
};

}  // namespace

extern "C" int sr_run_noalloc(int L, double J, double h, double T, int region_w, int region_h,
                              uint64_t seed, const int8_t* spins_in, double Tw, int n_windows,
                              int8_t* spins_out, uint64_t* counts_out, void* stream) {
  if (L < 3 || region_w < 1 || region_h < 1 || L % region_w || L % region_h) return SR_EINVAL;
  if (!(T > 0.0) || !std::isfinite(J) || !std::isfinite(h) || std::isnan(T)) return SR_EINVAL;
  if (!(Tw > 0.0) || !std::isfinite(Tw) || n_windows < 1 || !spins_out) return SR_EINVAL;
  if (region_w > 32 || region_h > 32) return SR_EUNSUPPORTED;

  // the same context a sr_create_ex would build, without any allocation
  sr_replica rp;
  std::memset(&rp, 0, sizeof rp);
  rp.L = L;
  rp.J = J;
  rp.h = h;
  rp.T = T;
  rp.seed = seed;
  rp.init_mode = SR_INIT_FAIR_COIN;
  rp.rates = SR_RATES_METROPOLIS;
  RepDesc hd;
  std::memset(&hd, 0, sizeof hd);
  double t_c = 0.0;
  unsigned wins = 0u;
  sr_ctx c;
  std::memset(&c, 0, sizeof c);
  c.prm.L = L;
  c.prm.region_w = region_w;
  c.prm.region_h = region_h;
  c.prm.max_iters = 1 << 16;
  c.prm.barrier_timeout_ms = 2000;
  c.prm.test_barrier_skip_block = -1;
  c.nrep = 1;
  c.reps = &rp;
  c.hdesc = &hd;
  c.t_c = &t_c;
  c.wins = &wins;
  c.F = 63 - bitlen((long long)region_w * region_h);
  c.scale = std::ldexp(1.0, -c.F);
  hd.L = L;
  hd.NX = L / region_w;
  hd.NY = L / region_h;
  hd.NR = hd.NX * hd.NY;
  hd.off = 0;
  hd.spans_x = hd.NX == 1;
  hd.spans_y = hd.NY == 1;
  hd.key0 = (uint32_t)seed;
  hd.key1 = (uint32_t)(seed >> 32);
  hd.init_mode = SR_INIT_FAIR_COIN;
  rate_table(rp, c.F, hd.P);
  for (int k = 0; k < 10; ++k) hd.Rp[k] = hd.P[k] ? ~0ull / hd.P[k] : 0ull;
  c.NR = hd.NR;
  c.Lmax = L;
  c.stream = (cudaStream_t)stream;

  // size check before touching the GPU
  const size_t nr = (size_t)c.NR, H = (size_t)region_h;
  Carver probe{nullptr, 0};
  probe.take<uint32_t>(2 * H * nr);               // rows
  probe.take<uint32_t>(4 * nr);                   // halos
  for (int a = 0; a < 7; ++a) probe.take<double>(2 * nr);   // carry
  probe.take<double>((size_t)2 * 4 * kNoallocCap * nr);     // list times
  probe.take<uint8_t>((size_t)2 * 4 * kNoallocCap * nr);    // list positions
  probe.take<uint32_t>(2 * 4 * nr);               // list lengths
  probe.take<uint8_t>(2 * nr);                    // list-changed flags
  probe.take<double>((size_t)kNoallocRing * nr);  // ring x
  probe.take<unsigned long long>((size_t)kNoallocRing * nr);  // ring V
  probe.take<unsigned long long>(nr);             // ring ends
  probe.take<DevStats>(1);
  probe.take<uint32_t>(2 * (size_t)kWinRing);
  probe.take<uint32_t>(2);                        // f of the running window
  probe.take<RepDesc>(1);                         // lattice descriptor and counters
  probe.take<RepStats>(1);
  probe.take<uint32_t>(3);                        // convergence flags
  probe.take<uint32_t>(3 * nr);                   // lattice, iteration, window of each region
  probe.take<double>(nr);                         // window start of each region
  probe.take<uint8_t>(2 * nr);                    // committed copy, ring top-up pending
  if (probe.used > (size_t)SR_NOALLOC_SCRATCH_BYTES) return SR_ETOOLARGE;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&c.clock_khz, cudaDevAttrClockRate, dev) != cudaSuccess)
    return SR_ECUDA;
  void* base = nullptr;
  int rc = noalloc_scratch(&base);
  if (rc != SR_OK) return rc;
  Carver cv{(unsigned char*)base, 0};
  c.rows = cv.take<uint32_t>(2 * H * nr);
  c.halo = cv.take<uint32_t>(4 * nr);
  c.ci = cv.take<unsigned long long>(2 * nr);
  c.cx = cv.take<double>(2 * nr);
  c.ckv = cv.take<unsigned long long>(2 * nr);
  c.cb = cv.take<double>(2 * nr);
  c.ct = cv.take<double>(2 * nr);
  c.cim = cv.take<double>(2 * nr);
  c.cib = cv.take<double>(2 * nr);
  c.ht = cv.take<double>((size_t)2 * 4 * kNoallocCap * nr);
  c.hp = cv.take<uint8_t>((size_t)2 * 4 * kNoallocCap * nr);
  c.hl = cv.take<uint32_t>(2 * 4 * nr);
  c.chg = cv.take<uint8_t>(2 * nr);
  c.rx = cv.take<double>((size_t)kNoallocRing * nr);
  c.rkv = cv.take<unsigned long long>((size_t)kNoallocRing * nr);
  c.rhi = cv.take<unsigned long long>(nr);
  c.st = cv.take<DevStats>(1);
  c.win_iters = cv.take<uint32_t>(2 * (size_t)kWinRing);
  c.curf = cv.take<uint32_t>(2);
  c.desc = cv.take<RepDesc>(1);
  c.rs = cv.take<RepStats>(1);
  c.rflags = cv.take<uint32_t>(3);
  c.rrep = cv.take<uint32_t>(nr);
  c.rn = cv.take<uint32_t>(nr);
  c.rwin = cv.take<uint32_t>(nr);
  c.rts = cv.take<double>(nr);
  c.rcidx = cv.take<uint8_t>(nr);
  c.rfill = cv.take<uint8_t>(nr);
  c.cap = kNoallocCap;
  c.K = kNoallocRing;
  c.Kcap = kNoallocRing;

  // launch shape as sr_create_ex chooses it
  const int per_sm = (c.NR + c.num_sms - 1) / c.num_sms;
  const int bps = (per_sm + 255) / 256;
  int rl = (per_sm + bps - 1) / bps;
  if (rl > 32) rl = ((rl + 31) / 32) * 32;
  if (rl > 256) rl = 256;
  if (rl < 1) rl = 1;
  int tpb = ((rl + 31) / 32) * 32;
  if (tpb < 128) tpb = 128;
  c.rl = rl;
  c.lanes = 32;            // lane mapping, every thread of a block a region lane
  c.tpb = tpb;
  c.smem = lane_smem_bytes(region_h, rl, false);
  int per_sm_blocks = 0;
  if (!allow_smem((const void*)relax_kernel<0, 0>, c.smem) ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_blocks, relax_kernel<0, 0>, tpb, c.smem) !=
          cudaSuccess ||
      per_sm_blocks < 1) {
    cudaGetLastError();
    return SR_EUNSUPPORTED;
  }
  int blocks = (c.NR + rl - 1) / rl;
  if (blocks > per_sm_blocks * c.num_sms) blocks = per_sm_blocks * c.num_sms;
  c.blocks = blocks;

  // the shared scratch keeps the previous call's contents: start from zero
  // where the kernels expect it (list lengths; every region is lattice 0)
  if (cudaMemsetAsync(c.hl, 0, 2 * 4 * nr * sizeof(uint32_t), c.stream) != cudaSuccess ||
      cudaMemsetAsync(c.rrep, 0, nr * sizeof(uint32_t), c.stream) != cudaSuccess)
    return SR_ECUDA;
  rc = init_state(&c, 0, spins_in);         // spins, halos, clocks, counters, rings
  if (rc != SR_OK) return rc;

  // one persistent launch for all windows, then read the status words
  hd.t0 = 0.0;
  hd.Tw = Tw;
  hd.nwin = n_windows;
  if (cudaMemcpyAsync(c.desc, &hd, sizeof hd, cudaMemcpyHostToDevice, c.stream) != cudaSuccess ||
      cudaMemsetAsync(c.st, 0, offsetof(DevStats, region_passes), c.stream) != cudaSuccess ||
      cudaMemsetAsync(c.rflags, 0, 3 * sizeof(uint32_t), c.stream) != cudaSuccess ||
      cudaMemsetAsync(c.curf, 0, 2 * sizeof(uint32_t), c.stream) != cudaSuccess)
    return SR_ECUDA;
  KParams k = make_params(&c);
  void* args[] = {&k};
  if (cudaLaunchCooperativeKernel((const void*)relax_kernel<0, 0>, dim3(c.blocks), dim3(c.tpb), args,
                                  c.smem, c.stream) != cudaSuccess) {
    cudaGetLastError();
    return SR_ECUDA;
  }
  DevStats hs;
  RepStats hr;
  if (cudaMemcpyAsync(&hs, c.st, sizeof hs, cudaMemcpyDeviceToHost, c.stream) != cudaSuccess ||
      cudaMemcpyAsync(&hr, c.rs, sizeof hr, cudaMemcpyDeviceToHost, c.stream) != cudaSuccess ||
      cudaStreamSynchronize(c.stream) != cudaSuccess)
    return SR_ECUDA;
  if (hs.status & ST_TIMEOUT) return SR_TIMEOUT;
  if (hs.status & ST_NOT_CONVERGED) return SR_NOT_CONVERGED;
  if (hs.status & ST_CAPACITY) return SR_CAPACITY;
  if (hs.status != 0u || (int)hr.windows_done != n_windows) return SR_ECUDA;

  // outputs
  unpack_rows_kernel<<<(unsigned)(((size_t)L * L + 255) / 256), 256, 0, c.stream>>>(k, 0, spins_out);
  if (cudaGetLastError() != cudaSuccess) return SR_ECUDA;
  if (counts_out) {
    // committed event index of each region = its committed events
    gather_carry_kernel<<<(unsigned)((nr + 255) / 256), 256, 0, c.stream>>>(
        k, 0, (unsigned long long*)counts_out, nullptr, nullptr, nullptr);
    if (cudaGetLastError() != cudaSuccess) return SR_ECUDA;
  }
  return cuda_rc(cudaStreamSynchronize(c.stream));
}
