// sr_kernel.cuh -- the kernels of libsr: the persistent relaxation kernel with
// its static, dynamic and asynchronous schedules (§4 boxed procedure), and the
// helper kernels (initial state, halos, observables, score statistics).
#pragma once
#include "sr_region.cuh"

namespace sr {

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

// Ring top-up of the regions of a commit task by the whole warp (asynchronous
// schedule).  The region r of a lane with `want` needs the pairs of events
// [max(rhi, i_c), i_c + K) (all K under the alternate step rule, whose window
// wg starts on new numbers); the warp draws the pairs of all its regions 32 at
// a time, so a region's top-up is not a serial chain of draws on its lattice's
// path.  Every lane of the warp calls it.
template <bool GEN>
__device__ void fill_warp(const KParams& p, bool want, int r, uint32_t loc, uint32_t key0,
                          uint32_t key1, unsigned wg) {
  constexpr unsigned kAll = 0xFFFFFFFFu;
  const int lane = threadIdx.x & 31;
  const size_t nr = (size_t)p.NR;
  const unsigned long long kmask = (unsigned long long)p.K - 1ull;
  const bool fresh = GEN && p.fresh;
  unsigned long long lo = 0ull, from = 0ull, to = 0ull;
  if (want) {
    lo = __ldcg(&p.ci[(size_t)p.rcidx[r] * nr + r]);
    const unsigned long long hi_old = p.rhi[r];
    from = (hi_old > lo && !fresh) ? hi_old : lo;
    to = lo + (unsigned long long)p.K;
  }
  const unsigned cnt = want ? (unsigned)(to - from) : 0u;     // at most K <= 4096
  unsigned incl = cnt;                                        // inclusive prefix over lanes
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned o = __shfl_up_sync(kAll, incl, d);
    if (lane >= d) incl += o;
  }
  const unsigned total = __shfl_sync(kAll, incl, 31);
  for (unsigned k0 = 0; k0 < total; k0 += 32) {
    const unsigned k = k0 + (unsigned)lane;
    // the lane whose range holds draw k: the number of lanes with prefix <= k
    int owner = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const unsigned v = __shfl_sync(kAll, incl, owner + step - 1);
      if (v <= k) owner += step;
    }
    owner &= 31;                                              // k >= total: no draw
    const unsigned excl = __shfl_sync(kAll, incl - cnt, owner);
    const unsigned long long ofrom = __shfl_sync(kAll, from, owner);
    const unsigned long long olo = __shfl_sync(kAll, lo, owner);
    const int orr = __shfl_sync(kAll, r, owner);
    const uint32_t oloc = __shfl_sync(kAll, loc, owner);
    const uint32_t ok0 = __shfl_sync(kAll, key0, owner), ok1 = __shfl_sync(kAll, key1, owner);
    if (k < total) {
      const unsigned long long i = ofrom + (unsigned long long)(k - excl);
      double x;
      unsigned long long kv;
      if (fresh)
        draw_event_fresh((unsigned)(i - olo), wg, oloc, ok0, ok1, x, kv);
      else
        draw_event(i, oloc, ok0, ok1, x, kv);
      const size_t a = (size_t)(i & kmask) * nr + (size_t)orr;
      p.rx[a] = x;
      p.rkv[a] = kv;
    }
  }
  if (want) p.rhi[r] = to;
}

// Task queue of the asynchronous schedule: a ring of qcap slots; ticket t
// (the t-th task published, and the t-th claim) lives in slot t mod qcap.  A
// task is (kind, lattice, chunk of `chunk` consecutive regions); kinds 0 =
// pass, 1 = commit.  Every item carries the low 20 bits of its ticket; a
// consumer takes only the item of its own ticket (qcap is odd, so an item of
// an earlier lap never carries the tag of the slot's current ticket) and
// clears it by compare-and-swap.  The items of a set are written one by one
// after their tickets are reserved, and a slow publisher (many chunks, a busy
// GPU) can find a slot still holding the item of the ticket one lap earlier,
// not yet taken: an item is therefore written only into an empty slot
// (compare-and-swap), waiting, within the bounded wait of SR_TIMEOUT, for the
// earlier one to be taken.  No item is ever overwritten, lost or taken twice.
// The publishing thread has made the lattice's state visible first (fence).
__host__ __device__ constexpr unsigned long long task_item(unsigned kind, unsigned b, unsigned c,
                                                           unsigned long long ticket) {
  return kTaskValid | ((unsigned long long)(kind & 1u) << 62) | ((unsigned long long)b << 42) |
         ((unsigned long long)c << 20) | (ticket & kTaskTag);
}

// Polling reads of words that other SMs write during the launch: the slot by
// an atomic (performed at L2, always current: a warp polling its own slot
// keeps the line hot in its SM's L1), the scheduler words by loads that bypass L1.
__device__ __forceinline__ unsigned long long poll_slot(unsigned long long* a) {
  return atomicOr(a, 0ull);
}
__device__ __forceinline__ unsigned long long poll_word(const unsigned long long* a) { return __ldcg(a); }
__device__ __forceinline__ unsigned poll_word(const unsigned* a) { return __ldcg(a); }

// The task set of lattice b (one task per chunk of `chunk` regions), published
// by all 32 lanes of the calling warp: lane 0 reserves the tickets, lane j
// writes the items of chunks j, j + 32, ...  An item goes into an empty slot
// only (compare-and-swap), waiting within the bounded wait for an older item
// still there to be taken.  One lane writing every item in turn kept the last
// task of a large lattice waiting for dozens of round trips to L2.
__device__ void enqueue_lattice(const KParams& p, int b, unsigned kind, int chunk, int lane) {
  const int nreg = p.reps[b].NR;
  const unsigned long long nch = (unsigned long long)((nreg + chunk - 1) / chunk);
  unsigned long long base = 0ull;
  if (lane == 0) base = atomicAdd(&p.st->qtail, nch);
  base = __shfl_sync(0xFFFFFFFFu, base, 0);
  __syncwarp();
  __threadfence();     // the lattice state lane 0 wrote comes before every item
  for (unsigned long long c = (unsigned long long)lane; c < nch; c += 32ull) {
    const unsigned long long t = base + c;
    const unsigned long long item = task_item(kind, (unsigned)b, (unsigned)c, t);
    unsigned long long* slot = &p.q[t % p.qcap];
    if (atomicCAS(slot, 0ull, item) == 0ull) continue;
    const long long t0 = clock64();
    unsigned nap = 32u;
    while (atomicCAS(slot, 0ull, item) != 0ull) {
      if (clock64() - t0 > p.timeout_cycles) {
        atomicOr(&p.st->status, ST_TIMEOUT);
        atomicOr(&p.st->cwork, 1ull << 63);
        return;
      }
      __nanosleep(nap);
      if (nap < 1024u) nap *= 2u;
    }
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
// b*rl + j + k*(gridDim.x*rl).  GEN = false: no score mode, alternate step
// rule or trace (see run_region); with the asynchronous schedule the rings
// are then filled for the whole launch at its start and commits draw nothing.
template <int MODE, int DYN, bool GEN>
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
    const int pt_words = ((p.H + 10 * g.hq) * stride + 1) & ~1;   // 8-byte aligned tables
    unsigned long long* tab = reinterpret_cast<unsigned long long*>(smem + pt_words);
    if (DYN == 2 && LANES) {
      // asynchronous schedule: the lanes of a warp all run one lattice's task,
      // so they share one rate table (a lane reading P_k and one reading P_k'
      // touch different banks; equal k is a broadcast) -- 160 bytes of shared
      // memory per region slot less, so more blocks fit on an SM
      g.PT = tab + 20 * warp;
      g.pts = 1;
      g.SX = tab + 20 * (int)(blockDim.x >> 5) + (is_slot ? slot : 0);   // score mode only
    } else {
      g.PT = tab + (LANES && is_slot ? slot : 0);
      g.pts = stride;
      g.SX = g.PT + 20 * stride;                                       // score mode only
    }
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
    int warp_rep = -1;       // lattice whose rates the warp's table holds
    for (;;) {
      unsigned long long item = 0ull;
      if (lane == 0) {
        const unsigned long long ticket = atomicAdd(&st->qhead, 1ull);
        const unsigned long long slot = ticket % p.qcap;
        // the wait ends with SR_TIMEOUT only after a whole timeout in which no
        // task was published anywhere: when one small lattice is left, the
        // waiting warps are served a few per iteration, in the order they came
        long long tw0 = clock64();
        unsigned long long seen = poll_word(&st->qtail);
        // idle warps back off (64 ns doubling to 2 us) so that their polls do
        // not crowd the memory system of the warps that work
        unsigned nap = 64u;
        for (;;) {
          item = poll_slot(&p.q[slot]);
          if (item && (item & kTaskTag) == (ticket & kTaskTag)) break;   // this ticket's task
          item = 0ull;
          if (poll_word(&st->active) == 0u) break;                     // all lattices done
          if (poll_word(&st->status) & ST_TIMEOUT) break;
          if (poll_word(&st->cwork) == kCworkStop) break;              // stopped, drained
          const unsigned long long qt = poll_word(&st->qtail);
          if (qt != seen) {
            seen = qt;
            tw0 = clock64();
          }
          if (clock64() - tw0 > p.timeout_cycles) {
            stop_all(ST_TIMEOUT);
            break;
          }
          __nanosleep(nap);
          if (nap < 2048u) nap *= 2u;
        }
        if (item) atomicCAS(&p.q[slot], item, 0ull);
        __threadfence();
      }
      item = __shfl_sync(0xFFFFFFFFu, item, 0);
      if (!item) break;
      __syncwarp();          // every lane's reads come after lane 0's acquire
      const unsigned kind = (unsigned)((item >> 62) & 1ull);
      const int b = (int)((item >> 42) & 0xFFFFFull);
      const int c = (int)((item >> 20) & 0x3FFFFFull);
      const RepDesc* d = p.reps + b;
      LatState* Ls = p.ls + b;
      if (kind == 0u && warp_rep != b) {
        // the warp's rate table for this lattice (every lane has finished
        // with the last one: the item's shuffle above synchronised the warp)
        if (lane < 10) {
          g.PT[lane] = d->P[lane];
          g.PT[10 + lane] = d->Rp[lane];
        }
        __syncwarp();
        warp_rep = b;
      }
      g.cur_rep = warp_rep;
      const int loc = c * CH + lane;
      const bool mine = is_slot && lane < CH && loc < d->NR;
      const int r = d->off + loc;
      const unsigned cnt = (unsigned)__popc(__ballot_sync(0xFFFFFFFFu, mine));
      const unsigned w = poll_word(&Ls->w);
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
          compute_halo(p, lat_of(p, r), r, cnew);
        }
        fill_warp<GEN>(p, mine && w + 1u < (unsigned)d->nwin, r, (uint32_t)loc, d->key0, d->key1,
                       d->w0 + w + 1u);
        __syncwarp();        // every lane's writes come before lane 0's release
        int enq = -1;        // task kind the warp publishes next (-1: none)
        bool last = false;   // this task completed the window's commit
        const unsigned wn = w + 1u;
        if (lane == 0) {
          __threadfence();
          const unsigned old = atomicSub(&Ls->pend, cnt);
          if (old == cnt) {
            __threadfence();
            last = true;
            const unsigned n = poll_word(&Ls->n);      // iterations of window w
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
            atomicExch(&Ls->w, wn);
            rs->windows_done = wn;
            if (wn < (unsigned)d->nwin && !(poll_word(&st->status) & kStop)) {
              atomicExch(&Ls->n, 1u);
              atomicExch(&Ls->chg, 0u);
              atomicExch(&Ls->ovf, 0u);
              atomicExch(&Ls->pend, (unsigned)d->NR);
              atomicExch((unsigned long long*)&Ls->ts, (unsigned long long)__double_as_longlong(
                  __dadd_rn(__ldcg(&Ls->ts), d->Tw)));
              enq = 0;
            }
          }
        }
        enq = __shfl_sync(0xFFFFFFFFu, enq, 0);
        if (enq >= 0) enqueue_lattice(p, b, (unsigned)enq, CH, lane);
        if (lane == 0) {
          if (last) {
            __threadfence();
            if (wn == (unsigned)d->nwin) atomicSub(&st->active, 1u);
          }
          atomicAdd(&st->cwork, 0ull - (unsigned long long)cnt);
        }
      } else {
        // ---- iteration n of window w; after an error no new passes run
        // (one lane's read decides for the warp: the reductions below need every lane)
        if (__shfl_sync(0xFFFFFFFFu, poll_word(&st->status), 0) & kStop) continue;
        const unsigned n = poll_word(&Ls->n);
        const double t_s = __ldcg(&Ls->ts);
        const double t_end = __dadd_rn(t_s, d->Tw);
        Acc ra = {0u, 0u, 0u, 0u, 0u, 0u, false, false};
        if (mine) {
          const Lat lt = lat_of(p, r);
          const unsigned cidx = p.rcidx[r];
          if (MODE == 2)
            run_region<1, GEN>(p, lt, r, (int)n, cidx, t_s, t_end, d->w0 + w, g, ra);
          else
            run_region<0, GEN>(p, lt, r, (int)n, cidx, t_s, t_end, d->w0 + w, g, ra);
        }
        // the task's counters, reduced over the warp: one atomic per counter
        const unsigned t_ev = __reduce_add_sync(0xFFFFFFFFu, ra.events);
        const unsigned t_br = __reduce_add_sync(0xFFFFFFFFu, ra.breaks);
        const unsigned t_pa = __reduce_add_sync(0xFFFFFFFFu, ra.passes);
        const unsigned t_sk = __reduce_add_sync(0xFFFFFFFFu, ra.skips);
        const unsigned t_fm = __reduce_max_sync(0xFFFFFFFFu, ra.fmax);
        const unsigned t_em = __reduce_max_sync(0xFFFFFFFFu, ra.emax);
        const bool anych = __any_sync(0xFFFFFFFFu, mine && ra.changed);
        const bool anyov = __any_sync(0xFFFFFFFFu, mine && ra.overflow);
        __syncwarp();        // every lane's writes come before lane 0's release
        int enq = -1;        // task kind the warp publishes next (-1: none)
        if (lane == 0) {
          if (t_fm) atomicMax(&p.curf[(w & 1u) * p.nrep + b], t_fm);
          if (t_ev) atomicAdd(&rs->generated, (unsigned long long)t_ev);
          if (t_br) atomicAdd(&rs->breaks, (unsigned long long)t_br);
          if (t_fm) atomicMax(&rs->max_f, t_fm);
          if (t_em) atomicMax(&rs->max_win_events, t_em);
          if (t_pa) atomicAdd(&st->region_passes, (unsigned long long)t_pa);
          if (t_sk) atomicAdd(&st->region_skips, (unsigned long long)t_sk);
          if (anych) atomicOr(&Ls->chg, 1u);
          if (anyov) atomicOr(&Ls->ovf, 1u);
          __threadfence();
          const unsigned old = atomicSub(&Ls->pend, cnt);
          if (old == cnt) {
            __threadfence();
            const unsigned ch = poll_word(&Ls->chg);
            const unsigned ov = poll_word(&Ls->ovf);
            if (ov) {
              stop_all(ST_CAPACITY);
            } else if (!ch) {
              // no region of this lattice changed its lists: the fixed point;
              // commit tasks follow (the window's statistics count at their end)
              atomicExch(&Ls->pend, (unsigned)d->NR);
              const unsigned long long before = atomicAdd(&st->cwork, (unsigned long long)d->NR);
              if (before & kCworkStop)
                atomicAdd(&st->cwork, 0ull - (unsigned long long)d->NR);   // stopped: no commit
              else
                enq = 1;
            } else if ((int)n >= p.max_iters) {
              stop_all(ST_NOT_CONVERGED);
            } else if (!(poll_word(&st->status) & kStop)) {
              atomicExch(&Ls->n, n + 1u);
              atomicExch(&Ls->chg, 0u);
              atomicExch(&Ls->pend, (unsigned)d->NR);
              enq = 0;
            }
          }
        }
        enq = __shfl_sync(0xFFFFFFFFu, enq, 0);
        if (enq >= 0) enqueue_lattice(p, b, (unsigned)enq, CH, lane);
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
        run_region<0, GEN>(p, lt, r, n, cidx, t_s, t_end, wg, g, ra);
      else if (MODE == 2)
        run_region<1, GEN>(p, lt, r, n, cidx, t_s, t_end, wg, g, ra);
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
              carry_lists(p, r, n + 1u, lt.spans_x, lt.spans_y);
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
  if (y >= lt.H) {
    // rows past the lattice's region height stay empty
  } else if (mode == SR_INIT_ALL_UP) {
    word = (lt.W == 32) ? 0xFFFFFFFFu : ((1u << lt.W) - 1u);
  } else if (mode == SR_INIT_FAIR_COIN) {
    const uint32_t gy = (uint32_t)(ry * lt.H + y);
    for (int x = 0; x < lt.W; ++x) {
      const uint32_t site = gy * (uint32_t)lt.L + (uint32_t)(rx * lt.W + x);
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
  if (t >= (size_t)d.NR * d.H) return;
  const int loc = (int)(t % d.NR), y = (int)(t / d.NR);
  const int r = d.off + loc;
  const int rx = loc % d.NX, ry = loc / d.NX;
  const size_t base = (size_t)(ry * d.H + y) * d.L + (size_t)rx * d.W;
  uint32_t word = 0;
  for (int x = 0; x < d.W; ++x) word |= (uint32_t)(spins[base + x] > 0) << x;
  p.rows[(size_t)y * p.NR + r] = word;
}

// Committed spins of lattice b as an int8 L x L array.
__global__ void unpack_rows_kernel(KParams p, int b, int8_t* spins) {
  const RepDesc& d = p.reps[b];
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)d.L * d.L) return;
  const int gx = (int)(t % d.L), gy = (int)(t / d.L);
  const int r = d.off + (gy / d.H) * d.NX + gx / d.W;
  const uint32_t word = p.rows[((size_t)p.rcidx[r] * p.H + gy % d.H) * p.NR + r];
  spins[t] = ((word >> (gx % d.W)) & 1u) ? 1 : -1;
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
    const int W = d.W, H = d.H;
    const uint32_t wmask = (W == 32) ? 0xFFFFFFFFu : ((1u << W) - 1u);
    const uint32_t* rows_c = p.rows + (size_t)p.rcidx[r] * p.H * nr;
    const uint32_t hS = p.halo[1 * nr + r], hE = p.halo[3 * nr + r];
    for (int y = 0; y < H; ++y) {
      const uint32_t rw = rows_c[(size_t)y * nr + r];
      const uint32_t dn = (y < H - 1) ? rows_c[(size_t)(y + 1) * nr + r]
                                      : (d.spans_y ? rows_c[r] : hS);
      const uint32_t rbit = d.spans_x ? (rw & 1u) : (hE >> y) & 1u;
      const uint32_t rt = (rw >> 1) | (rbit << (W - 1));
      mag += 2 * __popc(rw) - W;
      bonds += (W - 2 * __popc((rw ^ rt) & wmask)) + (W - 2 * __popc((rw ^ dn) & wmask));
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
