// sr_region.cuh -- one region's pass over a window (§3, §5): the lane mapping
// (one region per lane) and the warp mapping (one region per warp).
#pragma once
#include "sr_state.cuh"

namespace sr {

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
// GEN = false compiles out score mode, the alternate step rule and the
// event trace (a smaller loop body for the common case); GEN = true reads
// them from the launch parameters.
template <int SOFT>
__device__ __forceinline__ double tau_any(double t_last, double x, double b, unsigned long long lam,
                                          const Lat& lt) {
  return SOFT ? tau_soft(t_last, x, b, lam, lt.F) : tau_hat(t_last, x, b, lam, lt.scale);
}
template <int SOFT>
__device__ __forceinline__ double accrue_any(double b, double tb, double tl, unsigned long long lam,
                                             const Lat& lt) {
  return SOFT ? sf::add_pos(b, sf::mul_pos(sf::u64_scaled(lam, lt.F), sf::sub_pos(tb, tl)))
              : accrue(b, tb, tl, lam, lt.scale);
}

template <int SOFT, bool GEN>
__device__ void run_region(const KParams& p, const Lat& lt, int r, int n_iter, unsigned cidx,
                           double t_s, double t_end, unsigned wg, Region& g, Acc& acc) {
  // the lattice's region shape; per-region arrays are laid out for the launch's
  // largest shape (p.H rows)
  const int W = lt.W, H = lt.H, NR = p.NR, HL = p.H;
  const bool score = GEN && p.score, fresh = GEN && p.fresh;
  const int tcap = GEN ? p.tcap : 0;
  g.set_shape(W, H);
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
  // (when the last iteration left the lists as the one before it did, both in
  // this window, the buffer of parity wp already holds them)
  auto carry_over = [&]() {
    const bool copy = n_iter < 3 || __ldcg(&p.chg[(size_t)rp * nr + r]) != 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (!has[e] || !copy) continue;
      const unsigned n = __ldcg(&p.hl[((size_t)rp * 4 + e) * nr + r]);
#pragma unroll 4
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
  const size_t rwords = (size_t)kRecHead + HL;
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
      g.PT[k * g.pts] = lt.P[k];
      g.PT[(10 + k) * g.pts] = lt.Rp[k];
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
    for (int y = 0; y < H; ++y) cp_async4(&g.rows[y * g.stride], &rec[kRecHead + y]);
  } else {
    // ---- committed state
    const uint32_t* rows_c = p.rows + (size_t)cidx * HL * nr;
    for (int y = 0; y < H; ++y) cp_async4(&g.rows[y * g.stride], &rows_c[(size_t)y * nr + r]);
    g.hN = p.halo[0 * nr + r];
    g.hS = p.halo[1 * nr + r];
    g.hW = p.halo[2 * nr + r];
    g.hE = p.halo[3 * nr + r];
    i = p.ci[cidx * nr + r];        // first event of the window
    // the carry of §5 "Subsequent steps", or (alternate rule) a clock that
    // restarts at the window start with no hazard accrued
    b = fresh ? 0.0 : p.cb[cidx * nr + r];
    tl = fresh ? t_s : p.ct[cidx * nr + r];
  }
  // presimulated pairs (U, V) of the coming events (§4: the random numbers
  // as a list drawn before use); the pair of event i+1 is loaded one event ahead
  const unsigned long long hi = p.rhi[r];
  const unsigned kmask = (unsigned)p.K - 1u;     // K is a power of two <= 4096
  // events past the ring are drawn here (alternate rule: numbered from the window start)
  auto draw_at = [&](unsigned long long ii, double& xx, unsigned long long& kk) {
    if (fresh)
      draw_event_fresh((unsigned)(ii - p.ci[cidx * nr + r]), wg, (uint32_t)lt.loc, lt.key0,
                       lt.key1, xx, kk);
    else
      draw_event(ii, (uint32_t)lt.loc, lt.key0, lt.key1, xx, kk);
  };
  if (!resume && !fresh) {
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
  cp_async_wait_all();               // the rows copied above
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
  if (score) {
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
  double tau = tau_any<SOFT>(tl, x, b, lam, lt);
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
        if (score)                     // score statistics of the event and its class moves
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
            // the comparison with the last iteration's list (§4, statement
            // (c)) takes no branch on its loads, so the event chain does not
            // wait for them; only the pass end reads the flag (an entry past
            // the old length is read but does not count)
            const size_t pa = (((size_t)rp * 4 + e) * cap + n) * nr + r;
            const unsigned differs =
                (unsigned)(n >= plen(e)) |
                (unsigned)(__double_as_longlong(__ldcg(&p.ht[pa])) != __double_as_longlong(tau)) |
                (unsigned)(__ldcg(&p.hp[pa]) != (uint8_t)pos);
            changed = changed | (differs != 0u);
            olen[e] = n + 1;
          }
        }
      }
      if (boundary) ++bevents;
      if (tcap > 0 && i < (unsigned long long)tcap) {
        p.trt[(size_t)r * tcap + i] = tau;
        p.trs[(size_t)r * tcap + i] =
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
      b = accrue_any<SOFT>(b, tb, tl, lam, lt);
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
      if (score) g.occ_move(cu_old, cu_new, to_fixed(tb, frac));
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
    tau = tau_any<SOFT>(tl, x, b, lam, lt);
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
  uint32_t* rows_t = p.rows + (size_t)tc * HL * nr;
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
  if (score) {
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
  const int W = lt.W, H = lt.H, HL = p.H;
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
  uint32_t row = vlane ? __ldcg(&p.rows[((size_t)cidx * HL + lane) * nr + r]) : 0u;
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
  const int F = lt.F;

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
  if (vlane) p.rows[((size_t)tc * HL + lane) * nr + r] = row;
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
    hN = __ldcg(&rows_c[(size_t)(lt.H - 1) * nr + qN]);
    hS = __ldcg(&rows_c[qS]);
  }
  if (!lt.spans_x) {
    const int qW = lt.off + ry * lt.NX + (rx + lt.NX - 1) % lt.NX;
    const int qE = lt.off + ry * lt.NX + (rx + 1) % lt.NX;
    for (int y = 0; y < lt.H; ++y) {
      hW |= ((__ldcg(&rows_c[(size_t)y * nr + qW]) >> (lt.W - 1)) & 1u) << y;
      hE |= (__ldcg(&rows_c[(size_t)y * nr + qE]) & 1u) << y;
    }
  }
  p.halo[0 * nr + r] = hN;
  p.halo[1 * nr + r] = hS;
  p.halo[2 * nr + r] = hW;
  p.halo[3 * nr + r] = hE;
}

// A region whose inputs for iteration n_new equal those of the last one keeps
// its tentative state; its lists are carried to the new parity.  When the last
// iteration left them as the one before it did (both in this window), the
// buffer of the new parity already holds them.
__device__ void carry_lists(const KParams& p, int r, unsigned n_new, bool spans_x, bool spans_y) {
  const size_t nr = (size_t)p.NR, cap = (size_t)p.cap;
  const int wp = (int)(n_new & 1u);
  const int rp = wp ^ 1;
  const bool copy = n_new < 3u || __ldcg(&p.chg[(size_t)rp * nr + r]) != 0;
  for (int e = 0; e < 4; ++e) {
    if ((e < 2 && spans_y) || (e >= 2 && spans_x) || !copy) continue;
    const unsigned n = __ldcg(&p.hl[((size_t)rp * 4 + e) * nr + r]);
#pragma unroll 4
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

}  // namespace sr
