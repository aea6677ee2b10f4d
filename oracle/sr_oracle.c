/*
 * sr_oracle.c -- CPU oracle for the synchronous-relaxation n-fold-way Ising
 * simulation (Lubachevsky & Weiss, "Synchronous Relaxation for Parallel Ising
 * Spin Simulations").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, sequential, obviously
 * correct reference that the CUDA path is checked against.  Only the tests,
 * the smoke check and the benchmark's CPU-baseline leg may load it.  It shares
 * no code, header, table or constant generator with the CUDA library.
 *
 * What it computes: the exact continuous-time trajectory that a converged
 * synchronous relaxation must reproduce.  Every region is its own n-fold-way
 * process (§3) whose i-th event consumes the i-th pair (U_i, V_i) of its own
 * presimulated random list (§4, last paragraphs; §5 "Subsequent iterations").
 * Instead of iterating to a fixed point, the oracle processes the events of all
 * regions in global time order (a plain discrete-event simulation), so each
 * region always sees the true history of its neighbours.  A neighbour's flip is
 * a break point of the region's piecewise-constant total rate (§5, Eqs.
 * 5.2-5.6).
 *
 * Readings of the paper taken here (each is also listed in the design notes):
 *  R1  Eq. 2.1 counts each nearest-neighbour bond once; k_B = 1; H is h.
 *      Delta E(v) = 2 s(v) (J * sum_nb s(v') + h).
 *  R2  lambda = 1 (§3): an atom of class k flips at rate p_k.
 *  R3  Ten classes k = 5*[s=+1] + n_up (n_up = number of up neighbours),
 *      scanned in order k = 0..9 (§3, the 2 x 5 classes).
 *  R4  Rates are held on a fixed-point grid: P_k = round(p_k * 2^F) with
 *      F = 63 - bitlen(sites per region), so the total rate
 *      Lambda = sum_k N_k p_k (Eq. 3.3) is an exact integer multiple of 2^-F.
 *  R5  Class and site selection (Eqs. 3.5-3.8) are evaluated exactly: with
 *      V = (2 kV + 1) 2^-53, class k* is the unique k with
 *      A(k-1) < V*Lambda <= A(k), A(k) = sum_{j<=k} N_j p_j; the 0-based
 *      position within the class is floor((V*Lambda - A(k*-1)) / p_k*),
 *      i.e. the access index of Eq. 3.8 minus one, clamped to N_k* - 1.
 *  R6  The linear order inside a class (§3, Phase 3) is row-major order of the
 *      sites inside the region.
 *  R7  U = (2 kU + 1) 2^-53 and -log U uses a fixed artanh series (below).
 *  R8  Waiting time with break points (Eqs. 3.4, 5.2-5.6): each region keeps
 *      x = -log U_i, b = integral of Lambda since its last event up to t_last,
 *      and the candidate time tau = t_last + max(x - b, 0) / Lambda(t_last).
 *      A neighbour flip at t_b < tau is a break point:
 *      b <- b + Lambda * (t_b - t_last), t_last <- t_b.
 *      If tau rounds to a value <= t_last it becomes the next double above
 *      t_last, so a region's event times are strictly increasing.
 *  R9  An event at time tau sees every neighbour flip with time < tau and none
 *      with time >= tau; events of different regions at the same time are
 *      simultaneous (each selects with the state before the others' flips).
 * R10  Window ends are not break points: an event is committed in the window
 *      [t_c, t_c + T) iff tau < t_c + T (Eq. in §5, "t_c <= tau_1 < ... <
 *      tau_m < t_c + T_max"); the clock state carries over unchanged (§5,
 *      "Subsequent steps").
 * R11  Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with
 *      key = (seed_lo, seed_hi) and counter = (i_lo, i_hi, region, 0) for the
 *      i-th event of a region, counter = (site, 0, 0, 1) for the fair-coin
 *      initial spin of a site.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------ */
/* Philox4x32-10, written from the definition in Salmon et al. (SC'11): */
/* ten rounds of two 32x32->64 multiplies with the counter words xored  */
/* with the key, the key bumped by the Weyl constants between rounds.   */
/* ------------------------------------------------------------------ */
static const uint32_t PHILOX_M0 = 0xD2511F53u;
static const uint32_t PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u;
static const uint32_t PHILOX_W1 = 0xBB67AE85u;

ORC_EXPORT void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; round++) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += PHILOX_W0;
    k1 += PHILOX_W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------ */
/* Uniform (0,1) numbers and the fixed logarithm (reading R7).          */
/* ------------------------------------------------------------------ */

/* U = (2k+1) * 2^-53 for a 52-bit integer k: exactly representable, never 0 or 1. */
ORC_EXPORT double orc_unit_from_bits(uint64_t k52) {
  return ldexp((double)(2 * k52 + 1), -53);
}

/* -ln U for U = (2k+1) 2^-53, with IEEE double add/mul/div only:
 *   u = 2k+1 = 2^e * m with m in [sqrt(1/2), sqrt(2)),
 *   ln m = 2 artanh(s) = 2 (s + s^3/3 + ... + s^21/21), s = (m-1)/(m+1),
 *   evaluated by Horner in z = s^2 from the highest coefficient down,
 *   ln U = (e - 53) ln 2 + ln m.
 * |s| <= 0.1716, so the omitted tail is below 1e-18 relative. */
ORC_EXPORT double orc_neglog_unit(uint64_t k52) {
  uint64_t u = 2 * k52 + 1;
  int e = 0;
  while ((u >> e) > 1) e++;            /* u in [2^e, 2^(e+1)) */
  double m = ldexp((double)u, -e);     /* exact, m in [1, 2) */
  if (m >= 1.4142135623730951) {       /* nearest double to sqrt(2) */
    m = m * 0.5;
    e = e + 1;
  }
  double s = (m - 1.0) / (m + 1.0);
  double z = s * s;
  double poly = 1.0 / 21.0;
  for (int j = 9; j >= 0; j--) {
    poly = poly * z + 1.0 / (double)(2 * j + 1);
  }
  double ln_m = 2.0 * (s * poly);
  double ln_u = (double)(e - 53) * 0.6931471805599453 + ln_m;
  return -ln_u;
}

/* ------------------------------------------------------------------ */
/* Rates (Eqs. 2.2, 2.3) and their fixed-point grid (reading R4).       */
/* ------------------------------------------------------------------ */

/* p_k for k = 5*[s=+1] + n_up.  glauber = 0: p = min(1, theta) (Eq. 2.2);
 * glauber = 1: p = theta / (1 + theta) (Eq. 2.3); theta = exp(-dE/T). */
ORC_EXPORT void orc_rates(double J, double h, double T, int glauber, double p[10]) {
  for (int k = 0; k < 10; k++) {
    int s = (k >= 5) ? 1 : -1;
    int n_up = k % 5;
    int nb_sum = 2 * n_up - 4;                       /* sum of the 4 neighbour spins */
    double dE = 2.0 * (double)s * (J * (double)nb_sum + h);
    double theta = exp(-dE / T);
    if (glauber) {
      p[k] = theta / (1.0 + theta);
    } else {
      p[k] = theta < 1.0 ? theta : 1.0;
    }
  }
}

ORC_EXPORT int orc_frac_bits(int sites) {
  int bl = 0;
  while ((sites >> bl) > 0) bl++;
  return 63 - bl;
}

ORC_EXPORT void orc_rates_fixed(const double p[10], int F, uint64_t P[10]) {
  for (int k = 0; k < 10; k++) P[k] = (uint64_t)nearbyint(ldexp(p[k], F));
}

/* ------------------------------------------------------------------ */
/* Exact class and site selection (Eqs. 3.5-3.8, reading R5).           */
/* ------------------------------------------------------------------ */

/* Returns k* and writes the 0-based position within class k*.  N: class
 * counts, P: fixed-point rates, kV: the 52-bit integer of V.  Requires
 * Lambda > 0.  Plain definition: multiply the inequalities of Eq. 3.6 by
 * Lambda * 2^(53+F) so that every quantity is an integer. */
ORC_EXPORT int orc_select(const int N[10], const uint64_t P[10], uint64_t kV, uint64_t* pos_out) {
  unsigned __int128 lam = 0;
  for (int k = 0; k < 10; k++) lam += (unsigned __int128)N[k] * P[k];
  unsigned __int128 target = (unsigned __int128)(2 * kV + 1) * lam;   /* V*Lambda * 2^(53+F) */
  unsigned __int128 a_prev = 0;                                        /* A(k-1) * 2^F */
  for (int k = 0; k < 10; k++) {
    unsigned __int128 a_k = a_prev + (unsigned __int128)N[k] * P[k];
    if ((a_prev << 53) < target && target <= (a_k << 53)) {
      unsigned __int128 num = target - (a_prev << 53);
      unsigned __int128 den = (unsigned __int128)P[k] << 53;
      unsigned __int128 j = num / den;
      if (j > (unsigned __int128)(N[k] - 1)) j = (unsigned __int128)(N[k] - 1);
      *pos_out = (uint64_t)j;
      return k;
    }
    a_prev = a_k;
  }
  *pos_out = 0;
  return -1;
}

/* ------------------------------------------------------------------ */
/* Waiting time with break points (Eqs. 3.4, 5.2-5.6, reading R8).      */
/* ------------------------------------------------------------------ */

static double next_up(double t) {        /* next double above a finite t >= 0 */
  uint64_t bits;
  memcpy(&bits, &t, 8);
  bits += 1;
  memcpy(&t, &bits, 8);
  return t;
}

ORC_EXPORT double orc_lambda(uint64_t lam_fixed, int F) {
  return ldexp((double)lam_fixed, -F);
}

ORC_EXPORT double orc_tau(double t_last, double x, double b, uint64_t lam_fixed, int F) {
  if (lam_fixed == 0) return INFINITY;
  double lam = orc_lambda(lam_fixed, F);
  double d = x - b;
  if (d < 0.0) d = 0.0;
  double tau = t_last + d / lam;
  if (!(tau > t_last)) tau = next_up(t_last);
  return tau;
}

/* ------------------------------------------------------------------ */
/* The global-time-order discrete-event simulation.                     */
/* ------------------------------------------------------------------ */

typedef struct {
  int L;
  double J, h, T;
  int region_w, region_h;     /* region extent in x and y */
  uint64_t seed;
  int init_mode;              /* 0 fair coin (Philox INIT stream), 1 all +1, 2 all -1, 3 given spins */
  int glauber;                /* 0 Metropolis (Eq. 2.2), 1 Glauber (Eq. 2.3) */
  int debug;                  /* check the invariants after every event */
  int fresh_steps;            /* 0: the carry of §5 "Subsequent steps"; 1: §5 "An alternate
                                 approach to subsequent steps" -- at every window end all
                                 clocks restart with new random numbers */
} orc_params;

/* Caller-owned output buffers; any pointer may be NULL. */
typedef struct {
  int8_t* spins;              /* [n_windows][L*L] spins at each window end */
  uint64_t* counts;           /* [n_windows][n_regions] events of each region so far */
  int64_t* mag;               /* [n_windows] sum of spins at each window end */
  int64_t* bonds;             /* [n_windows] sum over bonds of s s' at each window end */
  double* int_mag;            /* [n_windows] integral of the spin sum from 0 */
  double* int_bonds;          /* [n_windows] integral of the bond sum from 0 */
  /* final per-region clock state (the carry of §5, "Subsequent steps") */
  uint64_t* carry_i;          /* [n_regions] index of the pending event */
  double* carry_x;            /* [n_regions] -log U of the pending event */
  double* carry_b;            /* [n_regions] integral of Lambda since the last event */
  double* carry_t;            /* [n_regions] time up to which b is taken */
  /* committed events in processing order */
  int64_t trace_cap;
  int64_t trace_len;          /* written: number of events (may exceed trace_cap) */
  uint32_t* tr_region;
  uint64_t* tr_index;
  double* tr_time;
  uint32_t* tr_site;          /* global site index y*L + x */
  int64_t debug_failures;     /* written: invariant violations seen */
  /* the path's sufficient statistics for its score function (log-likelihood
   * sum_events log p_k - integral sum_k N_k p_k dt, §3 rates): */
  uint64_t* ev_class;         /* [n_regions][10] committed events by the class of the flipped
                                 site before its flip */
  double* occupancy;          /* [n_regions][10] integral of N_k over [0, t_end[last]] */
} orc_outputs;

typedef struct {
  int L, rw, rh, nrx, nry, nreg, F;
  uint64_t P[10];
  uint32_t key[2];
  int fresh;                  /* the alternate step rule */
  uint32_t window;            /* index of the running window (alternate rule) */
  uint64_t* ev0;              /* per-region event index at the window start (alternate rule) */
  int8_t* s;                  /* spins, y*L + x */
  int8_t* cls;                /* class of every site */
  int (*N)[10];               /* per-region class counts */
  uint64_t* lam;              /* per-region Lambda on the grid */
  uint64_t* ev;               /* per-region pending event index */
  double* x;
  uint64_t* kv;
  double* b;
  double* tl;
  double* tau;
  int* heap;                  /* binary min-heap of regions keyed by (tau, region) */
  int* hpos;
  int64_t mag, bonds;
  double* tseg;               /* per region: time of its last class change (occupancy) */
  double (*occ)[10];          /* per region: integral of N_k dt so far */
  uint64_t (*evc)[10];        /* per region: events by class */
} orc_state;

static int site_region(const orc_state* st, int site) {
  int x = site % st->L, y = site / st->L;
  return (y / st->rh) * st->nrx + (x / st->rw);
}

static int nb_site(const orc_state* st, int site, int dir) {
  int L = st->L, x = site % L, y = site / L;
  switch (dir) {   /* neighbour order as listed in §2: (i+1,j), (i-1,j), (i,j+1), (i,j-1) */
    case 0: x = (x + 1) % L; break;
    case 1: x = (x + L - 1) % L; break;
    case 2: y = (y + 1) % L; break;
    default: y = (y + L - 1) % L; break;
  }
  return y * L + x;
}

static int class_of(const orc_state* st, int site) {
  int n_up = 0;
  for (int d = 0; d < 4; d++) n_up += st->s[nb_site(st, site, d)] > 0;
  return 5 * (st->s[site] > 0) + n_up;
}

static uint64_t region_lambda(const orc_state* st, int r) {
  uint64_t lam = 0;
  for (int k = 0; k < 10; k++) lam += (uint64_t)st->N[r][k] * st->P[k];
  return lam;
}

/* The pair (U, V) of region r's pending event.  Carry rule: counter
 * (i_lo, i_hi, r, 0) for event index i.  Alternate rule: the j-th event of
 * window w takes counter (j, w, r, 2), numbers no earlier window has used. */
static void draw(orc_state* st, int r) {
  uint32_t ctr[4] = {(uint32_t)st->ev[r], (uint32_t)(st->ev[r] >> 32), (uint32_t)r, 0u};
  if (st->fresh) {
    ctr[0] = (uint32_t)(st->ev[r] - st->ev0[r]);
    ctr[1] = st->window;
    ctr[3] = 2u;
  }
  uint32_t w[4];
  orc_philox4x32_10(ctr, st->key, w);
  uint64_t ku = ((((uint64_t)w[1]) << 32) | w[0]) >> 12;
  uint64_t kv = ((((uint64_t)w[3]) << 32) | w[2]) >> 12;
  st->x[r] = orc_neglog_unit(ku);
  st->kv[r] = kv;
}

static int heap_less(const orc_state* st, int a, int b) {
  if (st->tau[a] != st->tau[b]) return st->tau[a] < st->tau[b];
  return a < b;
}
static void heap_swap(orc_state* st, int i, int j) {
  int a = st->heap[i], b = st->heap[j];
  st->heap[i] = b; st->heap[j] = a;
  st->hpos[b] = i; st->hpos[a] = j;
}
static void heap_sift_down(orc_state* st, int i) {
  int n = st->nreg;
  for (;;) {
    int l = 2 * i + 1, r = l + 1, m = i;
    if (l < n && heap_less(st, st->heap[l], st->heap[m])) m = l;
    if (r < n && heap_less(st, st->heap[r], st->heap[m])) m = r;
    if (m == i) break;
    heap_swap(st, i, m);
    i = m;
  }
}
/* Restore the heap after the key of the entry at position i changed. */
static void heap_fix(orc_state* st, int i) {
  while (i > 0 && heap_less(st, st->heap[i], st->heap[(i - 1) / 2])) {
    heap_swap(st, i, (i - 1) / 2);
    i = (i - 1) / 2;
  }
  heap_sift_down(st, i);
}

/* Site of class k whose 0-based row-major rank among class-k sites of region r is pos (R6). */
static int site_of_rank(const orc_state* st, int r, int k, uint64_t pos) {
  int x0 = (r % st->nrx) * st->rw, y0 = (r / st->nrx) * st->rh;
  uint64_t seen = 0;
  for (int y = y0; y < y0 + st->rh; y++)
    for (int x = x0; x < x0 + st->rw; x++) {
      int site = y * st->L + x;
      if (st->cls[site] == k) {
        if (seen == pos) return site;
        seen++;
      }
    }
  return -1;
}

static int64_t count_debug(const orc_state* st) {
  int64_t bad = 0;
  int L = st->L;
  int64_t mag = 0, bonds = 0;
  int* Nc = calloc((size_t)st->nreg * 10, sizeof(int));
  for (int site = 0; site < L * L; site++) {
    int c = class_of(st, site);
    if (c != st->cls[site]) bad++;
    Nc[site_region(st, site) * 10 + c]++;
    mag += st->s[site];
    bonds += st->s[site] * st->s[nb_site(st, site, 0)] + st->s[site] * st->s[nb_site(st, site, 2)];
  }
  for (int r = 0; r < st->nreg; r++) {
    int tot = 0;
    for (int k = 0; k < 10; k++) {
      if (Nc[r * 10 + k] != st->N[r][k]) bad++;
      tot += st->N[r][k];
    }
    if (tot != st->rw * st->rh) bad++;
    if (region_lambda(st, r) != st->lam[r]) bad++;
  }
  if (mag != st->mag || bonds != st->bonds) bad++;
  free(Nc);
  return bad;
}

/* Flip one site and keep classes, counts, Lambda, magnetisation and bond sum current. */
static void flip_site(orc_state* st, int site) {
  int touched[5];
  touched[0] = site;
  for (int d = 0; d < 4; d++) touched[d + 1] = nb_site(st, site, d);
  int nb_sum = 0;
  for (int d = 0; d < 4; d++) nb_sum += st->s[touched[d + 1]];
  st->bonds -= 2 * (int64_t)st->s[site] * nb_sum;
  st->mag -= 2 * (int64_t)st->s[site];
  st->s[site] = (int8_t)(-st->s[site]);
  for (int j = 0; j < 5; j++) {
    int v = touched[j];
    int r = site_region(st, v);
    int old = st->cls[v], now = class_of(st, v);
    if (old == now) continue;
    st->N[r][old]--;
    st->N[r][now]++;
    st->cls[v] = (int8_t)now;
    st->lam[r] = st->lam[r] - st->P[old] + st->P[now];
  }
}

static void record_window(const orc_state* st, orc_outputs* out, int w, double int_mag, double int_bonds) {
  int L = st->L;
  if (out->spins) memcpy(out->spins + (size_t)w * L * L, st->s, (size_t)L * L);
  if (out->counts)
    for (int r = 0; r < st->nreg; r++) out->counts[(size_t)w * st->nreg + r] = st->ev[r];
  if (out->mag) out->mag[w] = st->mag;
  if (out->bonds) out->bonds[w] = st->bonds;
  if (out->int_mag) out->int_mag[w] = int_mag;
  if (out->int_bonds) out->int_bonds[w] = int_bonds;
}

/* Run from t = 0 through the window ends t_end[0] < t_end[1] < ...  Returns 0,
 * or a negative number on bad arguments / allocation failure. */
ORC_EXPORT int orc_run(const orc_params* prm, const int8_t* init_spins, int n_windows,
                       const double* t_end, orc_outputs* out) {
  int L = prm->L;
  if (L < 3 || prm->region_w < 1 || prm->region_h < 1 || L % prm->region_w || L % prm->region_h)
    return -1;
  if (!(prm->T > 0.0)) return -1;
  if (prm->init_mode == 3 && !init_spins) return -1;
  orc_state st;
  memset(&st, 0, sizeof st);
  st.L = L;
  st.rw = prm->region_w;
  st.rh = prm->region_h;
  st.nrx = L / st.rw;
  st.nry = L / st.rh;
  st.nreg = st.nrx * st.nry;
  st.F = orc_frac_bits(st.rw * st.rh);
  double p[10];
  orc_rates(prm->J, prm->h, prm->T, prm->glauber, p);
  orc_rates_fixed(p, st.F, st.P);
  st.key[0] = (uint32_t)prm->seed;
  st.key[1] = (uint32_t)(prm->seed >> 32);
  st.fresh = prm->fresh_steps != 0;
  st.window = 0;
  size_t nsite = (size_t)L * L, nreg = (size_t)st.nreg;
  st.s = malloc(nsite);
  st.cls = malloc(nsite);
  st.N = calloc(nreg, sizeof *st.N);
  st.lam = calloc(nreg, 8);
  st.ev = calloc(nreg, 8);
  st.ev0 = calloc(nreg, 8);
  st.tseg = calloc(nreg, 8);
  st.occ = calloc(nreg, sizeof *st.occ);
  st.evc = calloc(nreg, sizeof *st.evc);
  st.x = calloc(nreg, 8);
  st.kv = calloc(nreg, 8);
  st.b = calloc(nreg, 8);
  st.tl = calloc(nreg, 8);
  st.tau = calloc(nreg, 8);
  st.heap = calloc(nreg, sizeof(int));
  st.hpos = calloc(nreg, sizeof(int));
  int* tie = calloc(nreg, sizeof(int));
  int* chosen = calloc(nreg, sizeof(int));
  int* mark = calloc(nreg, sizeof(int));
  int* touched_regions = calloc(nreg * 3 + 8, sizeof(int));
  int rc = 0;
  if (!st.s || !st.cls || !st.N || !st.lam || !st.ev || !st.ev0 || !st.tseg || !st.occ ||
      !st.evc || !st.x || !st.kv || !st.b || !st.tl ||
      !st.tau || !st.heap || !st.hpos || !tie || !chosen || !mark || !touched_regions) {
    rc = -2;
    goto done;
  }

  /* initial spins */
  for (size_t site = 0; site < nsite; site++) {
    int8_t v;
    switch (prm->init_mode) {
      case 0: {
        uint32_t ctr[4] = {(uint32_t)site, 0u, 0u, 1u}, w[4];
        orc_philox4x32_10(ctr, st.key, w);
        v = (w[0] & 1u) ? 1 : -1;
        break;
      }
      case 1: v = 1; break;
      case 2: v = -1; break;
      default: v = init_spins[site] > 0 ? 1 : -1; break;
    }
    st.s[site] = v;
  }
  st.mag = 0;
  st.bonds = 0;
  for (size_t site = 0; site < nsite; site++) {
    int c = class_of(&st, (int)site);
    st.cls[site] = (int8_t)c;
    st.N[site_region(&st, (int)site)][c]++;
    st.mag += st.s[site];
    st.bonds += st.s[site] * st.s[nb_site(&st, (int)site, 0)] + st.s[site] * st.s[nb_site(&st, (int)site, 2)];
  }
  for (int r = 0; r < st.nreg; r++) {
    st.lam[r] = region_lambda(&st, r);
    st.ev[r] = 0;
    draw(&st, r);
    st.b[r] = 0.0;
    st.tl[r] = 0.0;
    st.tau[r] = orc_tau(st.tl[r], st.x[r], st.b[r], st.lam[r], st.F);
    st.heap[r] = r;
    st.hpos[r] = r;
  }
  for (int i = st.nreg / 2; i >= 0; i--) heap_sift_down(&st, i);   /* bottom-up heap build */
  out->trace_len = 0;
  out->debug_failures = 0;
  if (prm->debug) out->debug_failures += count_debug(&st);

  double int_mag = 0.0, int_bonds = 0.0, t_prev = 0.0;
  for (int w = 0; w < n_windows; w++) {
    double te = t_end[w];
    for (;;) {
      double t = st.tau[st.heap[0]];
      if (!(t < te)) break;
      /* the tie set: every region whose next event is at exactly t (R9) */
      int nt = 0;
      while (st.tau[st.heap[0]] == t) {
        int r = st.heap[0];
        tie[nt++] = r;
        st.tau[r] = INFINITY;          /* parked until recomputed below */
        heap_fix(&st, 0);
        if (nt == st.nreg) break;
      }
      /* select every site with the state before any flip at t (Eqs. 3.5-3.8) */
      for (int j = 0; j < nt; j++) {
        int r = tie[j];
        uint64_t pos;
        int k = orc_select(st.N[r], st.P, st.kv[r], &pos);
        chosen[j] = (k < 0) ? -1 : site_of_rank(&st, r, k, pos);
      }
      /* observables integrate the piecewise-constant path */
      int_mag += (double)st.mag * (t - t_prev);
      int_bonds += (double)st.bonds * (t - t_prev);
      t_prev = t;
      /* every region whose rate may change at t is first advanced to t with
       * its rate before the change (break point, Eqs. 5.2-5.4) */
      int ntr = 0;
      for (int j = 0; j < nt; j++) {
        int site = chosen[j];
        if (site < 0) continue;
        for (int d = -1; d < 4; d++) {
          int v = d < 0 ? site : nb_site(&st, site, d);
          int q = site_region(&st, v);
          if (!mark[q]) { mark[q] = 1; touched_regions[ntr++] = q; }
        }
      }
      for (int j = 0; j < nt; j++) mark[tie[j]] = 2;   /* own events reset b below */
      /* occupancy integrals of every region whose classes change at t */
      for (int a = 0; a < ntr; a++) {
        int q = touched_regions[a];
        for (int k = 0; k < 10; k++) st.occ[q][k] += (double)st.N[q][k] * (t - st.tseg[q]);
        st.tseg[q] = t;
      }
      /* events by the class of the flipped site, before any flip at t */
      for (int j = 0; j < nt; j++)
        if (chosen[j] >= 0) st.evc[tie[j]][st.cls[chosen[j]]] += 1;
      for (int a = 0; a < ntr; a++) {
        int q = touched_regions[a];
        if (mark[q] == 1) {
          double lam = orc_lambda(st.lam[q], st.F);
          st.b[q] = st.b[q] + lam * (t - st.tl[q]);
          st.tl[q] = t;
        }
      }
      for (int j = 0; j < nt; j++) {
        if (chosen[j] >= 0) flip_site(&st, chosen[j]);
      }
      for (int j = 0; j < nt; j++) {
        int r = tie[j];
        if (chosen[j] >= 0) {
          int64_t n = out->trace_len;
          if (n < out->trace_cap) {
            if (out->tr_region) out->tr_region[n] = (uint32_t)r;
            if (out->tr_index) out->tr_index[n] = st.ev[r];
            if (out->tr_time) out->tr_time[n] = t;
            if (out->tr_site) out->tr_site[n] = (uint32_t)chosen[j];
          }
          out->trace_len = n + 1;
        }
        st.ev[r] += 1;
        draw(&st, r);
        st.b[r] = 0.0;
        st.tl[r] = t;
      }
      /* new candidate times for every region whose state changed */
      for (int a = 0; a < ntr; a++) {
        int q = touched_regions[a];
        mark[q] = 0;
        st.tau[q] = orc_tau(st.tl[q], st.x[q], st.b[q], st.lam[q], st.F);
        heap_fix(&st, st.hpos[q]);
      }
      for (int j = 0; j < nt; j++) {
        int r = tie[j];
        if (chosen[j] >= 0) continue;   /* already in touched_regions */
        mark[r] = 0;
        st.tau[r] = orc_tau(st.tl[r], st.x[r], st.b[r], st.lam[r], st.F);
        heap_fix(&st, st.hpos[r]);
      }
      if (prm->debug) out->debug_failures += count_debug(&st);
    }
    int_mag += (double)st.mag * (te - t_prev);
    int_bonds += (double)st.bonds * (te - t_prev);
    t_prev = te;
    for (int r = 0; r < st.nreg; r++) {
      for (int k = 0; k < 10; k++) st.occ[r][k] += (double)st.N[r][k] * (te - st.tseg[r]);
      st.tseg[r] = te;
    }
    record_window(&st, out, w, int_mag, int_bonds);
    if (st.fresh && w + 1 < n_windows) {
      /* the alternate rule: wipe the slate at t_c = te; every region's clock
       * restarts there with the first pair of the next window's numbers
       * (exponential waiting times are memoryless, so the law is unchanged) */
      st.window = (uint32_t)(w + 1);
      for (int r = 0; r < st.nreg; r++) {
        st.ev0[r] = st.ev[r];
        draw(&st, r);
        st.b[r] = 0.0;
        st.tl[r] = te;
        st.tau[r] = orc_tau(st.tl[r], st.x[r], st.b[r], st.lam[r], st.F);
        st.heap[r] = r;
        st.hpos[r] = r;
      }
      for (int i = st.nreg / 2; i >= 0; i--) heap_sift_down(&st, i);
    }
  }
  for (int r = 0; r < st.nreg; r++) {
    for (int k = 0; k < 10; k++) {
      if (out->ev_class) out->ev_class[(size_t)r * 10 + k] = st.evc[r][k];
      if (out->occupancy) out->occupancy[(size_t)r * 10 + k] = st.occ[r][k];
    }
    if (out->carry_i) out->carry_i[r] = st.ev[r];
    if (out->carry_x) out->carry_x[r] = st.x[r];
    if (out->carry_b) out->carry_b[r] = st.b[r];
    if (out->carry_t) out->carry_t[r] = st.tl[r];
  }
done:
  free(st.s); free(st.cls); free(st.N); free(st.lam); free(st.ev); free(st.ev0); free(st.tseg);
  free(st.occ); free(st.evc); free(st.x);
  free(st.kv);
  free(st.b); free(st.tl); free(st.tau); free(st.heap); free(st.hpos);
  free(tie); free(chosen); free(mark); free(touched_regions);
  return rc;
}
