/*
 * qisg_oracle.c -- plain, slow CPU oracle for the MCQSG hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library may link, load
 * or call this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header or table with the CUDA
 * path: it rebuilds every table it needs from the formulas below.
 *
 * What it computes (the paper's notation):
 *   - the Trotter-Suzuki classical model of Eq. (2)-(3) (Sec. 1): spins
 *     S_{x,tau} = +-1 on an L x L x L_tau prism, periodic in x and y and
 *     periodic or antiperiodic in tau (Sec. 1: S_{x,L_tau} = +-S_{x,0}, so the
 *     antiperiodic wrap bond enters Eq. (3) as -S_{x,L_tau-1} S_{x,0}),
 *     with spatial bonds k*J_xy (J = +-1) and imaginary-time bonds k_tau.
 *     The paper's single coupling k is generalised to a (k, k_tau) pair per
 *     ladder slot, exp(-2 k_tau) = tanh(k Gamma); k_tau = k recovers the
 *     equal-coupling relation of Sec. 1.
 *   - checkerboard Metropolis (Sec. 2.1): red sites (x+y+tau even), then
 *     blue; the Metropolis factor is precomputed for every local energy
 *     class (Sec. 2.1) as a uint32 threshold built in FP64.
 *   - parallel tempering (Sec. 2.1): adjacent slots s, s+1 exchange their
 *     configurations with probability min(1, exp(Dk*DA + Dk_tau*DB)).
 *   - observables: integer energies and the replica overlap (Appendix E.1).
 *   - Philox4x32-10 (Sec. 2.1.1), the counter-based generator of Salmon et
 *     al. (SC'11), written here from its published definition.
 *   - the paper's own update rule (Sec. 2.1 and 2.1.1, Appendices B and C),
 *     for equal couplings k_tau = k: multi-site coding puts 32 tau-sites of
 *     one system in a word (site (x, y, tau) is bit
 *     tau / M of word (x, y, tau mod M), M = L_tau / 32), and a flip is taken
 *     iff u + d >= 3, with u the number of unsatisfied bonds of the site
 *     (0..6) and d the site's two-bit Ito-Kanada daemon.  The daemon is the
 *     number of leading ones in the bits (b4, b8, b12) of three words whose
 *     bits are independent and set with probability e^{-4k}; each byte of
 *     such a word is the inverse-cumulative image of a 64-bit "50/50" word
 *     whose upper half comes from Philox4x32-10 and lower half from one
 *     xoroshiro128++ state step (Blackman and Vigna, 2019) of the same
 *     Philox output.
 *
 * Storage is one int8 spin per (sample, replica, walker, site); every loop
 * runs in plain order.  Floating point is IEEE double with no contraction
 * (compile with -ffp-contract=off).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Philox counter domains: one per kind of draw. */
enum { ORC_DOM_J = 1, ORC_DOM_INIT = 2, ORC_DOM_SWEEP = 3, ORC_DOM_PT = 4, ORC_DOM_DAEMON = 5 };

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Sec. 2.1.1; Salmon, Moraes, Dror, Shaw, SC'11).            */
/* One round: (hi0,lo0) = M0*c0, (hi1,lo1) = M1*c2,                          */
/*   c' = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key is bumped by the  */
/*   Weyl constants between rounds.                                          */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    int round;
    for (round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Philox4x32-10 of n counters ctr[n][4] under one key (out[n][4]). */
void orc_philox4x32_10_many(int64_t n, const uint32_t *ctr, const uint32_t key[2], uint32_t *out)
{
    int64_t i;
    for (i = 0; i < n; ++i) orc_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

static uint32_t philox_word(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                            uint64_t seed, int which)
{
    uint32_t ctr[4], key[2], out[4];
    ctr[0] = c0; ctr[1] = c1; ctr[2] = c2; ctr[3] = c3;
    key[0] = (uint32_t)seed; key[1] = (uint32_t)(seed >> 32);
    orc_philox4x32_10(ctr, key, out);
    return out[which];
}

/* ------------------------------------------------------------------------ */
/* Ladder and tables (host FP64).                                           */
/* ------------------------------------------------------------------------ */

/* k_s linear in [lo, hi] (both ends included), k_tau from exp(-2 k_tau) =
 * tanh(k Gamma) (Sec. 1, generalised to a separate imaginary-time coupling). */
void orc_ladder_linear(double lo, double hi, int n, double gamma, double *k, double *ktau)
{
    int s;
    for (s = 0; s < n; ++s) {
        k[s] = (n == 1) ? lo : lo + (hi - lo) * (double)s / (double)(n - 1);
        ktau[s] = -0.5 * log(tanh(k[s] * gamma));
    }
}

/* Log Metropolis factor of flipping a spin with u_s unsatisfied spatial bonds
 * (of 4) and u_t unsatisfied imaginary-time bonds (of 2): flipping turns
 * satisfied bonds into unsatisfied ones and back, so the weight
 * exp(k*A + k_tau*B) changes by exp(-4k(2-u_s) - 4k_tau(1-u_t)). */
static double log_metropolis_factor(double k, double ktau, int us, int ut)
{
    double spatial = (double)(4 * (2 - us)) * k;     /* exact: 8k, 4k, 0, ... */
    double temporal = (double)(4 * (1 - ut)) * ktau; /* exact: 4k_tau, 0, ... */
    return -spatial - temporal;
}

/* T[s][u_s][u_t]: flip iff T == 0xFFFFFFFF or R < T, R a uniform uint32.
 * p = min(1, e^Delta); T = 0xFFFFFFFF when p >= 1, else
 * min(0xFFFFFFFE, floor(p * 2^32)), so P(flip) lies in [p - 2^-32, p].     */
void orc_thresholds(int n_slots, const double *k, const double *ktau, uint32_t *T)
{
    int s, us, ut;
    for (s = 0; s < n_slots; ++s)
        for (us = 0; us <= 4; ++us)
            for (ut = 0; ut <= 2; ++ut) {
                double p = exp(log_metropolis_factor(k[s], ktau[s], us, ut));
                uint32_t t;
                if (p >= 1.0) {
                    t = 0xFFFFFFFFu;
                } else {
                    double f = floor(ldexp(p, 32));
                    t = (f >= 4294967294.0) ? 0xFFFFFFFEu : (uint32_t)f;
                }
                T[(s * 5 + us) * 3 + ut] = t;
            }
}

/* PT bases for the pair (s, s+1): alpha+- = exp(+-(k_s - k_{s+1})),
 * beta+- = exp(+-(k_tau,s - k_tau,s+1)). */
void orc_pt_bases(int n_slots, const double *k, const double *ktau,
                  double *ap, double *am, double *bp, double *bm)
{
    int s;
    for (s = 0; s + 1 < n_slots; ++s) {
        double dk = k[s] - k[s + 1];
        double dkt = ktau[s] - ktau[s + 1];
        ap[s] = exp(dk);
        am[s] = exp(-dk);
        bp[s] = exp(dkt);
        bm[s] = exp(-dkt);
    }
}

/* b^e by right-to-left binary powering, round-to-nearest multiplies only. */
static double pow_by_squaring(double b, uint64_t e)
{
    double res = 1.0;
    while (e) {
        if (e & 1u) res = res * b;
        b = b * b;
        e >>= 1;
    }
    return res;
}

/* ------------------------------------------------------------------------ */
/* Disorder and start state (the paper keeps separate seeds for J, the      */
/* initial configuration and the Monte Carlo stream; here they are Philox    */
/* domains under one seed).                                                  */
/* ------------------------------------------------------------------------ */

/* J[a][x + L*y][dir], dir 0 = bond to (x+1, y), dir 1 = bond to (x, y+1). */
void orc_init_couplings(int L, int64_t a_lo, int64_t n_a, uint64_t seed, int8_t *J)
{
    int64_t ai;
    int i, dir;
    for (ai = 0; ai < n_a; ++ai)
        for (i = 0; i < L * L; ++i)
            for (dir = 0; dir < 2; ++dir) {
                uint32_t x0 = philox_word((uint32_t)i, (uint32_t)dir, (uint32_t)(a_lo + ai),
                                          (uint32_t)ORC_DOM_J << 28, seed, 0);
                J[(ai * L * L + i) * 2 + dir] = (x0 & 1u) ? 1 : -1;
            }
}

/* S[a][r][w][site]; walker w starts at slot w. */
void orc_init_spins(int L, int Ltau, int n_slots, int n_rep, int64_t a_lo, int64_t n_a,
                    uint64_t seed, int8_t *S)
{
    int64_t N = (int64_t)L * L * Ltau, ai, site;
    int r, w;
    for (ai = 0; ai < n_a; ++ai)
        for (r = 0; r < n_rep; ++r)
            for (w = 0; w < n_slots; ++w)
                for (site = 0; site < N; ++site) {
                    uint32_t x0 = philox_word((uint32_t)site, (uint32_t)w, (uint32_t)(a_lo + ai),
                                              ((uint32_t)ORC_DOM_INIT << 28) | (uint32_t)r, seed, 0);
                    S[((ai * n_rep + r) * n_slots + w) * N + site] = (x0 & 1u) ? 1 : -1;
                }
}

/* ------------------------------------------------------------------------ */
/* Daemon bits (Sec. 2.1.1, Appendices B and C).                             */
/* ------------------------------------------------------------------------ */

/* One state step of xoroshiro128++ (Blackman and Vigna, "Scrambled linear
 * pseudorandom number generators", 2019): with t = s1 xor s0, the new state
 * is (rotl(s0, 49) xor t xor (t << 21), rotl(t, 28)).  The "++" output
 * scrambler is not part of the state step. */
static uint64_t rotl64(uint64_t v, int k) { return (v << k) | (v >> (64 - k)); }

void orc_xoroshiro128pp_step(uint64_t st[2])
{
    uint64_t s0 = st[0];
    uint64_t tt = st[1] ^ s0;
    st[0] = rotl64(s0, 49) ^ tt ^ (tt << 21);
    st[1] = rotl64(tt, 28);
}

/* n* of a 64-bit word R under the cumulative table cum[0..254] of one k
 * (Sec. 2.1.1): the n with cumulative(n-1) <= R < cumulative(n), where
 * cumulative(-1) is below every word and cumulative(255) = 2^64 - 1 (R =
 * 2^64 - 1 gives 255).  Since the table is non-decreasing this is the number
 * of n in 0..254 with cum[n] <= R. */
uint32_t orc_daemon_nstar(const uint64_t *cum, uint64_t R)
{
    uint32_t c = 0;
    int n;
    for (n = 0; n < 255; ++n) c += (cum[n] <= R);
    return c;
}

/* Daemon word `which` (0: b4, 1: b8, 2: b12) of word-site wsite of system
 * (a, r, slot s) in sweep t.  One Philox4x32-10 call gives the upper halves
 * x_0..x_3 of four 64-bit words; the same 128 bits, read as the xoroshiro
 * state (x_0 | x_1 << 32, x_2 | x_3 << 32), take one state step, whose four
 * 32-bit quarters (same order) are the lower halves.  Byte i of the word is
 * n* of 64-bit word i. */
uint32_t orc_daemon_bword(uint64_t seed, int64_t a, int r, int s, uint32_t wsite, uint64_t t,
                          int which, const uint64_t *cum)
{
    uint32_t ctr[4], key[2], x[4], lo[4], b = 0;
    uint64_t st[2];
    int i;
    ctr[0] = wsite;
    ctr[1] = (uint32_t)t;
    ctr[2] = (uint32_t)s | ((uint32_t)r << 16);
    ctr[3] = ((uint32_t)ORC_DOM_DAEMON << 28) | ((uint32_t)which << 24) | (uint32_t)a;
    key[0] = (uint32_t)seed; key[1] = (uint32_t)(seed >> 32);
    orc_philox4x32_10(ctr, key, x);
    st[0] = (uint64_t)x[0] | ((uint64_t)x[1] << 32);
    st[1] = (uint64_t)x[2] | ((uint64_t)x[3] << 32);
    orc_xoroshiro128pp_step(st);
    lo[0] = (uint32_t)st[0]; lo[1] = (uint32_t)(st[0] >> 32);
    lo[2] = (uint32_t)st[1]; lo[3] = (uint32_t)(st[1] >> 32);
    for (i = 0; i < 4; ++i)
        b |= orc_daemon_nstar(cum, ((uint64_t)x[i] << 32) | lo[i]) << (8 * i);
    return b;
}

/* The daemon's level d in 0..3 from one bit of each of b4, b8, b12
 * (Appendix B): after b8 &= b4 and b12 &= b8 the four reachable patterns
 * 000, 100, 110, 111 stand for d = 0, 1, 2, 3, i.e. d is the number of
 * leading ones of (b4, b8, b12). */
int orc_daemon_level(int b4, int b8, int b12)
{
    if (!b4) return 0;
    if (!b8) return 1;
    if (!b12) return 2;
    return 3;
}

/* Metropolis with the daemon at equal couplings (Sec. 2.1, Ito and Kanada):
 * flipping a site with u unsatisfied bonds out of 6 changes the energy of
 * Eq. (3) by 12 - 4u, and the daemon pays for it iff u + d >= 3, which has
 * probability min(1, e^{-4k(3-u)}). */
int orc_daemon_flip(int u, int d) { return u + d >= 3; }

/* ------------------------------------------------------------------------ */
/* The Markov chain.                                                         */
/* ------------------------------------------------------------------------ */

typedef struct {
    int L, Ltau, n_slots, n_rep;
    int tau_ap;                         /* 1: antiperiodic along tau */
    uint64_t seed;
    const uint32_t *T;                  /* [n_slots][5][3] */
    const double *ap, *am, *bp, *bm;    /* [n_slots-1] */
    const uint64_t *cum;                /* daemon rule: [n_slots][255]; NULL: thresholds */
} orc_model;

/* A = sum over spatial bonds of J S S, B = sum over imaginary-time bonds of
 * S S (Eq. (3) splits -E into these two sums); with antiperiodic tau the
 * bond from tau = L_tau-1 to tau = 0 counts -S S. */
static void energies_of(const orc_model *m, const int8_t *J, const int8_t *S,
                        int64_t *A, int64_t *B)
{
    int L = m->L, Lt = m->Ltau, x, y, t;
    int64_t a = 0, b = 0;
    for (t = 0; t < Lt; ++t)
        for (y = 0; y < L; ++y)
            for (x = 0; x < L; ++x) {
                int64_t i = x + (int64_t)L * y + (int64_t)L * L * t;
                int64_t ix = ((x + 1) % L) + (int64_t)L * y + (int64_t)L * L * t;
                int64_t iy = x + (int64_t)L * ((y + 1) % L) + (int64_t)L * L * t;
                int64_t it = x + (int64_t)L * y + (int64_t)L * L * ((t + 1) % Lt);
                int i2 = x + L * y;
                a += J[i2 * 2 + 0] * S[i] * S[ix];
                a += J[i2 * 2 + 1] * S[i] * S[iy];
                b += (m->tau_ap && t == Lt - 1 ? -1 : 1) * S[i] * S[it];
            }
    *A = a;
    *B = b;
}

/* Metropolis update of site (x, y, tau) of the system (a, r, walker at slot
 * s) whose spins are Sw, in sweep t: u_s, u_t = unsatisfied spatial and
 * tau bonds; with the threshold rule the flip is taken iff T == 0xFFFFFFFF
 * or R < T[s][u_s][u_t]; with the daemon rule iff u_s + u_t + d >= 3. */
static void site_update(const orc_model *m, int64_t a, int r, int s, const int8_t *J, int8_t *Sw,
                        int x, int y, int tau, uint64_t t)
{
    int L = m->L, Lt = m->Ltau;
    int xp = (x + 1) % L, xm = (x + L - 1) % L;
    int yp = (y + 1) % L, ym = (y + L - 1) % L;
    int tp = (tau + 1) % Lt, tm = (tau + Lt - 1) % Lt;
    /* sign of the tau bonds: -1 on the antiperiodic wrap bond */
    int gp = (m->tau_ap && tau == Lt - 1) ? -1 : 1;
    int gm = (m->tau_ap && tau == 0) ? -1 : 1;
    int i2 = x + L * y;
    int64_t site = x + (int64_t)L * y + (int64_t)L * L * tau;
    int si = Sw[site];
    int us = 0, ut = 0;
    uint32_t thr, R;
    us += (J[i2 * 2 + 0] * si * Sw[xp + L * y + (int64_t)L * L * tau] == -1);
    us += (J[(xm + L * y) * 2 + 0] * si * Sw[xm + L * y + (int64_t)L * L * tau] == -1);
    us += (J[i2 * 2 + 1] * si * Sw[x + L * yp + (int64_t)L * L * tau] == -1);
    us += (J[(x + L * ym) * 2 + 1] * si * Sw[x + L * ym + (int64_t)L * L * tau] == -1);
    ut += (gp * si * Sw[x + L * y + (int64_t)L * L * tp] == -1);
    ut += (gm * si * Sw[x + L * y + (int64_t)L * L * tm] == -1);
    if (m->cum) {
        /* daemon rule: site (x, y, tau) is bit j = tau / M of word-site
         * x + L y + L^2 (tau mod M), M = L_tau / 32 */
        int M = Lt / 32, j = tau / M, d;
        uint32_t ws = (uint32_t)(x + L * y + (int64_t)L * L * (tau % M));
        const uint64_t *cs = m->cum + (int64_t)s * 255;
        uint32_t b4 = orc_daemon_bword(m->seed, a, r, s, ws, t, 0, cs);
        uint32_t b8 = orc_daemon_bword(m->seed, a, r, s, ws, t, 1, cs);
        uint32_t b12 = orc_daemon_bword(m->seed, a, r, s, ws, t, 2, cs);
        d = orc_daemon_level((b4 >> j) & 1, (b8 >> j) & 1, (b12 >> j) & 1);
        if (orc_daemon_flip(us + ut, d)) Sw[site] = (int8_t)(-si);
        return;
    }
    thr = m->T[(s * 5 + us) * 3 + ut];
    R = philox_word((uint32_t)site, (uint32_t)t,
                    (uint32_t)s | ((uint32_t)(r >> 2) << 16),
                    ((uint32_t)ORC_DOM_SWEEP << 28) | (uint32_t)(a >> 6),
                    m->seed, r & 3);
    if (thr == 0xFFFFFFFFu || R < thr) Sw[site] = (int8_t)(-si);
}

/* One half sweep of one sample a: every site of the given colour, every
 * replica r and slot s, for the walker w currently at slot s. */
static void half_sweep(const orc_model *m, int64_t a, const int8_t *J, int8_t *S_a,
                       const int32_t *walker_at_a, uint64_t t, int colour)
{
    int L = m->L, Lt = m->Ltau, n_slots = m->n_slots, n_rep = m->n_rep;
    int64_t N = (int64_t)L * L * Lt;
    int x, y, tau, r, s;
    for (tau = 0; tau < Lt; ++tau)
        for (y = 0; y < L; ++y)
            for (x = 0; x < L; ++x) {
                if (((x + y + tau) & 1) != colour) continue;
                for (r = 0; r < n_rep; ++r)
                    for (s = 0; s < n_slots; ++s) {
                        int w = walker_at_a[r * n_slots + s];
                        site_update(m, a, r, s, J, S_a + ((int64_t)r * n_slots + w) * N, x, y, tau, t);
                    }
            }
}

/* One sweep (red, then blue) of ONE system of the daemon rule: sample a,
 * replica r, slot s, spins S [N] in place, couplings J [L*L][2] of sample
 * a, cumulative tables cum [n_slots][255].  The daemon rule's update of a
 * system depends on no other system, so this is the same sweep the full
 * chain applies to it (for the tests at sizes where a full run is too slow). */
void orc_daemon_sweep_system(int L, int Ltau, uint64_t seed, int64_t a, int r, int s, uint64_t t,
                             int tau_ap, const int8_t *J, int8_t *S, const uint64_t *cum)
{
    orc_model m;
    int x, y, tau, colour;
    memset(&m, 0, sizeof(m));
    m.L = L; m.Ltau = Ltau; m.seed = seed; m.tau_ap = tau_ap; m.cum = cum;
    for (colour = 0; colour < 2; ++colour)
        for (tau = 0; tau < Ltau; ++tau)
            for (y = 0; y < L; ++y)
                for (x = 0; x < L; ++x)
                    if (((x + y + tau) & 1) == colour) site_update(&m, a, r, s, J, S, x, y, tau, t);
}

/* One PT pass of chain (a, r) after sweep t: pairs (s, s+1) in increasing s.
 * Walker X sits at s, Y at s+1; the exchange is accepted with probability
 * min(1, exp((k_s - k_{s+1})(A_Y - A_X) + (kt_s - kt_{s+1})(B_Y - B_X))),
 * evaluated as a product of powers of the precomputed bases. */
static void pt_pass(const orc_model *m, int64_t a, int r, uint64_t t,
                    int32_t *walker_at_ar, const int64_t *A_ar, const int64_t *B_ar)
{
    int s;
    for (s = 0; s + 1 < m->n_slots; ++s) {
        int X = walker_at_ar[s], Y = walker_at_ar[s + 1];
        int64_t dm = A_ar[Y] - A_ar[X];
        int64_t dn = B_ar[Y] - B_ar[X];
        double fa = pow_by_squaring(dm >= 0 ? m->ap[s] : m->am[s],
                                    (uint64_t)(dm >= 0 ? dm : -dm));
        double fb = pow_by_squaring(dn >= 0 ? m->bp[s] : m->bm[s],
                                    (uint64_t)(dn >= 0 ? dn : -dn));
        double P = fa * fb;
        uint32_t x = philox_word((uint32_t)s, (uint32_t)t, (uint32_t)a,
                                 ((uint32_t)ORC_DOM_PT << 28) | (uint32_t)(r >> 2), m->seed, r & 3);
        double u = ldexp((double)x, -32);
        if (u < P) {
            walker_at_ar[s] = Y;
            walker_at_ar[s + 1] = X;
        }
    }
}

/*
 * Run n_sweeps sweeps (sweep indices t0 .. t0+n_sweeps-1) for samples
 * a_lo .. a_lo+n_a-1.  Per sweep t: red half sweep, blue half sweep, then a
 * PT pass of every chain when pt_every > 0 and (t+1) % pt_every == 0, then
 * a measurement when measure_every > 0 and (t+1) % measure_every == 0.
 *
 * Arrays (per sample offset ai = a - a_lo):
 *   J         [n_a][L*L][2]                       int8 +-1
 *   S         [n_a][n_rep][n_slots walkers][N]    int8 +-1, in/out
 *   walker_at [n_a][n_rep][n_slots]               in/out
 *   A, B      [n_a][n_rep][n_slots] by slot       out: energies after the run
 *   sumA,sumB [n_a][n_rep][n_slots] by slot       in/out: measurement sums
 *   sumq,sumq2[n_a][n_slots][n_rep(n_rep-1)/2]    in/out: overlap sums
 *   n_meas                                        in/out: measurements taken
 * Observables may be NULL when measure_every == 0.  tau_ap: antiperiodic
 * boundary along tau (0: periodic).  daemon_cum: NULL for the threshold
 * rule; else the daemon rule with the cumulative tables [n_slots][255] of
 * Sec. 2.1.1 (needs k_tau = k for every slot and L_tau a multiple of 64).
 *
 * Records of Appendix A, indexed by the measurement number m (counted from
 * *n_meas on entry, which is the number of measurements already taken):
 *   hist      [m][n_a][n_rep][n_slots]  (NULL: not kept) history_betas: the
 *             slot, i.e. the ladder value k, of every walker (system copy)
 *   blkA/B    [m / maxit][n_a][n_rep][n_slots] by slot (NULL or maxit 0: not
 *             kept): sums of A and B over the maxit consecutive
 *             measurements of each block, whose averages are written out
 */
int orc_run(int L, int Ltau, int n_slots, int n_rep, int64_t a_lo, int64_t n_a, uint64_t seed,
            const double *k, const double *ktau, int pt_every, int measure_every,
            const int8_t *J, int8_t *S, int32_t *walker_at, uint64_t t0, int64_t n_sweeps,
            int64_t *A, int64_t *B, int64_t *sumA, int64_t *sumB, int64_t *sumq, int64_t *sumq2,
            int64_t *n_meas, int n_threads, int tau_ap, const uint64_t *daemon_cum,
            uint8_t *hist, int maxit, int64_t *blkA, int64_t *blkB)
{
    orc_model m;
    uint32_t *T;
    double *ap, *am, *bp, *bm;
    int64_t N = (int64_t)L * L * Ltau;
    int n_pairs = n_rep * (n_rep - 1) / 2;
    int64_t ai;
    int64_t meas_total = 0;
    const int64_t meas0 = n_meas ? *n_meas : 0;

    T = (uint32_t *)malloc(sizeof(uint32_t) * 15 * (size_t)n_slots);
    ap = (double *)malloc(sizeof(double) * 4 * (size_t)(n_slots > 1 ? n_slots : 2));
    if (!T || !ap) { free(T); free(ap); return -1; }
    am = ap + n_slots; bp = am + n_slots; bm = bp + n_slots;
    orc_thresholds(n_slots, k, ktau, T);
    orc_pt_bases(n_slots, k, ktau, ap, am, bp, bm);
    m.L = L; m.Ltau = Ltau; m.n_slots = n_slots; m.n_rep = n_rep; m.seed = seed;
    m.tau_ap = tau_ap;
    m.T = T; m.ap = ap; m.am = am; m.bp = bp; m.bm = bm;
    m.cum = daemon_cum;
    if (daemon_cum) {
        int s;
        if (Ltau % 64 != 0 || a_lo + n_a > ((int64_t)1 << 24) || n_rep > 4096) {
            free(T); free(ap); return -2;
        }
        for (s = 0; s < n_slots; ++s)
            if (k[s] != ktau[s]) { free(T); free(ap); return -2; }
    }

#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : meas_total)
#endif
    for (ai = 0; ai < n_a; ++ai) {
        int64_t a = a_lo + ai;
        const int8_t *Ja = J + ai * L * L * 2;
        int8_t *Sa = S + ai * n_rep * n_slots * N;
        int32_t *wa = walker_at + ai * n_rep * n_slots;
        int64_t *Aw = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)n_rep * n_slots);
        int64_t *Bw = Aw + n_rep * n_slots;   /* by walker */
        int64_t it;
        int r, s, w;
        int64_t local_meas = 0;
        for (it = 0; it < n_sweeps; ++it) {
            uint64_t t = t0 + (uint64_t)it;
            half_sweep(&m, a, Ja, Sa, wa, t, 0);
            half_sweep(&m, a, Ja, Sa, wa, t, 1);
            for (r = 0; r < n_rep; ++r)
                for (w = 0; w < n_slots; ++w)
                    energies_of(&m, Ja, Sa + ((int64_t)r * n_slots + w) * N,
                                &Aw[r * n_slots + w], &Bw[r * n_slots + w]);
            if (pt_every > 0 && (t + 1) % (uint64_t)pt_every == 0)
                for (r = 0; r < n_rep; ++r)
                    pt_pass(&m, a, r, t, wa + r * n_slots, Aw + r * n_slots, Bw + r * n_slots);
            if (measure_every > 0 && (t + 1) % (uint64_t)measure_every == 0) {
                int r1, r2, p;
                for (r = 0; r < n_rep; ++r)
                    for (s = 0; s < n_slots; ++s) {
                        w = wa[r * n_slots + s];
                        sumA[(ai * n_rep + r) * n_slots + s] += Aw[r * n_slots + w];
                        sumB[(ai * n_rep + r) * n_slots + s] += Bw[r * n_slots + w];
                    }
                /* overlap q = sum_i S^{r1}_i S^{r2}_i of the configurations at
                 * slot s of replicas r1 < r2 (Appendix E.1, same sample) */
                for (s = 0; s < n_slots; ++s) {
                    p = 0;
                    for (r1 = 0; r1 < n_rep; ++r1)
                        for (r2 = r1 + 1; r2 < n_rep; ++r2, ++p) {
                            const int8_t *S1 = Sa + ((int64_t)r1 * n_slots + wa[r1 * n_slots + s]) * N;
                            const int8_t *S2 = Sa + ((int64_t)r2 * n_slots + wa[r2 * n_slots + s]) * N;
                            int64_t q = 0, i;
                            for (i = 0; i < N; ++i) q += S1[i] * S2[i];
                            sumq[(ai * n_slots + s) * n_pairs + p] += q;
                            sumq2[(ai * n_slots + s) * n_pairs + p] += q * q;
                        }
                }
                {
                    const int64_t mi = meas0 + local_meas;
                    if (hist)   /* the PT walk: where every walker is now */
                        for (r = 0; r < n_rep; ++r)
                            for (s = 0; s < n_slots; ++s)
                                hist[((mi * n_a + ai) * n_rep + r) * n_slots + wa[r * n_slots + s]] = (uint8_t)s;
                    if (blkA && blkB && maxit > 0) {   /* block sums of maxit measurements */
                        const int64_t bi = mi / maxit;
                        const int first = mi % maxit == 0;
                        for (r = 0; r < n_rep; ++r)
                            for (s = 0; s < n_slots; ++s) {
                                const int64_t idx = ((bi * n_a + ai) * n_rep + r) * n_slots + s;
                                w = wa[r * n_slots + s];
                                blkA[idx] = (first ? 0 : blkA[idx]) + Aw[r * n_slots + w];
                                blkB[idx] = (first ? 0 : blkB[idx]) + Bw[r * n_slots + w];
                            }
                    }
                }
                ++local_meas;
            }
        }
        /* energies of the final state, reported by slot */
        for (r = 0; r < n_rep; ++r)
            for (w = 0; w < n_slots; ++w)
                energies_of(&m, Ja, Sa + ((int64_t)r * n_slots + w) * N,
                            &Aw[r * n_slots + w], &Bw[r * n_slots + w]);
        for (r = 0; r < n_rep; ++r)
            for (s = 0; s < n_slots; ++s) {
                w = wa[r * n_slots + s];
                A[(ai * n_rep + r) * n_slots + s] = Aw[r * n_slots + w];
                B[(ai * n_rep + r) * n_slots + s] = Bw[r * n_slots + w];
            }
        if (ai == 0) meas_total += local_meas;
        free(Aw);
    }
    if (n_meas) *n_meas += meas_total;
    free(T);
    free(ap);
    return 0;
}

/* Energies A, B (by walker) of given configurations: [n_a][n_rep][n_slots]. */
void orc_energies(int L, int Ltau, int n_slots, int n_rep, int64_t n_a, const int8_t *J,
                  const int8_t *S, int64_t *A, int64_t *B, int tau_ap)
{
    orc_model m;
    int64_t N = (int64_t)L * L * Ltau, c;
    m.L = L; m.Ltau = Ltau; m.n_slots = n_slots; m.n_rep = n_rep; m.tau_ap = tau_ap;
    m.cum = NULL;
    for (c = 0; c < n_a * n_rep * n_slots; ++c)
        energies_of(&m, J + (c / (n_rep * n_slots)) * L * L * 2, S + c * N, &A[c], &B[c]);
}

/* One PT pass with given energies by walker (for the PT-only tests). */
void orc_pt_only(int n_slots, int n_rep, int64_t a, uint64_t seed, const double *k,
                 const double *ktau, uint64_t t, int32_t *walker_at_a,
                 const int64_t *A_a, const int64_t *B_a)
{
    orc_model m;
    double *ap = (double *)malloc(sizeof(double) * 4 * (size_t)(n_slots > 1 ? n_slots : 2));
    int r;
    m.n_slots = n_slots; m.n_rep = n_rep; m.seed = seed;
    m.cum = NULL;
    m.ap = ap; m.am = ap + n_slots; m.bp = ap + 2 * n_slots; m.bm = ap + 3 * n_slots;
    orc_pt_bases(n_slots, k, ktau, ap, ap + n_slots, ap + 2 * n_slots, ap + 3 * n_slots);
    for (r = 0; r < n_rep; ++r)
        pt_pass(&m, a, r, t, walker_at_a + r * n_slots, A_a + r * n_slots, B_a + r * n_slots);
    free(ap);
}

double orc_pow_by_squaring(double b, uint64_t e) { return pow_by_squaring(b, e); }

/*
 * Imaginary-time observables of Appendix E.1 for the configuration now at
 * each slot: with q~_x(tau_1, tau) = S_{x,tau_1} S_{x,tau_1+tau} (tau_1 + tau
 * modulo L_tau) and Q~ = sum_x q~, over tau_1 = 0 .. L_tau-1:
 *   S1 = sum Q~, S2 = sum Q~^2, S4 = sum Q~^4 (int64),
 *   SF = sum ( |sum_x e^{i 2pi x_1/L} q~_x|^2 + |sum_x e^{i 2pi x_2/L} q~_x|^2 )
 * (FP64).  The two Fourier sums are taken over the column sums
 * C(x_1) = sum_{x_2} q~ and the row sums R(x_2) = sum_{x_1} q~, x = 0 .. L-1
 * in order, real and imaginary parts accumulated separately, no contraction.
 * S [n_a][n_rep][n_slots walkers][N] int8, walker_at [n_a][n_rep][n_slots];
 * outputs [n_a][n_rep][n_slots][L_tau].
 */
void orc_tau_observables(int L, int Ltau, int n_slots, int n_rep, int64_t n_a, const int8_t *S,
                         const int32_t *walker_at, int64_t *S1, int64_t *S2, int64_t *S4, double *SF)
{
    const double pi = 3.14159265358979323846;
    const int64_t N = (int64_t)L * L * Ltau, P = (int64_t)L * L;
    double *cs = (double *)malloc(sizeof(double) * 2 * (size_t)L);
    double *sn = cs + L;
    int64_t c;
    int x;
    for (x = 0; x < L; ++x) {
        cs[x] = cos(2.0 * pi * x / L);
        sn[x] = sin(2.0 * pi * x / L);
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (c = 0; c < n_a * n_rep * n_slots; ++c) {
        const int64_t ar = c / n_slots;
        const int w = walker_at[c];
        const int8_t *Sw = S + (ar * n_slots + w) * N;
        int tau;
        for (tau = 0; tau < Ltau; ++tau) {
            int64_t s1 = 0, s2 = 0, s4 = 0;
            double sf = 0.0;
            int t1;
            for (t1 = 0; t1 < Ltau; ++t1) {
                const int t2 = (t1 + tau) % Ltau;
                int64_t q = 0;
                double re1 = 0.0, im1 = 0.0, re2 = 0.0, im2 = 0.0;
                int xx;
                for (xx = 0; xx < L; ++xx) {
                    int64_t R = 0, C = 0;
                    int j;
                    for (j = 0; j < L; ++j) {
                        R += Sw[j + (int64_t)L * xx + P * t1] * Sw[j + (int64_t)L * xx + P * t2];   /* x_2 = xx */
                        C += Sw[xx + (int64_t)L * j + P * t1] * Sw[xx + (int64_t)L * j + P * t2];   /* x_1 = xx */
                    }
                    q += R;
                    re1 = re1 + cs[xx] * (double)C;
                    im1 = im1 + sn[xx] * (double)C;
                    re2 = re2 + cs[xx] * (double)R;
                    im2 = im2 + sn[xx] * (double)R;
                }
                s1 += q;
                s2 += q * q;
                s4 += (q * q) * (q * q);
                sf = sf + ((re1 * re1 + im1 * im1) + (re2 * re2 + im2 * im2));
            }
            S1[c * Ltau + tau] = s1;
            S2[c * Ltau + tau] = s2;
            S4[c * Ltau + tau] = s4;
            SF[c * Ltau + tau] = sf;
        }
    }
    free(cs);
}

/*
 * The transfer-matrix product of the exact-diagonalisation code (Sec. 2.2,
 * Eq. (transfer-matrix); Appendix D): out = T in on the even (parity = +1)
 * or odd (parity = -1) sector, in the parity-aware basis |n>_{e,o},
 * n = 0 .. 2^{L^2-1}-1.  With separate couplings (k, k_tau):
 *   T = e^{-k H0 / 2} prod_j [jP 1_j + jM sigma^X_j] e^{-k H0 / 2},
 *   jP = e^{k_tau} / (e^{k_tau} + e^{-k_tau}), jM = e^{-k_tau} / (...),
 * which is Eq. (expH1) when exp(-2 k_tau) = tanh(k Gamma) (k_tau = k for the
 * paper's equal coupling).  Steps, in the paper's order:
 *   psi[n] = in[n] w[n],  w[n] = exp((k/2) sum_bonds J S_x S_y), n read as an
 *            L^2-bit integer with the top bit 0 (bit j set <=> S_j = -1);
 *   rounds j = 0 .. L^2-2: psi'[n] = jP psi[n] + jM psi[n ^ 2^j];
 *   the last factor (j = L^2-1, Eq. (lr)): psi'[n] = jP psi[n] +
 *            parity jM psi[(2^{L^2-1}-1) - n];
 *   out[n] = psi[n] w[n].
 * Bonds: J [L*L][2] (+-1), bond 0 of site j = x1 + L x2 joins it to
 * (x1+1, x2), bond 1 to (x1, x2+1), periodic.  Vectors of 2^{L^2-1} doubles.
 */
int orc_transfer_matvec(int L, double k, double ktau, const int8_t *J, int parity, const double *in, double *out)
{
    const int nb = L * L - 1;
    const uint64_t n_el = (uint64_t)1 << nb;
    const double ek = exp(ktau), emk = exp(-ktau);
    const double jP = ek / (ek + emk), jM = emk / (ek + emk);
    double *w = (double *)malloc(sizeof(double) * n_el);
    double *psi = (double *)malloc(sizeof(double) * n_el);
    double *scra = (double *)malloc(sizeof(double) * n_el);
    uint64_t n;
    int j;
    if (!w || !psi || !scra) { free(w); free(psi); free(scra); return -1; }
    for (n = 0; n < n_el; ++n) {
        int64_t e = 0;
        int x1, x2;
        for (x2 = 0; x2 < L; ++x2)
            for (x1 = 0; x1 < L; ++x1) {
                const int i = x1 + L * x2;
                const int ix = (x1 + 1) % L + L * x2, iy = x1 + L * ((x2 + 1) % L);
                const int si = (n >> i) & 1u ? -1 : 1;
                const int sx = (n >> ix) & 1u ? -1 : 1;
                const int sy = (n >> iy) & 1u ? -1 : 1;
                e += J[2 * i] * si * sx + J[2 * i + 1] * si * sy;
            }
        w[n] = exp(0.5 * k * (double)e);
    }
    for (n = 0; n < n_el; ++n) psi[n] = in[n] * w[n];
    for (j = 0; j < nb; ++j) {
        for (n = 0; n < n_el; ++n) scra[n] = jP * psi[n] + jM * psi[n ^ ((uint64_t)1 << j)];
        { double *tmp = psi; psi = scra; scra = tmp; }
    }
    for (n = 0; n < n_el; ++n) scra[n] = jP * psi[n] + (double)parity * jM * psi[(n_el - 1) - n];
    for (n = 0; n < n_el; ++n) out[n] = scra[n] * w[n];
    free(w); free(psi); free(scra);
    return 0;
}
