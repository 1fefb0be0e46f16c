/*
 * pa_oracle.c -- TEST INFRASTRUCTURE, not part of the product.
 *
 * A plain, single-threaded, deliberately slow CPU restatement of population
 * annealing (PA) for the two-dimensional q-state Potts model, following
 * Barash, Weigel, Shchur & Janke, "Exploring first-order phase transitions
 * with population annealing" (arXiv:1704.01888).  Only the test suite,
 * __graft_entry__.smoke() and the CPU-baseline / reference legs of bench.py
 * may load this file's library.  The CUDA library never links or calls it and
 * the two share no source.
 *
 * Every function follows the paper's definitions in their plain order:
 *   - the Hamiltonian H = -J sum_<ij> delta(s_i, s_j), J = 1, periodic
 *     square lattice (Sec. 3, Eq. 3);
 *   - the magnetisation through the occupation of the most common state
 *     (Sec. 3, Eq. 5);
 *   - the PA loop: resample with tau_i(E_j) = exp(-(beta_i-beta_{i-1})E_j)/Q_i,
 *     Q_i = sum_j exp(-(beta_i-beta_{i-1})E_j)/R_{i-1}, then theta Metropolis
 *     rounds at beta_i, then population averages (Sec. 2, steps 1-5);
 *   - the free-energy estimator -beta_i F = ln Z_{beta_0} + sum_m ln Q_m
 *     (Sec. 2, Eq. 2), with Z_{beta_0=0} = q^N (Sec. 6) and the zero-temperature
 *     normalisation Z = q exp(-beta E_0), E_0 = -2N (Sec. 6, Eqs. 7-8);
 *   - ground-state initialisation for heating runs (Sec. 5, Eq. 6).
 * Choices the paper leaves open (random-number keying, the Metropolis proposal,
 * the copy-count rounding rule, the family-entropy definition) are fixed here
 * exactly as the CUDA library fixes them; each is marked "reading:".
 *
 * Floating point is IEEE double with contraction disabled (-ffp-contract=off);
 * spins, energies, counts and histograms are integers.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, from Salmon, Moraes, Dror & Shaw, "Parallel random numbers:  */
/* as easy as 1, 2, 3" (SC'11): 10 rounds of two 32x32->64 multiplies, the    */
/* high halves xored with the other counter words and the round key, the key  */
/* bumped by the Weyl constants between rounds.                               */
/* ------------------------------------------------------------------------- */
ORC_API void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* reading: the counter word c1 carries a 2-bit domain tag in its top bits so
 * that initialisation, sweeps, resampling and ground-state draws never share
 * a counter.  The top byte of c3 carries a stream number (0..255) that lets
 * several independent runs share one key; slots stay below 2^24. */
#define ORC_DOM_SWEEP    0x00000000u
#define ORC_DOM_INIT     0x40000000u
#define ORC_DOM_RESAMPLE 0x80000000u
#define ORC_DOM_GROUND   0xC0000000u

static void orc_draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t out[4])
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* floor(u * n / 2^32): an integer in [0, n) from one 32-bit word. */
static uint32_t orc_scale(uint32_t u, uint32_t n)
{
    return (uint32_t)(((uint64_t)u * (uint64_t)n) >> 32);
}

/* ------------------------------------------------------------------------- */
/* Model: Sec. 3, Eq. 3 and Eq. 5.  Lattices are stored row-major, s[y*L+x], */
/* states 0..q-1 (the paper's 1..q shifted by one).                           */
/* ------------------------------------------------------------------------- */

/* E = -sum over the 2N bonds of delta(s_i, s_j); each bond is visited once as
 * the (right, down) bond of its left/upper site.  reading: for L = 2 the right
 * and left neighbours coincide, so that pair is one site's right bond and the
 * other's, counted twice, which keeps E_0 = -2N (Sec. 6). */
ORC_API int64_t orc_energy(int L, const uint8_t *s)
{
    int64_t e = 0;
    for (int y = 0; y < L; ++y) {
        for (int x = 0; x < L; ++x) {
            int here = s[y * L + x];
            int right = s[y * L + (x + 1) % L];
            int down = s[((y + 1) % L) * L + x];
            if (here == right) e -= 1;
            if (here == down) e -= 1;
        }
    }
    return e;
}

/* M~ = max over states alpha of the number of sites in state alpha (Eq. 5). */
ORC_API int64_t orc_max_count(int q, int L, const uint8_t *s)
{
    int64_t counts[256];
    for (int a = 0; a < q; ++a) counts[a] = 0;
    for (int i = 0; i < L * L; ++i) counts[s[i]] += 1;
    int64_t best = 0;
    for (int a = 0; a < q; ++a)
        if (counts[a] > best) best = counts[a];
    return best;
}

/* ------------------------------------------------------------------------- */
/* Metropolis single-spin-flip update (Sec. 2 step 3, Sec. 3).                */
/*                                                                             */
/* reading (proposal): B = ceil(log2 q) bits hold a state.  An attempt draws  */
/* a direction bit sigma and a (B-1)-bit number u; with d = 1 + u (so         */
/* 1 <= d <= 2^(B-1) <= q - 1) the proposed state is s' = (s + d) mod q for   */
/* sigma = 0 and (s - d) mod q for sigma = 1.  s' never equals s, every other */
/* state is reachable, and the move s -> s' has the same probability as the   */
/* move s' -> s (+d under one direction is -d under the other), so the        */
/* Metropolis rule below satisfies detailed balance exactly.  For q - 1 a     */
/* power of two the proposal is uniform over the q - 1 other states.          */
/*                                                                             */
/* reading (acceptance): with dE = E(s') - E(s), an integer in [-4, 4], the   */
/* move is accepted if dE <= 0 and otherwise iff v < T[dE], v a uniform       */
/* 32-bit number and T[d] = floor(exp(-beta d) 2^32).                          */
/* ------------------------------------------------------------------------- */

/* Bits per state: the smallest B with 2^B >= q. */
ORC_API int orc_state_bits(int q)
{
    int B = 0;
    while ((1 << B) < q) ++B;
    return B;
}

/* T[d] = floor(exp(-beta d) 2^32) for d = 1..4 (T[0] = 2^32, unused). */
ORC_API void orc_thresholds(double beta, uint64_t T[5])
{
    T[0] = 4294967296ull;
    for (int d = 1; d <= 4; ++d) T[d] = (uint64_t)(exp(-beta * (double)d) * 4294967296.0);
}

/* The proposal: s' = (s + d) mod q for sigma = 0, (s - d) mod q for sigma = 1,
 * d = 1 + u. */
ORC_API int orc_propose(int q, int cur, int sigma, uint32_t u)
{
    int d = 1 + (int)u;
    return sigma ? ((cur - d) % q + q) % q : (cur + d) % q;
}

/* E = -(number of satisfied bonds): moving a site from `cur` to `prop` with
 * neighbours nb[0..3] changes E by n(cur) - n(prop), n(a) the number of
 * neighbours in state a. */
ORC_API int orc_delta_energy(int cur, int prop, const int nb[4])
{
    int n_cur = 0, n_prop = 0;
    for (int k = 0; k < 4; ++k) {
        if (nb[k] == cur) n_cur += 1;
        if (nb[k] == prop) n_prop += 1;
    }
    return n_cur - n_prop;
}

/* v < T for a 32-bit v whose bits are supplied most significant first by
 * bit(ctx, j), j = 0..31 (bit j has weight 2^(31-j)): the first bit in which v
 * and T differ decides, and v = T is not below.  Reading bits only until that
 * point is how an unsigned comparison works; it lets the sweep draw no more
 * random words than the decision needs. */
typedef int (*orc_bit_fn)(void *ctx, int j);

static int orc_below(orc_bit_fn bit, void *ctx, uint64_t T)
{
    if (T >= 4294967296ull) return 1;
    for (int j = 0; j < 32; ++j) {
        int vb = bit(ctx, j);
        int tb = (int)(T >> (31 - j)) & 1;
        if (vb != tb) return vb < tb;
    }
    return 0;
}

static int orc_value_bit(void *ctx, int j) { return (int)(*(const uint32_t *)ctx >> (31 - j)) & 1; }

/* orc_below on a given value (exported so that the tests can compare it with
 * the integer comparison). */
ORC_API int orc_below_value(uint32_t v, uint64_t T)
{
    return orc_below(orc_value_bit, &v, T);
}

/* The Metropolis acceptance: always for dE <= 0, else iff v < T[dE]. */
ORC_API int orc_accept(int dE, uint32_t v, const uint64_t T[5])
{
    if (dE <= 0) return 1;
    return (uint64_t)v < T[dE];
}

/* One attempt on a site in state `cur` whose four neighbours are nb[0..3],
 * with direction bit sigma, offset bits u and acceptance number v.  Returns
 * the state after the attempt. */
ORC_API int orc_metropolis_decide(int q, int cur, const int nb[4], int sigma, uint32_t u, uint32_t v,
                                  const uint64_t T[5])
{
    int prop = orc_propose(q, cur, sigma, u);
    return orc_accept(orc_delta_energy(cur, prop, nb), v, T) ? prop : cur;
}

static void orc_neighbours(int L, const uint8_t *s, int x, int y, int nb[4])
{
    nb[0] = s[y * L + (x + L - 1) % L];
    nb[1] = s[y * L + (x + 1) % L];
    nb[2] = s[((y + L - 1) % L) * L + x];
    nb[3] = s[((y + 1) % L) * L + x];
}

/* reading (random numbers of a sweep): the sites of one colour c ((x + y)
 * mod 2), with column index m = x >> 1, are grouped 32 to a "site word".  When
 * a whole number of that colour's rows fills 32 columns (L = 8, 16, 32, 64,
 * i.e. L/2 divides 32), the colour's sites in row-major order, h = y L/2 + m,
 * fill the words in turn: word w = h >> 5, bit b = h & 31.  When L is a
 * multiple of 16 but not of 64 and larger than 32 (L = 48, 80, 96, 112, ...),
 * the rows fall into four bands of L/4 rows and each row into L/16 segments
 * of 8 columns; word w = k (L/16) + j holds segment j of rows k, k + L/4,
 * k + L/2 and k + 3L/4, the site of band a (row y = k + a L/4) and column
 * m = 8j + t at bit b = 8a + t.  Otherwise each row starts a new word: word
 * t = m >> 5 of the row, bit b = m & 31, word index w = y ceil(L / 64) + t.
 * (At L = 64 the first and last rules coincide.)  In sweep k,
 * colour c, temperature step `step`, the word draws a stream Z_0, Z_1, ... of
 * 32-bit numbers, Z_{4n+i} being word i of the Philox call with counter
 * (w, SWEEP | ((2k + c) << 8) | n, step, slot | stream << 24), and the site at
 * bit b takes bit b of each:
 *   sigma = bit of Z_0,  u = sum_{i=1}^{B-1} bit(Z_i) 2^(i-1),
 *   v = sum_{j=0}^{31} bit(Z_{B+j}) 2^(31-j),
 * i.e. the acceptance bits follow the proposal bits with no gap.
 * The stream of one word is drawn once per half sweep (lazily, on first use). */
static int orc_rows_packed(int L)
{
    return L >= 8 && 64 % L == 0;
}

static int orc_rows_banded(int L)
{
    return L > 32 && L % 16 == 0 && L % 64 != 0;
}

/* Site words of one colour per replica. */
ORC_API int orc_colour_words(int L)
{
    return (orc_rows_packed(L) || orc_rows_banded(L)) ? L * L / 64 : L * ((L + 63) / 64);
}

/* The site that bit b of site word w of colour c holds, by the rule above:
 * returns 1 and sets (x, y), or 0 where that bit holds no site (the columns
 * past L/2 of a row's last word when rows are padded). */
ORC_API int orc_word_site(int L, int colour, int w, int b, int *x, int *y)
{
    int m, row;
    if (orc_rows_packed(L)) {
        int h = 32 * w + b;
        row = h / (L / 2);
        m = h % (L / 2);
    } else if (orc_rows_banded(L)) {
        int segs = L / 16, band_rows = L / 4;
        row = w / segs + (b >> 3) * band_rows;
        m = 8 * (w % segs) + (b & 7);
    } else {
        int words_per_row = (L + 63) / 64;
        row = w / words_per_row;
        m = 32 * (w % words_per_row) + b;
    }
    int col = 2 * m + ((colour + row) & 1);
    if (col >= L) return 0; /* (odd L, accepted by the oracle alone, ends rows early too) */
    *y = row;
    *x = col;
    return 1;
}

struct orc_word_stream {
    uint64_t seed;
    uint32_t w, c1base, step, c3;
    int have;             /* number of Philox calls drawn so far */
    uint32_t Z[48];
};

static uint32_t orc_stream_word(struct orc_word_stream *st, int i)
{
    while (st->have <= i / 4) {
        orc_draw(st->seed, st->w, st->c1base | (uint32_t)st->have, st->step, st->c3, st->Z + 4 * st->have);
        st->have += 1;
    }
    return st->Z[i];
}

/* Bit j (weight 2^(31-j)) of the acceptance number v of the site at bit b. */
struct orc_v_source {
    struct orc_word_stream *st;
    int first, b;  /* v's bit j is bit b of Z_{first + j} */
};

static int orc_v_bit(void *ctx, int j)
{
    struct orc_v_source *src = (struct orc_v_source *)ctx;
    return (int)(orc_stream_word(src->st, src->first + j) >> src->b) & 1;
}

/* One attempt on site (x, y), which takes bit b of the word stream st. */
static void orc_attempt(int q, int B, int L, uint8_t *s, int x, int y, struct orc_word_stream *st, int b,
                        const uint64_t T[5])
{
    int sigma = (int)(orc_stream_word(st, 0) >> b) & 1;
    uint32_t u = 0;
    for (int i = 1; i < B; ++i) u |= ((orc_stream_word(st, i) >> b) & 1u) << (i - 1);
    int nb[4];
    orc_neighbours(L, s, x, y, nb);
    int cur = s[y * L + x];
    int prop = orc_propose(q, cur, sigma, u);
    int dE = orc_delta_energy(cur, prop, nb);
    /* the Metropolis acceptance of orc_accept, with v read bit by bit and only
     * when the move raises the energy */
    int accept = 1;
    if (dE > 0) {
        struct orc_v_source src = {st, B, b};
        accept = orc_below(orc_v_bit, &src, T[dE]);
    }
    if (accept) s[y * L + x] = (uint8_t)prop;
}

/* theta checkerboard sweeps of one replica at the thresholds T; returns the
 * number of Philox calls drawn (a word draws its stream lazily, so this is
 * the number its deepest site needed).
 * reading: one sweep updates the colour-0 sites ((x+y) even) and then the
 * colour-1 sites, each colour row by row and, within a row, by increasing x.
 * With L even no two sites of one colour are neighbours, so this in-place
 * order equals a simultaneous update of each colour.  (For odd L the order is
 * still a product of single-site Metropolis steps, each of which keeps the
 * Boltzmann distribution stationary.) */
ORC_API int64_t orc_sweep_replica(int q, int L, uint8_t *s, const uint64_t T[5], int theta,
                                  uint32_t step, uint32_t slot, uint64_t seed, uint32_t stream)
{
    int B = orc_state_bits(q);
    int words = orc_colour_words(L);
    int64_t calls = 0; /* Philox calls the site words drew (each as many as its sites needed) */
    for (int k = 0; k < theta; ++k) {
        for (int colour = 0; colour < 2; ++colour) {
            struct orc_word_stream st;
            st.seed = seed;
            st.c1base = ORC_DOM_SWEEP | ((uint32_t)(2 * k + colour) << 8);
            st.step = step;
            st.c3 = slot | (stream << 24);
            for (int w = 0; w < words; ++w) {
                st.w = (uint32_t)w;
                st.have = 0;
                for (int b = 0; b < 32; ++b) {
                    int x, y;
                    if (orc_word_site(L, colour, w, b, &x, &y)) orc_attempt(q, B, L, s, x, y, &st, b, T);
                }
                calls += st.have;
            }
        }
    }
    return calls;
}

/* ------------------------------------------------------------------------- */
/* Initial populations.                                                        */
/* ------------------------------------------------------------------------- */

/* beta_0 = 0: every site independently uniform over the q states (Sec. 2,
 * step 1).  Site i = y L + x of slot r takes word (i & 3) of the call with
 * counter (i >> 2, INIT, 0, r). */
ORC_API void orc_init_random(int q, int L, int64_t slot_begin, int64_t count, uint64_t seed, uint32_t stream,
                             uint8_t *spins)
{
    int N = L * L;
    for (int64_t r = 0; r < count; ++r) {
        uint32_t slot = (uint32_t)(slot_begin + r);
        for (int i = 0; i < N; ++i) {
            uint32_t w[4];
            orc_draw(seed, (uint32_t)i >> 2, ORC_DOM_INIT, 0u, slot | (stream << 24), w);
            spins[r * N + i] = (uint8_t)orc_scale(w[i & 3], (uint32_t)q);
        }
    }
}

/* Heating runs: every replica in one of the q ground states, chosen uniformly
 * (Sec. 5, Eq. 6).  Slot r takes word (r & 3) of counter (r >> 2, GROUND, 0, 0). */
ORC_API void orc_init_ground(int q, int L, int64_t slot_begin, int64_t count, uint64_t seed, uint32_t stream,
                             uint8_t *spins)
{
    int N = L * L;
    for (int64_t r = 0; r < count; ++r) {
        uint32_t slot = (uint32_t)(slot_begin + r);
        uint32_t w[4];
        orc_draw(seed, slot >> 2, ORC_DOM_GROUND, 0u, stream << 24, w);
        uint8_t alpha = (uint8_t)orc_scale(w[slot & 3], (uint32_t)q);
        for (int i = 0; i < N; ++i) spins[r * N + i] = alpha;
    }
}

/* ------------------------------------------------------------------------- */
/* Resampling (Sec. 2, step 2).                                                */
/* ------------------------------------------------------------------------- */
enum { ORC_NEAREST_INT = 0, ORC_ROUND = 1, ORC_POISSON = 2, ORC_OFF = 3 };

/* reading (the normaliser): Q_i = sum_j w_j / R_{i-1} is a sum of positive
 * doubles whose value the paper defines exactly.  S = sum_j w_j is taken as
 * that exact sum rounded once to the nearest double (ties to even), so it does
 * not depend on any summation order.  The accumulator below holds a sum of
 * non-negative finite doubles as an integer count of 2^-1074 (the smallest
 * positive double) in 32-bit limbs; limb k holds bits 32k .. 32k + 31. */
#define ORC_ACC_LIMBS 72

typedef struct {
    uint32_t limb[ORC_ACC_LIMBS];
} orc_acc;

/* adds v * 2^(32 k) with carry propagation */
static void orc_acc_add_word(orc_acc *a, int k, uint64_t v)
{
    while (v != 0) {
        uint64_t s = (uint64_t)a->limb[k] + (v & 0xFFFFFFFFu);
        a->limb[k] = (uint32_t)s;
        v = (v >> 32) + (s >> 32);
        k += 1;
    }
}

/* adds x (finite, >= 0): x = m 2^(pos - 1074) with m an integer below 2^53 */
static void orc_acc_add(orc_acc *a, double x)
{
    uint64_t m;
    int pos;
    if (x == 0.0) return;
    if (x < 2.2250738585072014e-308) { /* subnormal: a multiple of 2^-1074 */
        m = (uint64_t)ldexp(x, 1074);
        pos = 0;
    } else {
        int e;
        double f = frexp(x, &e); /* x = f 2^e, 1/2 <= f < 1 */
        m = (uint64_t)ldexp(f, 53);
        pos = e - 53 + 1074;
    }
    int k = pos / 32, sh = pos % 32;
    orc_acc_add_word(a, k, (m & 0xFFFFFFFFu) << sh);
    orc_acc_add_word(a, k + 1, (m >> 32) << sh);
}

static int orc_acc_bit(const orc_acc *a, int i)
{
    return (int)(a->limb[i / 32] >> (i % 32)) & 1;
}

/* The accumulated value rounded to the nearest double, ties to even. */
static double orc_acc_round(const orc_acc *a)
{
    int top = -1;
    for (int i = 32 * ORC_ACC_LIMBS - 1; i >= 0; --i) {
        if (orc_acc_bit(a, i)) {
            top = i;
            break;
        }
    }
    if (top < 0) return 0.0;
    uint64_t m = 0;
    if (top < 53) { /* at most 53 significant bits: exact */
        for (int i = top; i >= 0; --i) m = 2 * m + (uint64_t)orc_acc_bit(a, i);
        return ldexp((double)m, -1074);
    }
    for (int i = top; i > top - 53; --i) m = 2 * m + (uint64_t)orc_acc_bit(a, i);
    int round = orc_acc_bit(a, top - 53), sticky = 0;
    for (int i = top - 54; i >= 0 && !sticky; --i) sticky = orc_acc_bit(a, i);
    if (round && (sticky || (m & 1))) m += 1; /* m = 2^53 is still exact */
    return ldexp((double)m, top - 52 - 1074);
}

/* sum_j x[j] exact, rounded once (x[j] finite and >= 0). */
ORC_API double orc_exact_sum(int64_t n, const double *x)
{
    orc_acc a;
    memset(&a, 0, sizeof(a));
    for (int64_t j = 0; j < n; ++j) orc_acc_add(&a, x[j]);
    return orc_acc_round(&a);
}

/* reading (near ties): a copy number is flagged as a near tie when the
 * quantity its rule compares lies closer to the decision boundary than
 * delta = 2^-48 max(1, rho_j), a bound well above the rounding error rho_j can
 * carry (a few units in the last place): for nearest-integer copy numbers when
 * frac(rho_j) lies within delta of u_j / 2^32, for ROUND when it lies within
 * delta of 1/2, for Poisson draws when a uniform of the inversion lies within
 * 2^-40 of the cumulative probability it is compared with.  (A last-place
 * change that moves rho_j across an integer changes floor(rho_j) and frac
 * together and leaves r_j as it is, except through u_j = 0, which the first
 * test covers.)  The flag changes nothing; it counts the draws whose outcome a
 * last-place difference in rho_j could change. */

/* One copy number with mean rho, nearest-integer (u the replica's uniform
 * word) or ROUND; *tie receives the near-tie flag. */
ORC_API int32_t orc_round_copies(int mode, double rho, uint32_t u, int *tie)
{
    double n = floor(rho);
    double frac = rho - n;
    double delta = 0x1p-48 * (rho > 1.0 ? rho : 1.0);
    if (mode == ORC_ROUND) {
        *tie = fabs(frac - 0.5) < delta;
        return (int32_t)n + (frac >= 0.5);
    }
    *tie = fabs(frac - (double)u * 0x1p-32) < delta;
    return (int32_t)n + ((double)u < frac * 4294967296.0);
}

/* A Poisson draw with mean rho for replica j (Sec. 2, Eq. 1), by inversion of
 * the cumulative distribution, the mean split into pieces of at most 64 (a
 * sum of independent Poisson variables is Poisson with the summed mean, and
 * exp(-64) is far from underflow).  The k-th uniform, (U_k + 1/2) / 2^32, is
 * word k & 3 of counter (j, RESAMPLE | (1 + k / 4), step, stream << 24). */
static int32_t orc_poisson(double rho, int64_t j, uint32_t step, uint64_t seed, uint32_t stream, int *tie)
{
    int32_t r = 0;
    *tie = 0;
    double remaining = rho;
    uint32_t k = 0;
    uint32_t w[4] = {0, 0, 0, 0};
    while (remaining > 0.0) {
        double mu = remaining < 64.0 ? remaining : 64.0;
        remaining = remaining - mu;
        if ((k & 3) == 0) orc_draw(seed, (uint32_t)j, ORC_DOM_RESAMPLE | (1u + (k >> 2)), step, stream << 24, w);
        double u = ((double)w[k & 3] + 0.5) / 4294967296.0;
        k += 1;
        double p = exp(-mu);
        double F = p;
        int32_t n = 0;
        for (;;) {
            if (fabs(u - F) < 0x1p-40) *tie = 1;
            if (!(u > F && n < 1000)) break;
            n += 1;
            p = p * mu / (double)n;
            F = F + p;
        }
        r += n;
    }
    return r;
}

/* Computes Q_i and the copy numbers r_j for the R_prev replicas with energies
 * E[j], from beta_{i-1} to beta_i = beta_{i-1} + dbeta.
 *
 * The Boltzmann factors are evaluated relative to E_ref, the lowest energy for
 * dbeta >= 0 and the highest for dbeta < 0, so that no factor overflows:
 *   w_j = exp(-dbeta (E_j - E_ref)),  S = sum_j w_j (exact, rounded once),
 *   ln Q_i = -dbeta E_ref + ln(S / R_prev)          (= ln of the paper's Q_i),
 *   rho_j = (R w_j) / S                              (= (R/R_{i-1}) tau_i(E_j)).
 * reading: "nearest-integer" copy numbers draw r_j from the two integers
 * nearest to rho_j with the mean kept exact: r_j = floor(rho_j) + [u_j <
 * frac(rho_j) 2^32], u_j = word (j & 3) of counter (j >> 2, RESAMPLE, step,
 * stream << 24).  ORC_ROUND instead takes the nearest integer, halves rounded
 * up; ORC_POISSON draws r_j ~ Pois(rho_j), the paper's Eq. 1; ORC_OFF keeps
 * every replica once (the resampling-off comparison of Sec. 5, Fig. 2 right).
 * rho_out and tie_out (optional) receive rho_j and the near-tie flag of each
 * replica, n_ties (optional) the number of flagged replicas.  Returns the new
 * population size. */
ORC_API int64_t orc_copy_numbers(int64_t R_prev, const int32_t *E, double dbeta, int64_t R_target,
                                 int mode, uint32_t step, uint64_t seed, uint32_t stream, int32_t *r,
                                 double *lnQ, double *rho_out, int32_t *tie_out, int64_t *n_ties)
{
    int32_t E_ref = E[0];
    for (int64_t j = 1; j < R_prev; ++j) {
        if (dbeta >= 0.0 ? (E[j] < E_ref) : (E[j] > E_ref)) E_ref = E[j];
    }
    double *w = (double *)calloc((size_t)(R_prev > 0 ? R_prev : 1), sizeof(double));
    for (int64_t j = 0; j < R_prev; ++j) w[j] = exp(-dbeta * (double)(E[j] - E_ref));
    double S = orc_exact_sum(R_prev, w);
    *lnQ = -dbeta * (double)E_ref + log(S / (double)R_prev);
    int64_t total = 0, ties = 0;
    for (int64_t j = 0; j < R_prev; ++j) {
        double rho = ((double)R_target * w[j]) / S;
        if (rho_out) rho_out[j] = rho;
        int tie = 0;
        if (mode == ORC_POISSON) {
            r[j] = orc_poisson(rho, j, step, seed, stream, &tie);
        } else if (mode == ORC_OFF) {
            r[j] = 1;
        } else if (mode == ORC_ROUND) {
            r[j] = orc_round_copies(ORC_ROUND, rho, 0u, &tie);
        } else {
            uint32_t u[4];
            orc_draw(seed, (uint32_t)(j >> 2), ORC_DOM_RESAMPLE, step, stream << 24, u);
            r[j] = orc_round_copies(ORC_NEAREST_INT, rho, u[j & 3], &tie);
        }
        if (tie_out) tie_out[j] = tie;
        ties += tie;
        total += r[j];
    }
    free(w);
    if (n_ties) *n_ties = ties;
    return total;
}

/* Children in ascending parent order: parent[sum_{l<j} r_l + c] = j, c < r_j. */
ORC_API void orc_parents(int64_t R_prev, const int32_t *r, int32_t *parent)
{
    int64_t at = 0;
    for (int64_t j = 0; j < R_prev; ++j)
        for (int32_t c = 0; c < r[j]; ++c) parent[at++] = (int32_t)j;
}

/* ------------------------------------------------------------------------- */
/* Population estimators (Sec. 3, Eq. 4; Sec. 2 step 4).                       */
/* ------------------------------------------------------------------------- */
typedef struct {
    double beta, lnQ, lnZ, meanE, meanE2, C, meanM, S_f;
    int64_t R, n_families, sumE, sumE2, sumMt, n_near_ties;
} orc_obs;

/* Population averages over R replicas with energies E and largest-state
 * occupations Mt at inverse temperature beta:
 *   <E> = sum E / R, <E^2> = sum E^2 / R (integer sums, one division each),
 *   C = beta^2 (<E^2> - <E>^2) / N           (fluctuation formula),
 *   <M> = (q sum Mt - N R) / ((q-1) R)       (Eq. 5 averaged, Eq. 4).
 * Family entropy (reading; the paper does not define it): with n_f the number
 * of current replicas descending from initial replica f and nu_f = n_f / R,
 * S_f = -sum_f nu_f ln nu_f, summed over ascending f. */
static void orc_measure(int q, int N, int64_t R, const int32_t *E, const int32_t *Mt, double beta,
                        const int32_t *anc, int64_t R0, orc_obs *o)
{
    int64_t sE = 0, sE2 = 0, sM = 0;
    for (int64_t j = 0; j < R; ++j) {
        sE += E[j];
        sE2 += (int64_t)E[j] * (int64_t)E[j];
        sM += Mt[j];
    }
    o->R = R;
    o->sumE = sE; o->sumE2 = sE2; o->sumMt = sM;
    o->beta = beta;
    o->meanE = (double)sE / (double)R;
    o->meanE2 = (double)sE2 / (double)R;
    o->C = ((beta * beta) * (o->meanE2 - o->meanE * o->meanE)) / (double)N;
    o->meanM = (double)((int64_t)q * sM - (int64_t)N * R) / ((double)(q - 1) * (double)R);
    o->S_f = 0.0;
    o->n_families = 0;
    o->n_near_ties = 0;
    if (anc) {
        int64_t *count = (int64_t *)calloc((size_t)R0, sizeof(int64_t));
        for (int64_t j = 0; j < R; ++j) count[anc[j]] += 1;
        double sf = 0.0;
        for (int64_t f = 0; f < R0; ++f) {
            if (count[f] == 0) continue;
            double nu = (double)count[f] / (double)R;
            sf -= nu * log(nu);
            o->n_families += 1;
        }
        o->S_f = sf;
        free(count);
    }
}

/* ------------------------------------------------------------------------- */
/* The PA driver (Sec. 2, steps 1-5).                                          */
/* ------------------------------------------------------------------------- */
enum { ORC_INIT_RANDOM = 0, ORC_INIT_GROUND = 1 };

/* Runs K temperature steps over betas[0..K].  Step 0 is the initial
 * population at betas[0] (no sweeps there); step i >= 1 resamples from
 * betas[i-1] to betas[i], sweeps theta times at betas[i] and measures.
 *   obs[0..K]          per-step estimators (orc_obs, see above);
 *   hist (optional)    (K+1) x (2N+1) energy histograms, bin E + 2N;
 *   spins/E/anc        final population, R_cap * N bytes / R_cap ints;
 * ln Z_0 = N ln q for random starts (Sec. 6) and ln q - beta_0 E_0 with
 * E_0 = -2N for ground-state starts (Sec. 6, Eqs. 7-8).
 * Returns the final population size, or -1 if a population outgrew R_cap
 * (outputs then hold the last complete step). */
ORC_API int64_t orc_run(int q, int L, int64_t R, int64_t R_cap, uint64_t seed, uint32_t stream, int theta, int K,
                        const double *betas, int mode, int init_mode, orc_obs *obs, int32_t *hist,
                        uint8_t *spins_out, int32_t *E_out, int32_t *anc_out)
{
    int N = L * L;
    uint8_t *cur = (uint8_t *)malloc((size_t)R_cap * N);
    uint8_t *nxt = (uint8_t *)malloc((size_t)R_cap * N);
    int32_t *E = (int32_t *)malloc(sizeof(int32_t) * (size_t)R_cap);
    int32_t *Mt = (int32_t *)malloc(sizeof(int32_t) * (size_t)R_cap);
    int32_t *anc = (int32_t *)malloc(sizeof(int32_t) * (size_t)R_cap);
    int32_t *anc2 = (int32_t *)malloc(sizeof(int32_t) * (size_t)R_cap);
    int32_t *r = (int32_t *)malloc(sizeof(int32_t) * (size_t)R_cap);
    int32_t *parent = (int32_t *)malloc(sizeof(int32_t) * (size_t)R_cap);
    int64_t Rc = R;
    int64_t result = R;

    if (init_mode == ORC_INIT_GROUND)
        orc_init_ground(q, L, 0, R, seed, stream, cur);
    else
        orc_init_random(q, L, 0, R, seed, stream, cur);
    for (int64_t j = 0; j < R; ++j) {
        E[j] = (int32_t)orc_energy(L, cur + j * N);
        Mt[j] = (int32_t)orc_max_count(q, L, cur + j * N);
        anc[j] = (int32_t)j;
    }
    double lnZ;
    if (init_mode == ORC_INIT_GROUND)
        lnZ = log((double)q) - betas[0] * (double)(-2 * N);
    else
        lnZ = (double)N * log((double)q);
    orc_measure(q, N, Rc, E, Mt, betas[0], anc, R, &obs[0]);
    obs[0].lnQ = 0.0;
    obs[0].lnZ = lnZ;
    if (hist) {
        memset(hist, 0, sizeof(int32_t) * (size_t)(2 * N + 1));
        for (int64_t j = 0; j < Rc; ++j) hist[E[j] + 2 * N] += 1;
    }

    for (int i = 1; i <= K; ++i) {
        double dbeta = betas[i] - betas[i - 1];
        double lnQ;
        int64_t ties = 0;
        int64_t Rn = orc_copy_numbers(Rc, E, dbeta, R, mode, (uint32_t)i, seed, stream, r, &lnQ, NULL, NULL, &ties);
        if (Rn > R_cap || Rn <= 0) {
            result = -1;
            break;
        }
        orc_parents(Rc, r, parent);
        for (int64_t t = 0; t < Rn; ++t) {
            memcpy(nxt + t * N, cur + (int64_t)parent[t] * N, (size_t)N);
            anc2[t] = anc[parent[t]];
        }
        uint8_t *tmp = cur; cur = nxt; nxt = tmp;
        int32_t *ta = anc; anc = anc2; anc2 = ta;
        Rc = Rn;

        uint64_t thr[5];
        orc_thresholds(betas[i], thr);
        for (int64_t t = 0; t < Rc; ++t) {
            orc_sweep_replica(q, L, cur + t * N, thr, theta, (uint32_t)i, (uint32_t)t, seed, stream);
            E[t] = (int32_t)orc_energy(L, cur + t * N);
            Mt[t] = (int32_t)orc_max_count(q, L, cur + t * N);
        }
        lnZ = lnZ + lnQ;
        orc_measure(q, N, Rc, E, Mt, betas[i], anc, R, &obs[i]);
        obs[i].lnQ = lnQ;
        obs[i].lnZ = lnZ;
        obs[i].n_near_ties = ties;
        if (hist) {
            int32_t *h = hist + (int64_t)i * (2 * N + 1);
            memset(h, 0, sizeof(int32_t) * (size_t)(2 * N + 1));
            for (int64_t j = 0; j < Rc; ++j) h[E[j] + 2 * N] += 1;
        }
        result = Rc;
    }
    if (spins_out) memcpy(spins_out, cur, (size_t)Rc * N);
    if (E_out) memcpy(E_out, E, sizeof(int32_t) * (size_t)Rc);
    if (anc_out) memcpy(anc_out, anc, sizeof(int32_t) * (size_t)Rc);
    free(cur); free(nxt); free(E); free(Mt); free(anc); free(anc2); free(r); free(parent);
    return result;
}

ORC_API int orc_obs_size(void) { return (int)sizeof(orc_obs); }

/* ------------------------------------------------------------------------- */
/* Exact results on tiny lattices (pins for the oracle itself).               */
/* ------------------------------------------------------------------------- */

/* Density of states g(E) by visiting all q^N configurations; g[E + 2N].
 * Any L >= 2 (odd L allowed).  Returns 0, or -1 if q^N exceeds 2^40. */
ORC_API int orc_density_of_states(int q, int L, uint64_t *g)
{
    int N = L * L;
    double states = pow((double)q, (double)N);
    if (states > 1099511627776.0) return -1;
    for (int k = 0; k <= 2 * N; ++k) g[k] = 0;
    uint8_t s[64];
    memset(s, 0, sizeof(s));
    for (;;) {
        int64_t e = orc_energy(L, s);
        g[e + 2 * N] += 1;
        int i = 0;
        while (i < N) {
            s[i] += 1;
            if (s[i] < q) break;
            s[i] = 0;
            ++i;
        }
        if (i == N) break;
    }
    return 0;
}

/* Exact transition matrix of one Metropolis attempt at `site` (= y L + x) of an
 * L x L lattice, over all q^N configurations (index = sum_i s_i q^i).  The
 * probabilities are read off orc_metropolis_decide itself: each of the 2^B
 * equally likely (sigma, u) pairs is tried, and for each the acceptance
 * probability is the length of the set of v in [0, 2^32) that move the site,
 * found by bisection for its first rejecting v (the accepting v form a prefix),
 * so a mistake in the update rule shows up in the matrix.  P is (q^N)^2
 * row-major, P[a][b] = Prob(a -> b).  Returns -1 if q^N > 4096. */
ORC_API int orc_site_matrix(int q, int L, int site, double beta, double *P)
{
    int N = L * L;
    int64_t n = 1;
    for (int i = 0; i < N; ++i) n *= q;
    if (n > 4096) return -1;
    uint64_t thr[5];
    orc_thresholds(beta, thr);
    int B = orc_state_bits(q);
    int n_u = 1 << (B > 0 ? B - 1 : 0);
    double w = 1.0 / (2.0 * (double)n_u);
    memset(P, 0, sizeof(double) * (size_t)(n * n));
    int x = site % L, y = site / L;
    int64_t place = 1;
    for (int i = 0; i < site; ++i) place *= q;
    for (int64_t a = 0; a < n; ++a) {
        uint8_t s[64];
        int64_t t = a;
        for (int i = 0; i < N; ++i) { s[i] = (uint8_t)(t % q); t /= q; }
        int nb[4];
        orc_neighbours(L, s, x, y, nb);
        int cur = s[site];
        for (int sigma = 0; sigma < 2; ++sigma) {
            for (int u = 0; u < n_u; ++u) {
                /* smallest v in [0, 2^32] whose attempt leaves the site unchanged */
                uint64_t lo = 0, hi = 4294967296ull;
                while (lo < hi) {
                    uint64_t mid = (lo + hi) / 2;
                    if (orc_metropolis_decide(q, cur, nb, sigma, (uint32_t)u, (uint32_t)mid, thr) == cur)
                        hi = mid;
                    else
                        lo = mid + 1;
                }
                double p_acc = (double)lo / 4294967296.0;
                int prop = cur;
                if (lo > 0) prop = orc_metropolis_decide(q, cur, nb, sigma, (uint32_t)u, 0u, thr);
                int64_t b = a + (int64_t)(prop - cur) * place;
                P[a * n + b] += w * p_acc;
                P[a * n + a] += w * (1.0 - p_acc);
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Reweighting as a function of dbeta (Sec. 2, step 2), for the differentiable */
/* form:  ln Q(dbeta) = ln( sum_j exp(-dbeta E_j) / R ),                        */
/*   d ln Q / d dbeta = -<E>_tau,  d^2 ln Q / d dbeta^2 = var_tau(E),           */
/*   d var_tau(E) / d dbeta = -k3_tau(E) (third central moment),                */
/*   <O>_tau = sum_j O_j tau_j / R,  d <O>_tau / d dbeta = -cov_tau(O, E),      */
/* with tau_j = exp(-dbeta E_j) / Q.  Sums run over ascending j, shifted by     */
/* E_ref as in orc_copy_numbers.  out[0..7] = ln Q, <E>_tau, var_tau(E),         */
/* <O>_tau, cov_tau(O, E), E_ref, S (the shifted sum), k3_tau(E).               */
/* ------------------------------------------------------------------------- */
ORC_API void orc_reweight(int64_t R, const int32_t *E, const double *O, double dbeta, double out[8])
{
    int32_t E_ref = E[0];
    for (int64_t j = 1; j < R; ++j)
        if (dbeta >= 0.0 ? (E[j] < E_ref) : (E[j] > E_ref)) E_ref = E[j];
    /* moments about E_ref (a plain identity) keep var and cov free of cancellation */
    double S = 0.0, S1 = 0.0, S2 = 0.0, S3 = 0.0, SO = 0.0, SOe = 0.0;
    for (int64_t j = 0; j < R; ++j) {
        double e = (double)(E[j] - E_ref);
        double w = exp(-dbeta * e);
        S += w;
        S1 += w * e;
        S2 += w * e * e;
        S3 += w * e * e * e;
        if (O) {
            SO += w * O[j];
            SOe += w * O[j] * e;
        }
    }
    double m1 = S1 / S;
    double var = S2 / S - m1 * m1;
    out[0] = -dbeta * (double)E_ref + log(S / (double)R);
    out[1] = (double)E_ref + m1;
    out[2] = var;
    out[3] = O ? SO / S : 0.0;
    out[4] = O ? SOe / S - (SO / S) * m1 : 0.0;
    out[5] = (double)E_ref;
    out[6] = S;
    out[7] = S3 / S - 3.0 * m1 * (S2 / S) + 2.0 * m1 * m1 * m1;
}

/* ------------------------------------------------------------------------- */
/* Adaptive temperature step.  reading (the paper uses constant steps and does */
/* not define an overlap): with mean-one weights tau'_j = R w_j / S, the weight */
/* overlap between the populations at beta and beta + dbeta is                  */
/*   alpha(dbeta) = (1/R) sum_j min(1, tau'_j),                                  */
/*   alpha'(dbeta) = (1/R) sum_{tau'_j < 1} tau'_j (<E>_tau - E_j).             */
/* out[0..1] = alpha, alpha'.                                                     */
/* ------------------------------------------------------------------------- */
ORC_API void orc_overlap(int64_t R, const int32_t *E, double dbeta, double out[2])
{
    double rw[8];
    orc_reweight(R, E, NULL, dbeta, rw);
    double E_ref = rw[5], S = rw[6], mE = rw[1];
    double a = 0.0, da = 0.0;
    for (int64_t j = 0; j < R; ++j) {
        double t = ((double)R * exp(-dbeta * ((double)E[j] - E_ref))) / S;
        if (t < 1.0) {
            a += t;
            da += t * (mE - (double)E[j]);
        } else {
            a += 1.0;
        }
    }
    out[0] = a / (double)R;
    out[1] = da / (double)R;
}

/* reading: the step solves alpha(dbeta) = target on [0, dbeta_max] by Newton
 * iterations safeguarded by bisection: the bracket [lo, hi] starts as [0,
 * dbeta_max]; if alpha(dbeta_max) >= target the step is dbeta_max; otherwise
 * at most `iters` iterations follow from the bracket midpoint, stopping once
 * |alpha - target| <= 1e-12 (a step leaving the bracket is replaced by the
 * bracket midpoint; the bracket shrinks with each evaluation).  Stopping there,
 * far above rounding noise, keeps a converged iterate from being thrown back
 * by a bracket test decided by the last bit.  The result is rounded down to a
 * multiple of 2^-24 so that runs with a different last-bit rounding of alpha
 * agree, and so that beta + dbeta stays exact. */
ORC_API double orc_newton_dbeta(int64_t R, const int32_t *E, double target, double dbeta_max, int iters)
{
    double ov[2];
    orc_overlap(R, E, dbeta_max, ov);
    if (ov[0] >= target) return dbeta_max;
    double lo = 0.0, hi = dbeta_max;
    double x = 0.5 * (lo + hi);
    for (int it = 0; it < iters; ++it) {
        orc_overlap(R, E, x, ov);
        double f = ov[0] - target;
        if (fabs(f) <= 1e-12) break;
        if (f > 0.0) lo = x; else hi = x;
        double nx = ov[1] != 0.0 ? x - f / ov[1] : 0.5 * (lo + hi);
        if (!(nx > lo && nx < hi)) nx = 0.5 * (lo + hi);
        x = nx;
    }
    double q = floor(x * 16777216.0) / 16777216.0;
    return q > 0.0 ? q : 1.0 / 16777216.0;
}

/* The PA driver with the adaptive step: from beta_0 = 0, step i uses
 * dbeta_i = orc_newton_dbeta(E, target, min(dbeta_max, beta_end - beta), iters)
 * and beta_i = beta_{i-1} + dbeta_i, the last step landing on beta_end
 * exactly.  Otherwise as orc_run (random start, no histograms).  Writes up to
 * max_steps + 1 estimator records and betas; returns the number of steps K
 * taken (K <= max_steps), or -1 on a capacity overflow. */
ORC_API int orc_run_adaptive(int q, int L, int64_t R, int64_t R_cap, uint64_t seed, uint32_t stream, int theta,
                             double beta_end,
                             double target, double dbeta_max, int iters, int max_steps, int mode, orc_obs *obs,
                             double *betas, uint8_t *spins_out, int32_t *E_out)
{
    int N = L * L;
    uint8_t *cur = (uint8_t *)malloc((size_t)R_cap * N);
    uint8_t *nxt = (uint8_t *)malloc((size_t)R_cap * N);
    int32_t *E = (int32_t *)malloc(sizeof(int32_t) * (size_t)R_cap);
    int32_t *Mt = (int32_t *)malloc(sizeof(int32_t) * (size_t)R_cap);
    int32_t *r = (int32_t *)malloc(sizeof(int32_t) * (size_t)R_cap);
    int32_t *parent = (int32_t *)malloc(sizeof(int32_t) * (size_t)R_cap);
    int64_t Rc = R;
    orc_init_random(q, L, 0, R, seed, stream, cur);
    for (int64_t j = 0; j < R; ++j) {
        E[j] = (int32_t)orc_energy(L, cur + j * N);
        Mt[j] = (int32_t)orc_max_count(q, L, cur + j * N);
    }
    double beta = 0.0;
    double lnZ = (double)N * log((double)q);
    orc_measure(q, N, Rc, E, Mt, beta, NULL, R, &obs[0]);
    obs[0].lnQ = 0.0;
    obs[0].lnZ = lnZ;
    betas[0] = beta;
    int K = 0;
    while (beta < beta_end && K < max_steps) {
        double room = beta_end - beta;
        double cap = dbeta_max < room ? dbeta_max : room;
        double dbeta = orc_newton_dbeta(Rc, E, target, cap, iters);
        double nb = (dbeta == room) ? beta_end : beta + dbeta;
        int i = K + 1;
        double lnQ;
        int64_t ties = 0;
        int64_t Rn = orc_copy_numbers(Rc, E, dbeta, R, mode, (uint32_t)i, seed, stream, r, &lnQ, NULL, NULL, &ties);
        if (Rn > R_cap || Rn <= 0) {
            K = -1;
            break;
        }
        orc_parents(Rc, r, parent);
        for (int64_t t = 0; t < Rn; ++t) memcpy(nxt + t * N, cur + (int64_t)parent[t] * N, (size_t)N);
        uint8_t *tmp = cur; cur = nxt; nxt = tmp;
        Rc = Rn;
        uint64_t thr[5];
        orc_thresholds(nb, thr);
        for (int64_t t = 0; t < Rc; ++t) {
            orc_sweep_replica(q, L, cur + t * N, thr, theta, (uint32_t)i, (uint32_t)t, seed, stream);
            E[t] = (int32_t)orc_energy(L, cur + t * N);
            Mt[t] = (int32_t)orc_max_count(q, L, cur + t * N);
        }
        lnZ = lnZ + lnQ;
        orc_measure(q, N, Rc, E, Mt, nb, NULL, R, &obs[i]);
        obs[i].lnQ = lnQ;
        obs[i].lnZ = lnZ;
        obs[i].n_near_ties = ties;
        betas[i] = nb;
        beta = nb;
        K = i;
    }
    if (K >= 0) {
        if (spins_out) memcpy(spins_out, cur, (size_t)Rc * N);
        if (E_out) memcpy(E_out, E, sizeof(int32_t) * (size_t)Rc);
    }
    free(cur); free(nxt); free(E); free(Mt); free(r); free(parent);
    return K;
}
