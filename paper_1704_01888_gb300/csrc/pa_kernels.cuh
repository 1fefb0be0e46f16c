// pa_kernels.cuh -- device bodies of the population-annealing kernels
// (Barash, Weigel, Shchur & Janke, arXiv:1704.01888), shared by the
// single-run kernels (pa_resample.cu) and the batched kernels (pa_batch.cu)
// so that both run the same arithmetic.  The sweep body is in
// pa_sweep_body.cuh (included here).
//
// Initial populations and layout conversions; resampling bodies (Sec. 2
// step 2, Eq. 2): weights and ln Q, copy numbers and their scan, parent map;
// estimators (Sec. 2 step 4, Eqs. 4-5).
#pragma once
#include <climits>
#include <type_traits>

#include "pa_sweep_body.cuh"

namespace pa {
namespace dev {

// ===========================================================================
// Block reductions (fixed order)
// ===========================================================================
template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Fixed-order block sum of doubles; result valid in thread 0.
__device__ __forceinline__ double block_sum_fixed(double v, double *scratch32)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_down_sync(0xFFFFFFFFu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) scratch32[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        r = (lane < (int)(blockDim.x >> 5)) ? scratch32[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r = __dadd_rn(r, __shfl_down_sync(0xFFFFFFFFu, r, o));
    }
    __syncthreads();
    return r;
}

// Block sum of int64; every thread receives the result.
__device__ __forceinline__ long long block_sum_ll(long long v, long long *scratch32)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) scratch32[warp] = v;
    __syncthreads();
    long long r = 0;
    if (warp == 0) {
        r = (lane < (int)(blockDim.x >> 5)) ? scratch32[lane] : 0;
        r = warp_sum(r);
        if (lane == 0) scratch32[0] = r;
    }
    __syncthreads();
    r = scratch32[0];
    __syncthreads();
    return r;
}

// Block-wide exclusive scan of one int per thread; returns the exclusive
// prefix, writes the block total to *total.
__device__ __forceinline__ int block_exclusive_scan(int v, int *scratch32, int *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) scratch32[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int s = (lane < (int)(blockDim.x >> 5)) ? scratch32[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, s, o);
            if (lane >= o) s += y;
        }
        scratch32[lane] = s;  // inclusive prefix over warps
    }
    __syncthreads();
    const int before = (warp > 0 ? scratch32[warp - 1] : 0) + x - v;
    *total = scratch32[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

// ===========================================================================
// Initial populations (Sec. 2 step 1; Sec. 5 Eq. 6)
// ===========================================================================

// One site word (32 columns of one colour and row) of one replica; i indexes
// (slot, colour, row, word).  Random start: canonical site i_s = y L + x takes
// floor(Z q / 2^32), Z = word (i_s & 3) of the Philox call with counter
// (i_s >> 2, INIT, 0, slot | stream).  Ground start: every site of the replica
// in the state floor(Z q / 2^32), Z = word (slot & 3) of counter
// (slot >> 2, GROUND, 0, stream).
__device__ __forceinline__ void init_item(uint32_t *spins, int32_t *anc, int q, int L, long long i, uint32_t k0,
                                          uint32_t k1, uint32_t stream_hi, int ground, uint32_t slot0 = 0u)
{
    const int B = state_bits(q);
    const int BP = plane_stride(B);
    const int WPR = row_words(L);
    const int nb_last = L / 2 - 32 * (WPR - 1);
    const int IPC = colour_words(L);
    const int IPR = 2 * IPC;  // site words per replica
    const int slot = (int)(i / IPR);
    const int rem = (int)(i - (long long)slot * IPR);
    const int c = rem / IPC;
    const int it = rem - c * IPC;
    const bool packed = rows_packed(L), banded = rows_banded(L);
    const int nb = (packed || banded) ? 32 : ((it % WPR) == WPR - 1 ? nb_last : 32);
    uint32_t planes[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    const uint32_t key_slot = slot0 + (uint32_t)slot;  // the random numbers follow the global slot
    if (ground) {
        const uint4 w = philox10(make_uint4(key_slot >> 2, DOM_GROUND, 0u, stream_hi), k0, k1);
        const uint32_t alpha = __umulhi(pick_word(w, key_slot & 3), (uint32_t)q);
        const uint32_t vm = nb == 32 ? 0xFFFFFFFFu : ((1u << nb) - 1u);
        for (int p = 0; p < B; ++p) planes[p] = ((alpha >> p) & 1u) ? vm : 0u;
    } else {
        int last = -1;
        uint4 w = make_uint4(0u, 0u, 0u, 0u);
        for (int b = 0; b < nb; ++b) {
            int y, m;
            if (packed) {
                const int h = 32 * it + b;
                y = h / (L / 2);
                m = h - y * (L / 2);
            } else if (banded) {
                const int k = it / (L / 16);
                y = k + (b >> 3) * (L / 4);
                m = 8 * (it - k * (L / 16)) + (b & 7);
            } else {
                y = it / WPR;
                m = 32 * (it - y * WPR) + b;
            }
            const int x = 2 * m + ((y + c) & 1);
            const int site = y * L + x;
            if ((site >> 2) != last) {
                last = site >> 2;
                w = philox10(make_uint4((uint32_t)last, DOM_INIT, 0u, key_slot | stream_hi), k0, k1);
            }
            const uint32_t s = __umulhi(pick_word(w, site & 3), (uint32_t)q);
            for (int p = 0; p < B; ++p) planes[p] |= ((s >> p) & 1u) << b;
        }
    }
    uint32_t *dst = spins + (size_t)slot * replica_words_of(B, L) + (size_t)rem * BP;
    for (int p = 0; p < BP; ++p) dst[p] = planes[p];
    if (rem == 0 && anc) anc[slot] = (int32_t)key_slot;
}

// One site word (i indexes (slot, colour, word) as in init_item) of the
// multi-spin-coded layout from a population in the canonical layout
// [slot][y][x], one byte per spin (the inverse of canonical_state).
__device__ __forceinline__ void from_canonical_item(uint32_t *spins, const uint8_t *canon, int q, int L, long long i)
{
    const int B = state_bits(q);
    const int BP = plane_stride(B);
    const int WPR = row_words(L);
    const int nb_last = L / 2 - 32 * (WPR - 1);
    const int IPC = colour_words(L);
    const int IPR = 2 * IPC;
    const long long slot = i / IPR;
    const int rem = (int)(i - slot * IPR);
    const int c = rem / IPC;
    const int it = rem - c * IPC;
    const bool packed = rows_packed(L), banded = rows_banded(L);
    const int nb = (packed || banded) ? 32 : ((it % WPR) == WPR - 1 ? nb_last : 32);
    const uint8_t *rep = canon + slot * (long long)L * L;
    uint32_t planes[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    for (int b = 0; b < nb; ++b) {
        int y, m;
        if (packed) {
            const int h = 32 * it + b;
            y = h / (L / 2);
            m = h - y * (L / 2);
        } else if (banded) {
            const int k = it / (L / 16);
            y = k + (b >> 3) * (L / 4);
            m = 8 * (it - k * (L / 16)) + (b & 7);
        } else {
            y = it / WPR;
            m = 32 * (it - y * WPR) + b;
        }
        const uint32_t s = rep[y * L + 2 * m + ((y + c) & 1)];
        for (int p = 0; p < B; ++p) planes[p] |= ((s >> p) & 1u) << b;
    }
    uint32_t *dst = spins + (size_t)slot * replica_words_of(B, L) + (size_t)rem * BP;
    for (int p = 0; p < BP; ++p) dst[p] = planes[p];
}

// State of canonical site i (= r N + y L + x) of a multi-spin-coded population.
__device__ __forceinline__ uint8_t canonical_state(const uint32_t *spins, int q, int L, long long i)
{
    const int N = L * L;
    const int B = state_bits(q);
    const int BP = plane_stride(B);
    const int IPC = colour_words(L);
    const long long r = i / N;
    const int site = (int)(i - r * N);
    const int y = site / L, x = site - y * L;
    const int c = (x + y) & 1;
    const int m = x >> 1;
    int it, b;
    if (rows_packed(L)) {
        const int h = y * (L / 2) + m;
        it = h >> 5;
        b = h & 31;
    } else if (rows_banded(L)) {
        const int a = y / (L / 4), k = y - a * (L / 4);
        it = k * (L / 16) + (m >> 3);
        b = 8 * a + (m & 7);
    } else {
        it = y * row_words(L) + (m >> 5);
        b = m & 31;
    }
    const uint32_t *w = spins + (size_t)r * replica_words_of(B, L) + (size_t)((c * IPC + it) * BP);
    uint32_t s = 0;
    for (int p = 0; p < B; ++p) s |= ((w[p] >> b) & 1u) << p;
    return (uint8_t)s;
}

// ===========================================================================
// Resampling bodies (Sec. 2 step 2, Eq. 2)
// ===========================================================================

// Exact sum of the weights.  S = sum_k h_k w_k over the occupied energy bins
// (h_k < 2^24 replicas, w_k a double in [0, 1]) is accumulated exactly and
// rounded once to the nearest double, ties to even, so that S -- and with it
// every rho_j -- does not depend on which lane, warp or block adds which term.
// The accumulator counts units of 2^-1074 (the smallest positive double): a
// term h m 2^(pos - 1074) (m the 53-bit significand) is the integer h m < 2^77
// placed at bit pos <= 1022.  Limb i of the shared array collects bits
// 32 i .. 32 i + 31 in a 64-bit counter, so the carries of up to 2^32
// additions fit and are propagated once, at the end.  The sum is below
// R_cap < 2^24, i.e. below bit 1098: 36 limbs.
constexpr int kSumLimbs = 36;

// The term h w (w > 0) as four 32-bit chunks c[0..3] of limbs li .. li + 3.
__device__ __forceinline__ int exact_term(uint32_t h, double w, uint32_t (&c)[4])
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(w);
    const int ef = (int)(bits >> 52) & 0x7FF;
    const unsigned long long m = (bits & 0xFFFFFFFFFFFFFull) | (ef ? (1ull << 52) : 0ull);
    const int pos = ef ? ef - 1 : 0;
    const unsigned long long lo = m * (unsigned long long)h;
    const unsigned long long hi = __umul64hi(m, (unsigned long long)h);
    const int sh = pos & 31;
    const unsigned long long lo_s = lo << sh;
    const unsigned long long hi_s = (hi << sh) | (sh ? lo >> (64 - sh) : 0ull);
    c[0] = (uint32_t)lo_s;
    c[1] = (uint32_t)(lo_s >> 32);
    c[2] = (uint32_t)hi_s;
    c[3] = (uint32_t)(hi_s >> 32);
    return pos >> 5;
}

// Adds the terms of the occupied bins among k_begin .. k_end - 1 to the
// shared limbs.  Consecutive bins have weights within a few binades of one
// another, so a thread sums its terms in five register limbs (li - 1 .. li +
// 3 of the first term) and adds them to the shared array only when a term
// falls outside them: a handful of shared atomics per thread instead of four
// per term.
__device__ __forceinline__ void exact_add_range(unsigned long long *acc, const int32_t *hist, const double *wtab,
                                                int kref, int k_begin, int k_end)
{
    unsigned long long w0 = 0ull, w1 = 0ull, w2 = 0ull, w3 = 0ull, w4 = 0ull;
    int base = -2;
    auto flush = [&]() {
        if (base < 0) return;
        if (w0) atomicAdd(acc + base, w0);
        if (w1) atomicAdd(acc + base + 1, w1);
        if (w2) atomicAdd(acc + base + 2, w2);
        if (w3) atomicAdd(acc + base + 3, w3);
        if (w4) atomicAdd(acc + base + 4, w4);
        w0 = w1 = w2 = w3 = w4 = 0ull;
    };
    // four bins at a time: their loads issue together
    for (int k0 = k_begin; k0 < k_end; k0 += 4) {
        int h[4];
        double wk[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) h[i] = k0 + i < k_end ? hist[k0 + i] : 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int k = k0 + i;
            wk[i] = h[i] > 0 ? wtab[k >= kref ? k - kref : kref - k] : 0.0;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (h[i] <= 0 || wk[i] == 0.0) continue;
            uint32_t c[4];
            const int li = exact_term((uint32_t)h[i], wk[i], c);
            if (li < base || li > base + 1) {
                flush();
                base = li > 0 ? li - 1 : 0;
            }
            if (li == base) {
                w0 += c[0];
                w1 += c[1];
                w2 += c[2];
                w3 += c[3];
            } else {
                w1 += c[0];
                w2 += c[1];
                w3 += c[2];
                w4 += c[3];
            }
        }
    }
    flush();
}

// Bits lowpos .. lowpos + 63 of normalised 32-bit limbs (lowpos >= 0).
__device__ __forceinline__ unsigned long long limb_bits64(const unsigned long long *acc, int lowpos)
{
    const int li = lowpos >> 5, sh = lowpos & 31;
    auto limb = [&](int i) -> unsigned long long { return i < kSumLimbs ? acc[i] : 0ull; };
    const unsigned long long lo64 = limb(li) | (limb(li + 1) << 32);
    return sh ? (lo64 >> sh) | (limb(li + 2) << (64 - sh)) : lo64;
}

// Propagates the carries and rounds the accumulated value to the nearest
// double (one thread; the value must be at least 1, i.e. bit 1074 or above).
__device__ __forceinline__ double exact_round(unsigned long long *acc)
{
    unsigned long long carry = 0ull;
    for (int i = 0; i < kSumLimbs; ++i) {
        const unsigned long long v = acc[i] + carry;
        acc[i] = v & 0xFFFFFFFFull;
        carry = v >> 32;
    }
    int t = kSumLimbs - 1;
    while (t > 0 && acc[t] == 0ull) --t;
    int p = 32 * t + 31 - __clz((uint32_t)acc[t]);  // top bit
    const unsigned long long x = limb_bits64(acc, p - 63);  // bit 63 = top bit
    unsigned long long mant = x >> 11;
    const bool round = (x >> 10) & 1ull;
    bool sticky = (x & 0x3FFull) != 0ull;
    const int low = p - 63;  // bits below it
    for (int i = 0; i < (low >> 5) && !sticky; ++i) sticky = acc[i] != 0ull;
    if (!sticky && (low & 31)) sticky = (acc[low >> 5] & ((1ull << (low & 31)) - 1ull)) != 0ull;
    if (round && (sticky || (mant & 1ull))) mant += 1ull;
    if (mant >> 53) {
        mant >>= 1;
        p += 1;
    }
    // value = mant 2^(p - 52 - 1074): biased exponent p - 1074 + 1023
    return __longlong_as_double((long long)(((unsigned long long)(p - 51) << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

// One block: reference bin, S (exact sum of h_k w_k, weights from the host
// table wtab by distance |k - k_ref|) and ln Q of the pending resample.
// R_prev_all: the population size R_{i-1} when the histogram covers several
// GPUs' replicas (0: this GPU's own, st->pop).
__device__ __forceinline__ void weights_body(const int32_t *hist, int nbins, double dbeta, const double *wtab,
                                             DevState *st, unsigned long long *s_acc, long long *s_l,
                                             int R_prev_all = 0)
{
    if (st->err) return;
    const int tid = threadIdx.x;
    // reference bin: lowest occupied for dbeta >= 0, highest for dbeta < 0
    long long best = dbeta >= 0.0 ? (long long)INT_MAX : -1;
#pragma unroll 4
    for (int k = tid; k < nbins; k += blockDim.x) {
        if (hist[k] > 0) best = dbeta >= 0.0 ? min(best, (long long)k) : max(best, (long long)k);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long other = __shfl_down_sync(0xFFFFFFFFu, best, o);
        best = dbeta >= 0.0 ? min(best, other) : max(best, other);
    }
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0) s_l[warp] = best;
    for (int i = tid; i < kSumLimbs; i += blockDim.x) s_acc[i] = 0ull;
    __syncthreads();
    if (warp == 0) {
        long long v = (lane < (int)(blockDim.x >> 5)) ? s_l[lane] : (dbeta >= 0.0 ? (long long)INT_MAX : -1);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long other = __shfl_down_sync(0xFFFFFFFFu, v, o);
            v = dbeta >= 0.0 ? min(v, other) : max(v, other);
        }
        if (lane == 0) s_l[0] = v;
    }
    __syncthreads();
    const int kref = (int)s_l[0];
    const int per = (nbins + (int)blockDim.x - 1) / (int)blockDim.x;  // a contiguous range of bins per thread
    exact_add_range(s_acc, hist, wtab, kref, min(nbins, tid * per), min(nbins, (tid + 1) * per));
    __syncthreads();
    if (tid == 0) {
        const double S = exact_round(s_acc);
        const int E_ref = kref - (nbins - 1);
        st->S = S;
        st->E_ref = E_ref;
        st->ties = 0;
        const int R_prev = R_prev_all > 0 ? R_prev_all : st->pop;
        st->lnQ = __dadd_rn(__dmul_rn(-dbeta, (double)E_ref), log(S / (double)R_prev));
    }
    __syncthreads();
}

// A Poisson draw with mean rho for replica j (Sec. 2, Eq. 1): inversion of
// the cumulative distribution with the mean split into pieces of at most 64;
// the k-th uniform (U_k + 1/2) / 2^32 is word k & 3 of counter
// (j, RESAMPLE | (1 + k / 4), step, stream).
__device__ __forceinline__ int poisson_draw(double rho, int j, int step, uint32_t stream_hi, uint32_t k0, uint32_t k1,
                                            bool &tie)
{
    int r = 0;
    tie = false;
    double remaining = rho;
    uint32_t k = 0;
    uint4 w = make_uint4(0u, 0u, 0u, 0u);
    while (remaining > 0.0) {
        const double mu = remaining < 64.0 ? remaining : 64.0;
        remaining = __dsub_rn(remaining, mu);
        if ((k & 3) == 0)
            w = philox10(make_uint4((uint32_t)j, DOM_RESAMPLE | (1u + (k >> 2)), (uint32_t)step, stream_hi), k0, k1);
        const double u = __ddiv_rn(__dadd_rn((double)pick_word(w, k & 3), 0.5), 4294967296.0);
        k += 1;
        double p = exp(-mu);
        double F = p;
        int n = 0;
        for (;;) {
            if (fabs(__dsub_rn(u, F)) < 0x1p-40) tie = true;
            if (!(u > F && n < 1000)) break;
            n += 1;
            p = __ddiv_rn(__dmul_rn(p, mu), (double)n);
            F = __dadd_rn(F, p);
        }
        r += n;
    }
    return r;
}

// Near-tie flag of a rounded copy number: frac(rho) within 2^-48 max(1, rho)
// of the rule's boundary (u / 2^32 for nearest-integer copy numbers, 1/2 for
// ROUND), where a last-place change of rho could change the outcome.
__device__ __forceinline__ bool round_tie(double rho, double frac, double boundary)
{
    return fabs(__dsub_rn(frac, boundary)) < __dmul_rn(0x1p-48, fmax(1.0, rho));
}

// One block of 1024 old replicas (chunk): copy numbers and their block scan.
// w(E_j) comes from the host table wtab by distance |E_j - E_ref|.
// j0: global index of local replica 0 (a population shared by several GPUs):
// the random numbers of replica j follow j0 + j.
__device__ __forceinline__ void counts_body(int chunk, const int32_t *E, int twoN, int R_target, int mode, int step,
                                            uint32_t stream_hi, uint32_t k0, uint32_t k1, const double *wtab,
                                            int32_t *counts, int32_t *local_off, int32_t *blocksum, DevState *st,
                                            int *s_i, int j0 = 0)
{
    if (st->err) return;
    const int R_prev = st->pop;
    if (chunk * (int)blockDim.x >= R_prev) return;
    const int j = chunk * blockDim.x + threadIdx.x;
    int r = 0;
    bool tie = false;
    if (j < R_prev) {
        const int d = E[j] - st->E_ref;
        const double w = wtab[d >= 0 ? d : -d];
        const double rho = __ddiv_rn(__dmul_rn((double)R_target, w), st->S);
        const double n = floor(rho);
        const double frac = __dsub_rn(rho, n);
        const int jg = j0 + j;
        if (mode == 2) {
            r = poisson_draw(rho, jg, step, stream_hi, k0, k1, tie);
        } else if (mode == 3) {
            r = 1;
        } else if (mode == 1) {
            r = (int)n + (frac >= 0.5);
            tie = round_tie(rho, frac, 0.5);
        } else {
            const uint4 u = philox10(make_uint4((uint32_t)jg >> 2, DOM_RESAMPLE, (uint32_t)step, stream_hi), k0, k1);
            const uint32_t uj = pick_word(u, jg & 3);
            r = (int)n + ((double)uj < __dmul_rn(frac, 4294967296.0));
            tie = round_tie(rho, frac, __dmul_rn((double)uj, 0x1p-32));
        }
        counts[j] = r;
    }
    const unsigned nt = __popc(__ballot_sync(0xFFFFFFFFu, tie));
    if ((threadIdx.x & 31) == 0 && nt) atomicAdd(&st->ties, (int)nt);
    int total;
    const int before = block_exclusive_scan(r, s_i, &total);
    if (j < R_prev) local_off[j] = before;
    if (threadIdx.x == 0) blocksum[chunk] = total;
}

// One block (chunk of nchunks): block offsets, new size (capacity check),
// parent map; the chunks also clear the histogram for the next sweep.
// min_total: smallest valid number of children (1; 0 for one GPU's share of
// a population spread over several, which may receive all its replicas from
// the others).
__device__ __forceinline__ void scatter_body(int chunk, int nchunks, const int32_t *counts, const int32_t *local_off,
                                             const int32_t *blocksum, int32_t *parent, int R_cap, int32_t *hist_zero,
                                             int nbins, DevState *st, long long *s_l, int min_total = 1)
{
    if (st->err) return;
    const int R_prev = st->pop;
    const int nb = (R_prev + blockDim.x - 1) / blockDim.x;
    long long off = 0, tot = 0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const long long v = blocksum[b];
        tot += v;
        if (b < chunk) off += v;
    }
    tot = block_sum_ll(tot, s_l);
    off = block_sum_ll(off, s_l);
    if (tot > R_cap || tot < min_total) {
        if (chunk == 0 && threadIdx.x == 0) st->err = 2;  // PA_ERR_CAPACITY
        return;
    }
    if (chunk == 0 && threadIdx.x == 0) st->pop_next = (int)tot;
    for (int k = chunk * blockDim.x + threadIdx.x; k < nbins; k += nchunks * blockDim.x) hist_zero[k] = 0;
    if (chunk >= nb) return;
    const int j = chunk * blockDim.x + threadIdx.x;
    if (j < R_prev) {
        const int o = (int)off + local_off[j];
        const int r = counts[j];
        for (int c = 0; c < r; ++c) parent[o + c] = j;
    }
}

// One block: estimators of the step (Sec. 2 step 4, Eqs. 4-5), family
// entropy, ln Z of Eq. 2, buffer parity flip.
// R_all: the population size when the sums and family counts cover several
// GPUs' replicas (0: this GPU's own).
__device__ __forceinline__ void finalize_body(DevState *st, unsigned long long *acc, int32_t *fam, int R0, DevObs *obs,
                                              double beta, int q, int N, int gathered, int resampled, double *s_d,
                                              long long *s_l, int R_all = 0)
{
    if (st->err) return;
    const int R_local = gathered ? st->pop_next : st->pop;
    const int R = R_all > 0 ? R_all : R_local;
    double part = 0.0;
    long long nf = 0;
    if (fam) {
        for (int f = threadIdx.x; f < R0; f += blockDim.x) {
            const int c = fam[f];
            if (c > 0) {
                const double nu = (double)c / (double)R;
                part = __dsub_rn(part, __dmul_rn(nu, log(nu)));
                nf += 1;
                fam[f] = 0;
            }
        }
    }
    const double Sf = block_sum_fixed(part, s_d);
    nf = block_sum_ll(nf, s_l);
    if (threadIdx.x == 0) {
        const long long sE = (long long)acc[0], sE2 = (long long)acc[1], sM = (long long)acc[2];
        acc[0] = acc[1] = acc[2] = 0ull;
        const double meanE = (double)sE / (double)R;
        const double meanE2 = (double)sE2 / (double)R;
        const double C =
            __ddiv_rn(__dmul_rn(__dmul_rn(beta, beta), __dsub_rn(meanE2, __dmul_rn(meanE, meanE))), (double)N);
        const double meanM = (double)((long long)q * sM - (long long)N * R) / __dmul_rn((double)(q - 1), (double)R);
        double lnQ = 0.0;
        if (resampled) {
            lnQ = st->lnQ;
            st->lnZ = __dadd_rn(st->lnZ, lnQ);
        }
        if (gathered) {
            st->pop = R_local;
            st->parity ^= 1;
        }
        DevObs o;
        o.beta = beta;
        o.lnQ = lnQ;
        o.lnZ = st->lnZ;
        o.meanE = meanE;
        o.meanE2 = meanE2;
        o.C = C;
        o.meanM = meanM;
        o.S_f = fam ? Sf : 0.0;
        o.R = R;
        o.n_families = fam ? nf : 0;
        // several GPUs: acc[3] holds the near ties summed over them
        o.n_near_ties = resampled ? (R_all > 0 ? (long long)acc[3] : (long long)st->ties) : 0;
        if (R_all > 0) acc[3] = 0ull;
        o.sumE = sE;
        o.sumE2 = sE2;
        o.sumMt = sM;
        *obs = o;
    }
}

}  // namespace dev
}  // namespace pa
