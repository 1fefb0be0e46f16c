// pa_sweep_body.cuh -- device body of the Metropolis sweep of population
// annealing (Barash, Weigel, Shchur & Janke, arXiv:1704.01888, Sec. 2 step 3
// and Sec. 3), with the replica gather of step 2 fused into its load and the
// measurements of step 4 (Eq. 3 energy, Eq. 5 largest-state occupation, the
// energy histogram) in its epilogue.  Shared by the single-run sweep kernel
// (pa_sweep.cu) and the batched sweep kernels (pa_batch.cuh).
//
// One block holds a group of whole lattices in shared memory and runs theta
// checkerboard sweeps on them.  Spins are multi-spin coded (layout in
// pa_internal.cuh): every logic instruction of the update acts on the 32 sites
// of one site word.
#pragma once
#include <climits>
#include <type_traits>

#include "pa_internal.cuh"

namespace pa {
namespace dev {

// ===========================================================================
// Bit-plane helpers
// ===========================================================================

// BP consecutive words (the planes of one site word): one 16-byte access per
// four planes (BP = 4: the site word's planes start on a 16-byte boundary),
// 8-byte accesses for BP = 2 and 6, single words for BP = 1, 5 and 7 (a
// warp's loads of one plane then fall in distinct banks: the words of
// consecutive site words lie an odd number of words apart).
template <int BP>
__device__ __forceinline__ void load_planes(uint32_t (&v)[BP], const uint32_t *src)
{
    if constexpr (BP % 4 == 0) {
#pragma unroll
        for (int h = 0; h < BP / 4; ++h) {
            const uint4 a = reinterpret_cast<const uint4 *>(src)[h];
            v[4 * h + 0] = a.x;
            v[4 * h + 1] = a.y;
            v[4 * h + 2] = a.z;
            v[4 * h + 3] = a.w;
        }
    } else if constexpr (BP % 2 == 0) {
#pragma unroll
        for (int h = 0; h < BP / 2; ++h) {
            const uint2 a = reinterpret_cast<const uint2 *>(src)[h];
            v[2 * h + 0] = a.x;
            v[2 * h + 1] = a.y;
        }
    } else {
#pragma unroll
        for (int p = 0; p < BP; ++p) v[p] = src[p];
    }
}

template <int BP>
__device__ __forceinline__ void store_planes(uint32_t *dst, const uint32_t (&v)[BP])
{
    if constexpr (BP % 4 == 0) {
#pragma unroll
        for (int h = 0; h < BP / 4; ++h)
            reinterpret_cast<uint4 *>(dst)[h] = make_uint4(v[4 * h], v[4 * h + 1], v[4 * h + 2], v[4 * h + 3]);
    } else if constexpr (BP % 2 == 0) {
#pragma unroll
        for (int h = 0; h < BP / 2; ++h) reinterpret_cast<uint2 *>(dst)[h] = make_uint2(v[2 * h], v[2 * h + 1]);
    } else {
#pragma unroll
        for (int p = 0; p < BP; ++p) dst[p] = v[p];
    }
}

// Bit set where the B-bit states held in planes a and b differ.
template <int B, int BP>
__device__ __forceinline__ uint32_t differ(const uint32_t (&a)[BP], const uint32_t (&b)[BP])
{
    uint32_t d = a[0] ^ b[0];
#pragma unroll
    for (int p = 1; p < B; ++p) d |= a[p] ^ b[p];
    return d;
}

// Bit set where the B-bit state in planes a equals the constant state s.
template <int B, int BP>
__device__ __forceinline__ uint32_t equal_state(const uint32_t (&a)[BP], int s)
{
    uint32_t d = 0;
#pragma unroll
    for (int p = 0; p < B; ++p) d |= a[p] ^ (((s >> p) & 1) ? 0xFFFFFFFFu : 0u);
    return ~d;
}

// Division by a divisor d fixed for a replica group (d < 2^15) of x < 2^16,
// without a division instruction sequence per use: with inv = ceil(2^31 / d)
// = (2^31 + e) / d, 0 <= e < d, floor(x inv / 2^31) = floor(x / d) because
// x e < x d < 2^31.
__device__ __forceinline__ uint32_t div_inverse(uint32_t d) { return (uint32_t)((0x80000000ull + d - 1u) / d); }
__device__ __forceinline__ int div_by(int x, uint32_t inv) { return (int)__umulhi((uint32_t)x << 1, inv); }

__device__ __forceinline__ void full_add(uint32_t a, uint32_t b, uint32_t c, uint32_t &sum, uint32_t &carry)
{
    sum = a ^ b ^ c;
    carry = (a & b) | (c & (a ^ b));
}

// Valid-column mask of word t of a row with WPR words and nb_last valid bits
// in its last word.
__device__ __forceinline__ uint32_t valid_mask(int t, int WPR, int nb_last)
{
    return (t < WPR - 1 || nb_last == 32) ? 0xFFFFFFFFu : ((1u << nb_last) - 1u);
}

// The row word H (other colour, row y) shifted so that bit b holds the
// horizontal neighbour of column 32 t + b that is not at the same column:
// column m + 1 when par = 1, column m - 1 when par = 0 (par = (x & 1) of the
// row's sites).  E is the adjacent word of the row (t + 1 for par = 1, t - 1
// for par = 0, cyclically); MODE 0 is L = 64 (one full word per row), MODE 1
// rows of full words, MODE 2 rows whose last word holds nb_last < 32 columns.
template <int MODE>
__device__ __forceinline__ uint32_t shifted_row(uint32_t H, uint32_t E, int par, int nb, int nbe)
{
    if constexpr (MODE == 0) {
        return __funnelshift_l(H, H, par ? 31 : 1);
    } else if constexpr (MODE == 1) {
        return par ? __funnelshift_r(H, E, 1) : __funnelshift_r(E, H, 31);
    } else {
        return par ? ((H >> 1) | ((E & 1u) << (nb - 1))) : ((H << 1) | ((E >> (nbe - 1)) & 1u));
    }
}

// Packed rows (MODE 3, L = 8, 16, 32): the horizontal neighbour word of H.
// Each word holds 32 / S rows of S = L/2 columns; in a row whose sites sit at
// odd x (par = 1) the neighbour not at the same column is column m + 1, else
// m - 1, both cyclic within the row's S-bit segment.  Rows alternate par, and
// `odd` marks the segments with par = 1 (the same in every word of a colour).
template <int S>
__device__ __forceinline__ uint32_t shifted_packed(uint32_t H, uint32_t odd)
{
    constexpr uint32_t bot = S == 4 ? 0x11111111u : S == 8 ? 0x01010101u : 0x00010001u;
    constexpr uint32_t top = bot << (S - 1);
    const uint32_t right = ((H >> 1) & ~top) | ((H << (S - 1)) & top);  // column m + 1
    const uint32_t left = ((H << 1) & ~bot) | ((H >> (S - 1)) & bot);   // column m - 1
    return (odd & right) | (~odd & left);
}

template <int S>
__device__ __forceinline__ constexpr uint32_t odd_segments()
{
    return S == 4 ? 0xF0F0F0F0u : S == 8 ? 0xFF00FF00u : 0xFFFF0000u;
}

// The four neighbour words of site word `it` (its index within its colour) of
// colour c: up, down and same-row words of the other colour (oth) and the
// same-row word shifted by one column.  Returns the mask of the word's valid
// columns.  MODE as for shifted_row, 3 for packed rows, 4 for banded rows;
// inv_row = div_inverse of the words per row (MODE 1, 2) or of the segments
// per row (MODE 4).
template <int B, int MODE, int BP>
__device__ __forceinline__ uint32_t neighbour_planes(const uint32_t *oth, int L, int IPC, int WPR, int nb_last,
                                                     uint32_t inv_row, int it, int c, uint32_t (&U)[BP],
                                                     uint32_t (&D)[BP], uint32_t (&H)[BP], uint32_t (&X)[BP])
{
    if constexpr (MODE == 4) {
        // word (k, j): segment j of rows k + a L/4 in byte a.  The rows above
        // and below are the same bytes of words (k -+ 1, j), except across the
        // band edges: above row 0 of a band lies the last row of the band
        // before (byte a - 1 of word (L/4 - 1, j), cyclically), below its last
        // row the first row of the next band (byte a + 1 of word (0, j)).
        const int segs = L >> 4, band_rows = L >> 2;
        const int k = div_by(it, inv_row), j = it - k * segs;
        const int ku = k == 0 ? band_rows - 1 : k - 1;
        const int kd = k == band_rows - 1 ? 0 : k + 1;
        const int par = (k + c) & 1;  // band heights are even: one parity per word
        const int je = par ? (j + 1 == segs ? 0 : j + 1) : (j == 0 ? segs - 1 : j - 1);
        uint32_t Uw[BP], Dw[BP], Eg[BP];
        load_planes<BP>(H, oth + it * BP);
        load_planes<BP>(Uw, oth + (ku * segs + j) * BP);
        load_planes<BP>(Dw, oth + (kd * segs + j) * BP);
        load_planes<BP>(Eg, oth + (k * segs + je) * BP);
        const uint32_t ru = k == 0 ? 8u : 0u, rd = k == band_rows - 1 ? 8u : 0u;
#pragma unroll
        for (int p = 0; p < B; ++p) {
            U[p] = __funnelshift_l(Uw[p], Uw[p], ru);
            D[p] = __funnelshift_r(Dw[p], Dw[p], rd);
            // column m + 1 (par = 1) or m - 1 (par = 0) within each 8-column
            // byte, the edge column from the adjacent segment Eg
            X[p] = par ? (((H[p] >> 1) & 0x7F7F7F7Fu) | ((Eg[p] << 7) & 0x80808080u))
                       : (((H[p] << 1) & 0xFEFEFEFEu) | ((Eg[p] >> 7) & 0x01010101u));
        }
        return 0xFFFFFFFFu;
    } else if constexpr (MODE == 3) {
        const int wu = it == 0 ? IPC - 1 : it - 1;
        const int wd = it == IPC - 1 ? 0 : it + 1;
        uint32_t Hu[BP], Hd[BP];
        load_planes<BP>(H, oth + it * BP);
        load_planes<BP>(Hu, oth + wu * BP);
        load_planes<BP>(Hd, oth + wd * BP);
        auto body = [&](auto S_tag) {
            constexpr int S = decltype(S_tag)::value;
            const uint32_t seg = c ? ~odd_segments<S>() : odd_segments<S>();
#pragma unroll
            for (int p = 0; p < B; ++p) {
                U[p] = (H[p] << S) | (Hu[p] >> (32 - S));
                D[p] = (H[p] >> S) | (Hd[p] << (32 - S));
                X[p] = shifted_packed<S>(H[p], seg);
            }
        };
        if (L == 8) body(std::integral_constant<int, 4>{});
        else if (L == 16) body(std::integral_constant<int, 8>{});
        else body(std::integral_constant<int, 16>{});
        return 0xFFFFFFFFu;
    } else {
        const int y = MODE == 0 ? it : div_by(it, inv_row);
        const int t = MODE == 0 ? 0 : it - y * WPR;
        const int yu = (y == 0) ? L - 1 : y - 1;
        const int yd = (y == L - 1) ? 0 : y + 1;
        const int par = (y + c) & 1;
        load_planes<BP>(U, oth + (yu * WPR + t) * BP);
        load_planes<BP>(D, oth + (yd * WPR + t) * BP);
        load_planes<BP>(H, oth + (y * WPR + t) * BP);
        if constexpr (MODE == 0) {
#pragma unroll
            for (int p = 0; p < B; ++p) X[p] = shifted_row<0>(H[p], 0u, par, 32, 32);
            return 0xFFFFFFFFu;
        } else {
            const int te = par ? (t + 1 == WPR ? 0 : t + 1) : (t == 0 ? WPR - 1 : t - 1);
            uint32_t Eg[BP];
            load_planes<BP>(Eg, oth + (y * WPR + te) * BP);
            const int nb = t == WPR - 1 ? nb_last : 32;
            const int nbe = te == WPR - 1 ? nb_last : 32;
#pragma unroll
            for (int p = 0; p < B; ++p) X[p] = shifted_row<MODE>(H[p], Eg[p], par, nb, nbe);
            return valid_mask(t, WPR, nb_last);
        }
    }
}

// Block-wide sum of ints; every thread receives it.  All threads must call.
__device__ __forceinline__ int block_sum_int(int v)
{
    __shared__ int s_red[33];
    v = __reduce_add_sync(0xFFFFFFFFu, v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int x = lane < (int)(blockDim.x >> 5) ? s_red[lane] : 0;
        x = __reduce_add_sync(0xFFFFFFFFu, x);
        if (lane == 0) s_red[32] = x;
    }
    __syncthreads();
    const int r = s_red[32];
    __syncthreads();
    return r;
}

// ===========================================================================
// One group of resident replicas
// ===========================================================================
struct Group {
    const uint32_t *in;      // buffer holding the parents (or the replicas themselves)
    uint32_t *out;           // buffer receiving the swept replicas
    const int32_t *parent;   // parent map of a pending resample (used when gather)
    const int32_t *anc_in;   // family ids (null: no families)
    int32_t *anc_out;
    int32_t *fam;            // family counts (null: no families)
    int32_t *E, *Mt, *hist;  // per-replica energies and occupations, energy histogram
    int first, nrep;         // slots [first, first + nrep): global slots (random keys); the
                             // arrays above are indexed by them
    int q, theta, step;
    uint32_t stream_hi;      // stream number << 24, or'ed into the slot counter word
    bool gather, write_back;
#if PA_CHECKED
    int src_limit;           // a gather's parent slots lie in [0, src_limit)
    int32_t *err;            // the run's error flag
#endif
};

__device__ __forceinline__ void record_replica(const Group &G, int slot, int E, int Mt, int N, long long &sE,
                                               long long &sE2, long long &sM)
{
    G.E[slot] = E;
    G.Mt[slot] = Mt;
#if PA_CHECKED
    if (E < -2 * N || E > 0) {
        atomicExch(G.err, 1);  // PA_ERR_INVALID
        return;
    }
#endif
    atomicAdd(G.hist + (E + 2 * N), 1);
    sE += E;
    sE2 += (long long)E * (long long)E;
    sM += Mt;
}

__device__ __forceinline__ void group_families(const Group &G)
{
    if (!G.fam) return;
    for (int r = threadIdx.x; r < G.nrep; r += blockDim.x) {
        const int slot = G.first + r;
        const int f = G.anc_in[G.gather ? G.parent[slot] : slot];
        if (G.gather) G.anc_out[slot] = f;
        atomicAdd(G.fam + f, 1);
    }
}

// Shared-memory table of the acceptance thresholds for the bitwise
// comparison v < T[dE]: entry j (0..31) holds, for d = 1..4, all ones where
// bit 31 - j of T[d] is set; entries 32..39 are zero (planes past the last bit
// of v, which the loop may draw when it takes acceptance words four at a time:
// a zero threshold bit never accepts); entry 40 marks T[d] = 2^32.  The
// block's threads share the 41 entries (blocks may have as few as 32 threads).
constexpr int kThresholdEntries = 41;
constexpr int kThresholdFull = 40;

// Two-pass acceptance.  In the first pass every site word draws at most
// kFirstPassCalls Philox calls of acceptance words (the warp stops early when
// all its sites are decided); a word with sites still undecided after that
// (about 8 % of words at low temperature) goes to a block-wide queue, and in
// the second pass whole warps serve only queued words, so a warp no longer
// waits for the slowest of its ~700 sites.  Queue layout in shared memory:
// two counters, QCAP entries of (site-word index, outcome bits acc,
// undecided, class bits c0, e1, B proposal planes).  A full queue is not an error: the
// word's own thread finishes it.  The single-run kernel with up to four planes
// takes 384 entries (its 48 lattices give up to ~250 queued words at low
// temperature, so 256 entries overflowed: 1846 against 1837 attempts/ns over
// the at-scale schedule; two blocks per SM still fit); the batched kernel
// keeps 256, whose 96 KB lattice budget two blocks per SM would not fit with more.
constexpr int kFirstPassCalls = 2;
constexpr int kQueueCap = 256;
__host__ __device__ constexpr int queue_words(int B, int cap = kQueueCap) { return 2 + (5 + B) * cap; }
// Entry j holds, for the threshold bits t_1..t_4 of plane j (bit 31 - j of
// T[1..4]), the coefficients of two multiply-adds: c0 * (t_1 - t_2) - t_2
// gives the threshold bits of the dE = 1, 2 sites (c0: dE odd) and
// c0 * (t_3 - t_4) - t_4 those of the dE = 3, 4 sites, bit for bit: the four
// results 0, c0, ~c0 = -c0 - 1 and ~0 are the four two-way selections.  The
// selections thus run on the multiply-add pipe; only the choice by e1 is a
// logic operation.
__device__ __forceinline__ void build_threshold_table(uint4 *tab, const Thresholds &th)
{
    auto coef = [](uint32_t ta, uint32_t tb) { return make_uint2(ta - tb, 0u - tb); };
    for (int j = threadIdx.x; j < kThresholdEntries; j += blockDim.x) {
        uint32_t t[4] = {0u, 0u, 0u, 0u};
        if (j < 32) {
            for (int d = 0; d < 4; ++d) t[d] = (th.T[d] >> (31 - j)) & 1u;
        } else if (j == kThresholdFull) {
            for (int d = 0; d < 4; ++d) t[d] = (th.full >> d) & 1u;
        }
        const uint2 lo = coef(t[0], t[1]), hi = coef(t[2], t[3]);
        tab[j] = make_uint4(lo.x, lo.y, hi.x, hi.y);
    }
}

// Threshold bit of plane entry tb for each site: the site's dE class is
// given by c0 (dE odd) and e1 (dE >= 3).
__device__ __forceinline__ uint32_t threshold_bits(const uint4 &tb, uint32_t c0, uint32_t e1)
{
    const uint32_t lo = c0 * tb.x + tb.y;  // dE = 1 where c0, dE = 2 elsewhere
    const uint32_t hi = c0 * tb.z + tb.w;  // dE = 3 where c0, dE = 4 elsewhere
    return (e1 & hi) | (~e1 & lo);
}

// One bit plane j of the acceptance numbers v (bits of the word v_bits).  A
// site still undecided takes T's bit into acc -- the outcome of v < T if v's
// bit differs from it -- and stays undecided where the two bits agree.  So
// once the planes are done a site is accepted where acc is set and und is
// clear (a site whose v equals T in every plane is rejected).
__device__ __forceinline__ void acceptance_plane(uint32_t v_bits, int j, const uint4 *s_tab, uint32_t c0, uint32_t e1,
                                                 uint32_t &acc, uint32_t &und)
{
    const uint32_t tj = threshold_bits(s_tab[j], c0, e1);
    acc = (und & tj) | (~und & acc);
    und &= ~(v_bits ^ tj);
}

// Acceptance words of Philox calls n = ch_begin .. ch_end - 1 of a site word's
// stream (words 4n .. 4n + 3, i.e. planes j = 4n - B ..), drawn while a site is
// undecided: in the whole warp (WARP_VOTE, all lanes must take part) or in this
// thread's word alone.
template <int B, bool WARP_VOTE>
__device__ __forceinline__ void acceptance_calls(int ch_begin, int ch_end, uint32_t w, uint32_t ctr1, uint32_t step,
                                                 uint32_t slot, const uint32_t *rk0, const uint32_t *rk1,
                                                 const uint4 *s_tab, uint32_t c0, uint32_t e1, uint32_t &acc,
                                                 uint32_t &und)
{
#pragma unroll 1
    for (int ch = ch_begin; ch < ch_end; ++ch) {
        if (WARP_VOTE ? !__any_sync(0xFFFFFFFFu, und) : !und) break;
        const uint4 z = philox10_rk(make_uint4(w, ctr1 | (uint32_t)ch, step, slot), rk0, rk1);
        const int j0 = 4 * ch - B;
        acceptance_plane(z.x, j0, s_tab, c0, e1, acc, und);
        acceptance_plane(z.y, j0 + 1, s_tab, c0, e1, acc, und);
        acceptance_plane(z.z, j0 + 2, s_tab, c0, e1, acc, und);
        acceptance_plane(z.w, j0 + 3, s_tab, c0, e1, acc, und);
    }
}

// Multi-spin-coded sweep body.  B = bits per state (compile time), MODE as
// for neighbour_planes, Q = q when fixed at compile time (0: q from G).  Each loop step of a thread updates one site word: 32
// same-colour sites of one row.  The random numbers follow this rule: in
// sweep k, colour c, the site word with index w = y WPR + t draws the stream
// Z_0, Z_1, ... (Z_{4n+i} = word i of the Philox call with counter
// (w, SWEEP | (2k + c) << 8 | n, step, slot | stream)); the site at bit b takes
// bit b of each: direction sigma from Z_0, offset u from Z_1..Z_{B-1}, and
// acceptance bits v_j from Z_{B+j}, most significant first.  Proposal
// s' = s + (1 + u) mod q (sigma = 0) or s - (1 + u) mod q (sigma = 1) by two
// ripple-carry additions over the planes; dE + 4 is the count of eight
// indicator bits (neighbours equal to s, neighbours different from s'), summed
// by a carry-save tree; moves with dE > 0 compare v with T[dE] bit by bit, and
// the warp draws further acceptance words only while some site is undecided.
template <int B, int MODE, int Q = 0, bool HOIST = false, int QCAP = kQueueCap, bool SPLIT = false>
__device__ __forceinline__ void sweep_group_bits(const Group &G, int Lrt, uint32_t *sw, const uint4 *s_tab,
                                                 uint32_t *qbuf, const uint32_t *rk0, const uint32_t *rk1,
                                                 long long &sE, long long &sE2, long long &sM)
{
    constexpr int BP = plane_stride(B);
    // the measurement's per-replica counts reuse the queue (at most 16 replicas x (q + 1))
    static_assert(16 * ((1 << B) + 1) <= queue_words(B, QCAP), "queue too small for the counts");
    const int L = MODE == 0 ? 64 : Lrt;
    const int N = L * L;
    const int WPR = MODE == 0 ? 1 : row_words(L);
    const int nb_last = L / 2 - 32 * (WPR - 1);
    const int IPC = colour_words(L);  // site words per colour per replica
    const int RW = replica_words_of(B, L);  // words per replica
    const int UPR = RW / 4;       // uint4 per replica
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    const int q = Q > 0 ? Q : G.q;  // Q > 0: q fixed at compile time, the mod-q masks fold
    const int first = G.first, nrep = G.nrep;
    uint4 *smem4 = reinterpret_cast<uint4 *>(sw);

    // gather: replica first + r comes from its parent's lattice
    for (int i = tid; i < nrep * UPR; i += blockDim.x) {
        const int r = i / UPR;
        const int o = i - r * UPR;
        const int slot = first + r;
#if PA_CHECKED
        int src = G.gather ? G.parent[slot] : slot;
        if (G.gather && (src < 0 || src >= G.src_limit)) {
            atomicExch(G.err, 1);  // PA_ERR_INVALID
            src = 0;
        }
#else
        const int src = G.gather ? G.parent[slot] : slot;
#endif
        smem4[r * UPR + o] = reinterpret_cast<const uint4 *>(G.in + (size_t)src * RW)[o];
    }
    __syncthreads();

    // q and 2^(B+1) - q as plane masks, for the reduction mod q
    uint32_t qm[B + 1], nqm[B + 1];
#pragma unroll
    for (int p = 0; p <= B; ++p) {
        qm[p] = ((q >> p) & 1) ? 0xFFFFFFFFu : 0u;
        nqm[p] = ((((1 << (B + 1)) - q) >> p) & 1) ? 0xFFFFFFFFu : 0u;
    }
    const bool any_full = s_tab[kThresholdFull].x | s_tab[kThresholdFull].y | s_tab[kThresholdFull].z |
                          s_tab[kThresholdFull].w;
    const int total = nrep * IPC;

    // site words still undecided after the first pass wait in qbuf for the second
    int *q_count = reinterpret_cast<int *>(qbuf);
    int *q_item = q_count + 2;
    uint32_t(*q_mask)[QCAP] = reinterpret_cast<uint32_t(*)[QCAP]>(qbuf + 2 + QCAP);  // acc, und, c0, e1
    uint32_t(*q_prop)[QCAP] = reinterpret_cast<uint32_t(*)[QCAP]>(qbuf + 2 + 5 * QCAP);
    if (tid < 2) q_count[tid] = 0;
    __syncthreads();
    int half = 0;
    // HOIST: when each pass of the block's threads covers whole replicas and
    // a warp stays within one replica (IPC a multiple of 32 dividing the
    // threads), a thread keeps one site word index through all passes: its
    // row, neighbour offsets and counter word are computed once instead of per
    // word.  (The batched kernel, one function over every body, leaves it out:
    // a second copy of each first pass doubles its size and build time.)
    const bool whole_passes = HOIST && IPC % 32 == 0 && (nwarps * 32) % IPC == 0;
    const int it_fixed = (warp * 32 + lane) % IPC;
    const int r_first = (warp * 32) / IPC;
    const int r_step = (nwarps * 32) / IPC;
    // replica of a block-wide word index, and row (segment row) of a word
    const uint32_t inv_ipc = div_inverse(IPC);
    const uint32_t inv_row = div_inverse(MODE == 4 ? L >> 4 : WPR);
    auto replica_of = [&](int x) { return MODE == 0 ? x / IPC : div_by(x, inv_ipc); };

    for (int k = 0; k < G.theta; ++k) {
        for (int c = 0; c < 2; ++c, ++half) {
            const uint32_t ctr1 = DOM_SWEEP | ((uint32_t)(2 * k + c) << 8);
            if (tid == 0) q_count[(half + 1) & 1] = 0;
            int *qc = q_count + (half & 1);
            // one site word: replica r, word it within the colour (its counter
            // word w); lanes that are not live run along for the warp votes
            auto site_word = [&](const int r, const int it, const bool live) {
                const int ii = r * IPC + it;
                uint32_t *rep = sw + r * RW;
                uint32_t *own = rep + (c * IPC + it) * BP;
                const uint32_t *oth = rep + (c ^ 1) * IPC * BP;
                uint32_t W[BP], U[BP], D[BP], H[BP], X[BP];
                load_planes<BP>(W, own);
                const uint32_t vmask =
                    neighbour_planes<B, MODE, BP>(oth, L, IPC, WPR, nb_last, inv_row, it, c, U, D, H, X);

                // proposal: direction sigma = Z_0, offset bits u = Z_1..Z_{B-1}
                const uint32_t slot = (uint32_t)(first + r) | G.stream_hi;
                const uint32_t w = (uint32_t)it;
                uint32_t Z[8];
                {
                    const uint4 z = philox10_rk(make_uint4(w, ctr1, (uint32_t)G.step, slot), rk0, rk1);
                    Z[0] = z.x;
                    Z[1] = z.y;
                    Z[2] = z.z;
                    Z[3] = z.w;
                }
                if constexpr (B > 4) {
                    const uint4 z = philox10_rk(make_uint4(w, ctr1 | 1u, (uint32_t)G.step, slot), rk0, rk1);
                    Z[4] = z.x;
                    Z[5] = z.y;
                    Z[6] = z.z;
                    Z[7] = z.w;
                }
                const uint32_t sg = Z[0];
                // S = s + 1 + u (sigma = 0) or s - 1 - u (sigma = 1), B + 1 bits
                uint32_t S[B + 1];
                uint32_t cy = ~sg;
#pragma unroll
                for (int p = 0; p < B; ++p) {
                    const uint32_t x = (p < B - 1) ? (Z[p + 1] ^ sg) : sg;
                    full_add(W[p], x, cy, S[p], cy);
                }
                S[B] = sg ^ cy;
                // Tq = S - q (sigma = 0) or S + q (sigma = 1); take Tq where S >= q
                // (sigma = 0) or S < 0 (sigma = 1)
                uint32_t Tq[B + 1];
                uint32_t cz = 0;
#pragma unroll
                for (int p = 0; p <= B; ++p) {
                    const uint32_t yb = (sg & qm[p]) | (~sg & nqm[p]);
                    full_add(S[p], yb, cz, Tq[p], cz);
                }
                const uint32_t take = (sg & S[B]) | (~sg & ~Tq[B]);
                uint32_t P[BP];
#pragma unroll
                for (int p = 0; p < BP; ++p) P[p] = p < B ? ((take & Tq[p]) | (~take & S[p])) : 0u;

                // dE + 4 = #(neighbours equal to s) + #(neighbours different from s')
                const uint32_t a1 = ~differ<B, BP>(W, U), a2 = ~differ<B, BP>(W, D);
                const uint32_t a3 = ~differ<B, BP>(W, H), a4 = ~differ<B, BP>(W, X);
                const uint32_t b1 = differ<B, BP>(P, U), b2 = differ<B, BP>(P, D);
                const uint32_t b3 = differ<B, BP>(P, H), b4 = differ<B, BP>(P, X);
                uint32_t s1, k1, s2, k2, s3, k3, s5, k5;
                full_add(a1, a2, a3, s1, k1);
                full_add(a4, b1, b2, s2, k2);
                full_add(b3, b4, s1, s3, k3);
                const uint32_t c0 = s2 ^ s3, k4 = s2 & s3;
                full_add(k1, k2, k3, s5, k5);
                const uint32_t c1 = s5 ^ k4, k6 = s5 & k4;
                const uint32_t c2 = k5 ^ k6, c3 = k5 & k6;
                const uint32_t pos = vmask & (c3 | (c2 & (c1 | c0)));  // dE > 0
                const uint32_t e1 = c3 | (c1 & c0);                     // dE >= 3

                // acceptance: dE <= 0 always; otherwise v < T[dE], bit by bit
                uint32_t acc = live ? (vmask & ~pos) : 0u;
                uint32_t und = live ? pos : 0u;
                if (any_full) {
                    const uint32_t tj = threshold_bits(s_tab[kThresholdFull], c0, e1);
                    acc |= und & tj;
                    und &= ~tj;
                }
                // acceptance bit j is word B + j: the rest of the last proposal call first
                if constexpr (B % 4 != 0) {
                    if (__any_sync(0xFFFFFFFFu, und)) {
#pragma unroll
                        for (int wi = B; wi < 4 * ((B + 3) / 4); ++wi)
                            acceptance_plane(Z[wi], wi - B, s_tab, c0, e1, acc, und);
                    }
                }
                constexpr int fc = (B + 3) / 4;
                acceptance_calls<B, true>(fc, fc + kFirstPassCalls, w, ctr1, (uint32_t)G.step, slot, rk0, rk1, s_tab,
                                          c0, e1, acc, und);
                bool queued = false;
                if (und) {
                    const int e = atomicAdd(qc, 1);
                    if (e < QCAP) {
                        q_item[e] = ii;
                        q_mask[0][e] = acc;
                        q_mask[1][e] = und;
                        q_mask[2][e] = c0;
                        q_mask[3][e] = e1;
#pragma unroll
                        for (int p = 0; p < B; ++p) q_prop[p][e] = P[p];
                        queued = true;
                    } else {
                        // queue full: this thread finishes its word alone (no warp votes)
                        acceptance_calls<B, false>(fc + kFirstPassCalls, fc + 8, w, ctr1, (uint32_t)G.step, slot, rk0,
                                                   rk1, s_tab, c0, e1, acc, und);
                    }
                }
                if (live && !queued) {
                    const uint32_t a = acc & ~und;
#pragma unroll
                    for (int p = 0; p < B; ++p) W[p] = (a & P[p]) | (~a & W[p]);
                    store_planes<BP>(own, W);
                }
            };
            if (HOIST && whole_passes) {
                for (int r = r_first; r < nrep; r += r_step) site_word(r, it_fixed, true);
            } else {
                for (int base = warp * 32; base < total; base += nwarps * 32) {
                    const int i = base + lane;
                    const bool live = i < total;
                    const int ii = live ? i : total - 1;
                    const int r = replica_of(ii);
                    site_word(r, ii - r * IPC, live);
                }
            }
            __syncthreads();
            // second pass: the queued site words, 32 to a warp
            const int nq = min(*qc, QCAP);
            for (int base = warp * 32; base < nq; base += nwarps * 32) {
                const int e = base + lane;
                const bool live = e < nq;
                const int ee = live ? e : nq - 1;
                const int ii = q_item[ee];
                const int r = replica_of(ii);
                const int it = ii - r * IPC;
                uint32_t acc = q_mask[0][ee];
                uint32_t und = live ? q_mask[1][ee] : 0u;
                const uint32_t c0 = q_mask[2][ee], e1 = q_mask[3][ee];
                const uint32_t slot = (uint32_t)(first + r) | G.stream_hi;
                const uint32_t w = (uint32_t)it;
                constexpr int fc = (B + 3) / 4;
                acceptance_calls<B, true>(fc + kFirstPassCalls, fc + 8, w, ctr1, (uint32_t)G.step, slot, rk0, rk1,
                                          s_tab, c0, e1, acc, und);
                if (live) {
                    uint32_t *own = sw + r * RW + (c * IPC + it) * BP;
                    uint32_t W[BP];
                    load_planes<BP>(W, own);
                    const uint32_t a = acc & ~und;
#pragma unroll
                    for (int p = 0; p < B; ++p) W[p] = (a & q_prop[p][ee]) | (~a & W[p]);
                    store_planes<BP>(own, W);
                }
            }
            __syncthreads();
        }
    }

    if (SPLIT && 2 * nrep <= nwarps) {
        // measurements of a block holding fewer replicas than twice its warps
        // (SPLIT: the single-run kernel, whose blocks may hold a few large
        // lattices): every warp takes a share of each replica's words and the
        // warps' counts are summed in shared memory (the queue's, idle now),
        // with one barrier for the group instead of three per count
        // (nrep <= nwarps / 2 <= 16 replicas x (q + 1) counts fit the queue)
        int *s_cnt = reinterpret_cast<int *>(qbuf);
        for (int i = tid; i < nrep * (q + 1); i += blockDim.x) s_cnt[i] = 0;
        __syncthreads();
        for (int r = 0; r < nrep; ++r) {
            const uint32_t *rep = sw + r * RW;
            int *cnt_r = s_cnt + r * (q + 1);
            int agree = 0;
            // each bond has one colour-0 end: count equal neighbours of colour-0 sites
            for (int it = tid; it < IPC; it += blockDim.x) {
                uint32_t W[BP], U[BP], D[BP], H[BP], X[BP];
                load_planes<BP>(W, rep + it * BP);
                const uint32_t vmask =
                    neighbour_planes<B, MODE, BP>(rep + IPC * BP, L, IPC, WPR, nb_last, inv_row, it, 0, U, D, H, X);
                agree += __popc(vmask & ~differ<B, BP>(W, U)) + __popc(vmask & ~differ<B, BP>(W, D)) +
                         __popc(vmask & ~differ<B, BP>(W, H)) + __popc(vmask & ~differ<B, BP>(W, X));
            }
            agree = __reduce_add_sync(0xFFFFFFFFu, agree);
            if (lane == 0 && agree) atomicAdd(cnt_r + q, agree);
            for (int s = 0; s < q; ++s) {
                int cnt = 0;
                for (int it = tid; it < 2 * IPC; it += blockDim.x) {
                    uint32_t W[BP];
                    load_planes<BP>(W, rep + it * BP);
                    const uint32_t vmask =
                        (MODE == 0 || MODE == 3 || MODE == 4)
                            ? 0xFFFFFFFFu
                            : valid_mask(it - div_by(it, inv_row) * WPR, WPR, nb_last);
                    cnt += __popc(vmask & equal_state<B, BP>(W, s));
                }
                cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
                if (lane == 0 && cnt) atomicAdd(cnt_r + s, cnt);
            }
        }
        __syncthreads();
        // lane 0 of warp r records replica r (lane 0 of each warp carries the sums)
        if (lane == 0 && warp < nrep) {
            const int *cnt_r = s_cnt + warp * (q + 1);
            int best = 0;
            for (int s = 0; s < q; ++s) best = max(best, cnt_r[s]);
            record_replica(G, first + warp, -cnt_r[q], best, N, sE, sE2, sM);
        }
    } else {
        // measurements: one warp per replica, or the whole block per replica when
        // the block holds fewer replicas than warps
        const bool per_warp = 2 * nrep > nwarps;
        const int n_owner = per_warp ? nwarps : 1;
        const int owner = per_warp ? warp : 0;
        const int stride = per_warp ? 32 : (int)blockDim.x;
        const int me = per_warp ? lane : tid;
        for (int r0 = 0; r0 < nrep; r0 += n_owner) {
            const int r = r0 + owner;
            const bool have = r < nrep;
            const uint32_t *rep = sw + (have ? r : 0) * RW;
            int agree = 0;
            if (have) {
                // each bond has one colour-0 end: count equal neighbours of colour-0 sites
                for (int it = me; it < IPC; it += stride) {
                    uint32_t W[BP], U[BP], D[BP], H[BP], X[BP];
                    load_planes<BP>(W, rep + it * BP);
                    const uint32_t vmask = neighbour_planes<B, MODE, BP>(rep + IPC * BP, L, IPC, WPR, nb_last,
                                                                         inv_row, it, 0, U, D, H, X);
                    agree += __popc(vmask & ~differ<B, BP>(W, U)) + __popc(vmask & ~differ<B, BP>(W, D)) +
                             __popc(vmask & ~differ<B, BP>(W, H)) + __popc(vmask & ~differ<B, BP>(W, X));
                }
            }
            agree = per_warp ? __reduce_add_sync(0xFFFFFFFFu, agree) : block_sum_int(agree);
            int best = 0;
            for (int s = 0; s < q; ++s) {
                int cnt = 0;
                if (have) {
                    for (int it = me; it < 2 * IPC; it += stride) {
                        uint32_t W[BP];
                        load_planes<BP>(W, rep + it * BP);
                        const uint32_t vmask =
                            (MODE == 0 || MODE == 3 || MODE == 4)
                                ? 0xFFFFFFFFu
                                : valid_mask(it - div_by(it, inv_row) * WPR, WPR, nb_last);
                        cnt += __popc(vmask & equal_state<B, BP>(W, s));
                    }
                }
                cnt = per_warp ? __reduce_add_sync(0xFFFFFFFFu, cnt) : block_sum_int(cnt);
                best = max(best, cnt);
            }
            if (have && me == 0) record_replica(G, first + r, -agree, best, N, sE, sE2, sM);
        }
    }
    group_families(G);
    __syncthreads();
    if (G.write_back) {
        for (int i = tid; i < nrep * UPR; i += blockDim.x) {
            const int r = i / UPR;
            const int o = i - r * UPR;
            reinterpret_cast<uint4 *>(G.out + (size_t)(first + r) * RW)[o] = smem4[r * UPR + o];
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void accumulate_totals(unsigned long long *acc, long long sE, long long sE2, long long sM)
{
    atomicAdd(acc + 0, (unsigned long long)sE);
    atomicAdd(acc + 1, (unsigned long long)sE2);
    atomicAdd(acc + 2, (unsigned long long)sM);
}

}  // namespace dev
}  // namespace pa
