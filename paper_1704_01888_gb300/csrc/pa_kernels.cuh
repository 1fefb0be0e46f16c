// pa_kernels.cuh -- device bodies of the population-annealing kernels
// (Barash, Weigel, Shchur & Janke, arXiv:1704.01888), shared by the
// single-run kernels (pa_sweep.cu, pa_resample.cu) and the batched kernels
// (pa_batch.cu) so that both run the same arithmetic.
//
// Sweep bodies: one block holds a group of whole lattices in shared memory
// (the gather of Sec. 2 step 2 fused into the load), runs theta
// checkerboard Metropolis sweeps (Sec. 2 step 3) and measures each replica's
// energy (Eq. 3), largest-state occupation (Eq. 5) and the energy histogram.
// Spins are multi-spin coded (layout in pa_internal.cuh): every logic
// instruction of the update acts on the 32 sites of one site word.
// Resampling bodies (Sec. 2 step 2, Eq. 2): weights and ln Q, copy numbers and
// their scan, parent map; estimators (Sec. 2 step 4, Eqs. 4-5).
#pragma once
#include <climits>
#include <type_traits>

#include "pa_internal.cuh"

namespace pa {
namespace dev {

// ===========================================================================
// Bit-plane helpers
// ===========================================================================

// BP consecutive words (the planes of one site word) with one vector access.
template <int BP>
__device__ __forceinline__ void load_planes(uint32_t (&v)[BP], const uint32_t *src)
{
    if constexpr (BP == 1) {
        v[0] = src[0];
    } else if constexpr (BP == 2) {
        const uint2 a = *reinterpret_cast<const uint2 *>(src);
        v[0] = a.x;
        v[1] = a.y;
    } else {
#pragma unroll
        for (int h = 0; h < BP / 4; ++h) {
            const uint4 a = reinterpret_cast<const uint4 *>(src)[h];
            v[4 * h + 0] = a.x;
            v[4 * h + 1] = a.y;
            v[4 * h + 2] = a.z;
            v[4 * h + 3] = a.w;
        }
    }
}

template <int BP>
__device__ __forceinline__ void store_planes(uint32_t *dst, const uint32_t (&v)[BP])
{
    if constexpr (BP == 1) {
        dst[0] = v[0];
    } else if constexpr (BP == 2) {
        *reinterpret_cast<uint2 *>(dst) = make_uint2(v[0], v[1]);
    } else {
#pragma unroll
        for (int h = 0; h < BP / 4; ++h)
            reinterpret_cast<uint4 *>(dst)[h] = make_uint4(v[4 * h], v[4 * h + 1], v[4 * h + 2], v[4 * h + 3]);
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
};

__device__ __forceinline__ void record_replica(const Group &G, int slot, int E, int Mt, int N, long long &sE,
                                               long long &sE2, long long &sM)
{
    G.E[slot] = E;
    G.Mt[slot] = Mt;
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
// two counters, kQueueCap entries of (site-word index, outcome bits acc,
// undecided, class bits c0, e1, B proposal planes).  A full queue is not an error: the
// word's own thread finishes it.
constexpr int kFirstPassCalls = 2;
constexpr int kQueueCap = 256;
__host__ __device__ constexpr int queue_words(int B) { return 2 + (5 + B) * kQueueCap; }
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
template <int B, int MODE, int Q = 0, bool HOIST = false>
__device__ __forceinline__ void sweep_group_bits(const Group &G, int Lrt, uint32_t *sw, const uint4 *s_tab,
                                                 uint32_t *qbuf, const uint32_t *rk0, const uint32_t *rk1,
                                                 long long &sE, long long &sE2, long long &sM)
{
    constexpr int BP = plane_stride(B);
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
        const int src = G.gather ? G.parent[slot] : slot;
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
    uint32_t(*q_mask)[kQueueCap] = reinterpret_cast<uint32_t(*)[kQueueCap]>(qbuf + 2 + kQueueCap);  // acc, und, c0, e1
    uint32_t(*q_prop)[kQueueCap] = reinterpret_cast<uint32_t(*)[kQueueCap]>(qbuf + 2 + 5 * kQueueCap);
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
                    if (e < kQueueCap) {
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
            const int nq = min(*qc, kQueueCap);
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
                const uint32_t vmask =
                    neighbour_planes<B, MODE, BP>(rep + IPC * BP, L, IPC, WPR, nb_last, inv_row, it, 0, U, D, H, X);
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
