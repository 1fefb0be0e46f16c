// pa_kernels.cuh -- device bodies of the population-annealing kernels
// (Barash, Weigel, Shchur & Janke, arXiv:1704.01888), shared by the
// single-run kernels (pa_sweep.cu, pa_resample.cu) and the batched kernels
// (pa_batch.cu) so that both run the same arithmetic.
//
// Sweep bodies: one block holds a group of whole lattices in shared memory
// (the gather of Sec. 2 step 2 fused into the load), runs theta
// checkerboard Metropolis sweeps (Sec. 2 step 3) and measures each replica's
// energy (Eq. 3), largest-state occupation (Eq. 5) and the energy histogram.
// Resampling bodies (Sec. 2 step 2, Eq. 2): weights and ln Q, copy numbers and
// their scan, parent map; estimators (Sec. 2 step 4, Eqs. 4-5).
#pragma once
#include <climits>

#include "pa_internal.cuh"

namespace pa {
namespace dev {

// ===========================================================================
// SWAR helpers (four spins per 32-bit word, all values < 128)
// ===========================================================================

// Bit 7 of each byte is set where the bytes of a and b differ.
__device__ __forceinline__ uint32_t differ_bits(uint32_t a, uint32_t b)
{
    return ((a ^ b) + 0x7F7F7F7Fu) & 0x80808080u;
}

// Per byte: how many of the four neighbour words differ from a (0..4).
__device__ __forceinline__ uint32_t count_differ(uint32_t a, uint32_t n0, uint32_t n1, uint32_t n2, uint32_t n3)
{
    return (differ_bits(a, n0) >> 7) + (differ_bits(a, n1) >> 7) + (differ_bits(a, n2) >> 7) +
           (differ_bits(a, n3) >> 7);
}

struct Neighbours {
    uint32_t up, down, same, shifted;
};

// Neighbour words of word t in row y of a colour whose row offset is p =
// (y + colour) & 1.  `oth` is the other colour's sublattice of the replica.
__device__ __forceinline__ Neighbours load_neighbours(const uint32_t *oth, int L, int L8, int y, int t, int p)
{
    Neighbours nb;
    const int yu = (y == 0) ? L - 1 : y - 1;
    const int yd = (y == L - 1) ? 0 : y + 1;
    const int row = y * L8;
    nb.up = oth[yu * L8 + t];
    nb.down = oth[yd * L8 + t];
    nb.same = oth[row + t];
    if (p == 0) {
        const int tl = (t == 0) ? L8 - 1 : t - 1;
        nb.shifted = __funnelshift_l(oth[row + tl], nb.same, 8);  // bytes m-1
    } else {
        const int tr = (t == L8 - 1) ? 0 : t + 1;
        nb.shifted = __funnelshift_r(nb.same, oth[row + tr], 8);  // bytes m+1
    }
    return nb;
}

template <int S>
struct Vec;
template <>
struct Vec<1> {
    uint32_t v[1];
    __device__ __forceinline__ void load(const uint32_t *p) { v[0] = p[0]; }
    __device__ __forceinline__ void store(uint32_t *p) const { p[0] = v[0]; }
};
template <>
struct Vec<2> {
    uint32_t v[2];
    __device__ __forceinline__ void load(const uint32_t *p)
    {
        const uint2 x = *reinterpret_cast<const uint2 *>(p);
        v[0] = x.x;
        v[1] = x.y;
    }
    __device__ __forceinline__ void store(uint32_t *p) const { *reinterpret_cast<uint2 *>(p) = make_uint2(v[0], v[1]); }
};
template <>
struct Vec<4> {
    uint32_t v[4];
    __device__ __forceinline__ void load(const uint32_t *p)
    {
        const uint4 x = *reinterpret_cast<const uint4 *>(p);
        v[0] = x.x;
        v[1] = x.y;
        v[2] = x.z;
        v[3] = x.w;
    }
    __device__ __forceinline__ void store(uint32_t *p) const
    {
        *reinterpret_cast<uint4 *>(p) = make_uint4(v[0], v[1], v[2], v[3]);
    }
};

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
    const uint8_t *in;       // buffer holding the parents (or the replicas themselves)
    uint8_t *out;            // buffer receiving the swept replicas
    const int32_t *parent;   // parent map of a pending resample (used when gather)
    const int32_t *anc_in;   // family ids (null: no families)
    int32_t *anc_out;
    int32_t *fam;            // family counts (null: no families)
    int32_t *E, *Mt, *hist;  // per-replica energies and occupations, energy histogram
    int first, nrep;         // slots [first, first + nrep)
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

// Row-segment body (L % 8 == 0).  LT > 0 fixes L at compile time; S is the
// number of 32-bit words (4 same-colour sites each) one thread updates per
// loop step: S consecutive words of one row of one colour, read and written
// with one vector access per neighbour row.  Each site takes one 32-bit
// Philox word u: the high and low halves of u (q - 1) are its proposal offset
// and its acceptance uniform.  s_thr holds T[dE + 4]; rk0 / rk1 the round keys.
template <int LT, int S>
__device__ __forceinline__ void sweep_group_rows(const Group &G, int Lrt, uint4 *smem4, const uint32_t *s_thr,
                                                 const uint32_t *rk0, const uint32_t *rk1, long long &sE,
                                                 long long &sE2, long long &sM)
{
    uint32_t *sw = reinterpret_cast<uint32_t *>(smem4);
    const int L = LT > 0 ? LT : Lrt;
    const int N = L * L;
    const int L8 = L / 8;     // words per row of one colour
    const int WPC = N / 8;    // words per colour per replica
    const int WPR = N / 4;    // words per replica
    const int UPR = N / 16;   // uint4 per replica
    const int SPR = L8 / S;   // segments per row
    const int UPC = L * SPR;  // segments per colour per replica
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    const uint32_t qm1 = (uint32_t)(G.q - 1);
    const uint32_t qb = (uint32_t)G.q;
    const char *thr_bytes = reinterpret_cast<const char *>(s_thr);
    const int first = G.first, nrep = G.nrep;

    // gather: replica first + r comes from its parent's lattice
    for (int i = tid; i < nrep * UPR; i += blockDim.x) {
        const int r = i / UPR;
        const int o = i - r * UPR;
        const int slot = first + r;
        const int src = G.gather ? G.parent[slot] : slot;
        smem4[r * UPR + o] = reinterpret_cast<const uint4 *>(G.in + (size_t)src * N)[o];
    }
    __syncthreads();

    for (int k = 0; k < G.theta; ++k) {
        for (int c = 0; c < 2; ++c) {
            const uint32_t ctr1 = DOM_SWEEP | (uint32_t)(2 * k + c);
            for (int i = tid; i < nrep * UPC; i += blockDim.x) {
                const int r = i / UPC;
                const int u = i - r * UPC;
                const int y = u / SPR;
                const int t0 = (u - y * SPR) * S;
                uint32_t *own = sw + r * WPR + c * WPC;
                const uint32_t *oth = sw + r * WPR + (c ^ 1) * WPC;
                const int p = (y + c) & 1;  // 0: horizontal neighbours at m-1, m; 1: at m, m+1
                const int row = y * L8;
                const int yu = (y == 0) ? L - 1 : y - 1;
                const int yd = (y == L - 1) ? 0 : y + 1;
                Vec<S> W, U, D, H;
                W.load(own + row + t0);
                U.load(oth + yu * L8 + t0);
                D.load(oth + yd * L8 + t0);
                H.load(oth + row + t0);
                const int te = p ? (t0 + S == L8 ? 0 : t0 + S) : (t0 == 0 ? L8 - 1 : t0 - 1);
                const uint32_t edge = oth[row + te];
                const uint32_t sh = p ? 8u : 24u;
                // sublattice index of byte 0 of word t0 is y*L/2 + 4*t0; one Philox
                // call serves the four sites of a word (counter = index / 4)
                const uint32_t quad0 = (uint32_t)(y * (L / 8) + t0);
                const uint32_t slot = (uint32_t)(first + r) | G.stream_hi;
                Vec<S> NW;
#pragma unroll
                for (int j = 0; j < S; ++j) {
                    const uint32_t lo = p ? H.v[j] : (j == 0 ? edge : H.v[j > 0 ? j - 1 : 0]);
                    const uint32_t hi = p ? (j == S - 1 ? edge : H.v[j < S - 1 ? j + 1 : 0]) : H.v[j];
                    const uint32_t shifted = __funnelshift_r(lo, hi, sh);
                    const uint32_t Wj = W.v[j];
                    // one word per site: (high, low) of the 64-bit product u (q-1) are the
                    // proposal offset and the acceptance uniform
                    const uint4 ru = philox10_rk(make_uint4(quad0 + j, ctr1, (uint32_t)G.step, slot), rk0, rk1);
                    const uint64_t px = (uint64_t)ru.x * qm1, py = (uint64_t)ru.y * qm1;
                    const uint64_t pz = (uint64_t)ru.z * qm1, pw = (uint64_t)ru.w * qm1;
                    const uint32_t m = __byte_perm(__byte_perm((uint32_t)(px >> 32), (uint32_t)(py >> 32), 0x0040),
                                                   __byte_perm((uint32_t)(pz >> 32), (uint32_t)(pw >> 32), 0x0040),
                                                   0x5410);
                    // proposals s' = s + 1 + m, reduced mod q bytewise
                    uint32_t P = Wj + m + 0x01010101u;
                    const uint32_t ge = (P + (0x80u - qb) * 0x01010101u) & 0x80808080u;
                    P -= (ge >> 7) * qb;
                    // 4 (dE + 4) per byte: byte offsets into the threshold table
                    const uint32_t dW = count_differ(Wj, U.v[j], D.v[j], H.v[j], shifted);
                    const uint32_t dP = count_differ(P, U.v[j], D.v[j], H.v[j], shifted);
                    const uint32_t idx4 = (dP + 0x04040404u - dW) << 2;
                    const uint32_t T0 = *reinterpret_cast<const uint32_t *>(thr_bytes + __byte_perm(idx4, 0, 0x4440));
                    const uint32_t T1 = *reinterpret_cast<const uint32_t *>(thr_bytes + __byte_perm(idx4, 0, 0x4441));
                    const uint32_t T2 = *reinterpret_cast<const uint32_t *>(thr_bytes + __byte_perm(idx4, 0, 0x4442));
                    const uint32_t T3 = *reinterpret_cast<const uint32_t *>(thr_bytes + __byte_perm(idx4, 0, 0x4443));
                    uint32_t sel = 0x3210u;
                    sel += ((uint32_t)px < T0) ? 0x4u : 0u;
                    sel += ((uint32_t)py < T1) ? 0x40u : 0u;
                    sel += ((uint32_t)pz < T2) ? 0x400u : 0u;
                    sel += ((uint32_t)pw < T3) ? 0x4000u : 0u;
                    NW.v[j] = __byte_perm(Wj, P, sel);
                }
                NW.store(own + row + t0);
            }
            __syncthreads();
        }
    }

    // measurements: one warp per replica, or the whole block per replica when
    // the block holds fewer replicas than warps
    if (2 * nrep > nwarps) {
        for (int r = warp; r < nrep; r += nwarps) {
            const uint32_t *rep = sw + r * WPR;
            int agree = 0;
            for (int w = lane; w < WPC; w += 32) {
                const int y = w / L8;
                const int t = w - y * L8;
                const Neighbours nb = load_neighbours(rep + WPC, L, L8, y, t, y & 1);
                const uint32_t d = count_differ(rep[w], nb.up, nb.down, nb.same, nb.shifted);
                agree += 16 - (int)((d * 0x01010101u) >> 24);
            }
            agree = __reduce_add_sync(0xFFFFFFFFu, agree);
            int best = 0;
            for (int s = 0; s < G.q; ++s) {
                const uint32_t S4 = (uint32_t)s * 0x01010101u;
                int cnt = 0;
                for (int w = lane; w < WPR; w += 32) cnt += 4 - __popc(differ_bits(rep[w], S4));
                cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
                best = max(best, cnt);
            }
            if (lane == 0) record_replica(G, first + r, -agree, best, N, sE, sE2, sM);
        }
    } else {
        for (int r = 0; r < nrep; ++r) {
            const uint32_t *rep = sw + r * WPR;
            int agree = 0;
            for (int w = tid; w < WPC; w += blockDim.x) {
                const int y = w / L8;
                const int t = w - y * L8;
                const Neighbours nb = load_neighbours(rep + WPC, L, L8, y, t, y & 1);
                const uint32_t d = count_differ(rep[w], nb.up, nb.down, nb.same, nb.shifted);
                agree += 16 - (int)((d * 0x01010101u) >> 24);
            }
            agree = block_sum_int(agree);
            int best = 0;
            for (int s = 0; s < G.q; ++s) {
                const uint32_t S4 = (uint32_t)s * 0x01010101u;
                int cnt = 0;
                for (int w = tid; w < WPR; w += blockDim.x) cnt += 4 - __popc(differ_bits(rep[w], S4));
                cnt = block_sum_int(cnt);
                best = max(best, cnt);
            }
            if (tid == 0) record_replica(G, first + r, -agree, best, N, sE, sE2, sM);
        }
    }
    group_families(G);
    __syncthreads();
    if (G.write_back) {
        for (int i = tid; i < nrep * UPR; i += blockDim.x) {
            const int r = i / UPR;
            const int o = i - r * UPR;
            reinterpret_cast<uint4 *>(G.out + (size_t)(first + r) * N)[o] = smem4[r * UPR + o];
        }
    }
    __syncthreads();
}

// Per-site body for any even L (used where L % 8 != 0), same random-number
// assignment as the row-segment body.
__device__ __forceinline__ void sweep_group_sites(const Group &G, int L, uint4 *smem4, const uint32_t *s_thr,
                                                  const uint32_t *rk0, const uint32_t *rk1, long long &sE,
                                                  long long &sE2, long long &sM)
{
    uint8_t *sb = reinterpret_cast<uint8_t *>(smem4);
    const int L2 = L / 2;
    const int N = L * L;
    const int NH = N / 2;
    const int NP = (N + 15) & ~15;  // padded bytes per replica in shared memory
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    const uint32_t qm1 = (uint32_t)(G.q - 1);
    const int first = G.first, nrep = G.nrep;

    for (int i = tid; i < nrep * N; i += blockDim.x) {
        const int r = i / N;
        const int o = i - r * N;
        const int slot = first + r;
        const int src = G.gather ? G.parent[slot] : slot;
        sb[r * NP + o] = G.in[(size_t)src * N + o];
    }
    __syncthreads();
    for (int k = 0; k < G.theta; ++k) {
        for (int c = 0; c < 2; ++c) {
            const uint32_t ctr1 = DOM_SWEEP | (uint32_t)(2 * k + c);
            for (int i = tid; i < nrep * NH; i += blockDim.x) {
                const int r = i / NH;
                const int h = i - r * NH;
                const int y = h / L2;
                const int m = h - y * L2;
                const int p = (y + c) & 1;
                uint8_t *own = sb + r * NP + c * NH;
                const uint8_t *oth = sb + r * NP + (c ^ 1) * NH;
                const int yu = (y == 0) ? L - 1 : y - 1;
                const int yd = (y == L - 1) ? 0 : y + 1;
                const int mo = p ? (m + 1 == L2 ? 0 : m + 1) : (m == 0 ? L2 - 1 : m - 1);
                const int n0 = oth[yu * L2 + m], n1 = oth[yd * L2 + m], n2 = oth[y * L2 + m], n3 = oth[y * L2 + mo];
                const int s = own[h];
                const uint4 rw = philox10_rk(
                    make_uint4((uint32_t)h >> 2, ctr1, (uint32_t)G.step, (uint32_t)(first + r) | G.stream_hi), rk0, rk1);
                const uint32_t u = pick_word(rw, h & 3);
                int prop = s + 1 + (int)__umulhi(u, qm1);
                if (prop >= G.q) prop -= G.q;
                const int ns = (n0 == s) + (n1 == s) + (n2 == s) + (n3 == s);
                const int np = (n0 == prop) + (n1 == prop) + (n2 == prop) + (n3 == prop);
                if (u * qm1 < s_thr[ns - np + 4]) own[h] = (uint8_t)prop;
            }
            __syncthreads();
        }
    }
    for (int r = warp; r < nrep; r += nwarps) {
        const uint8_t *rep = sb + r * NP;
        int agree = 0;
        for (int h = lane; h < NH; h += 32) {
            const int y = h / L2;
            const int m = h - y * L2;
            const int p = y & 1;
            const uint8_t *oth = rep + NH;
            const int yu = (y == 0) ? L - 1 : y - 1;
            const int yd = (y == L - 1) ? 0 : y + 1;
            const int mo = p ? (m + 1 == L2 ? 0 : m + 1) : (m == 0 ? L2 - 1 : m - 1);
            const int s = rep[h];
            agree += (oth[yu * L2 + m] == s) + (oth[yd * L2 + m] == s) + (oth[y * L2 + m] == s) +
                     (oth[y * L2 + mo] == s);
        }
        agree = __reduce_add_sync(0xFFFFFFFFu, agree);
        int best = 0;
        for (int s = 0; s < G.q; ++s) {
            int cnt = 0;
            for (int i = lane; i < N; i += 32) cnt += rep[i] == s;
            cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
            best = max(best, cnt);
        }
        if (lane == 0) record_replica(G, first + r, -agree, best, N, sE, sE2, sM);
    }
    group_families(G);
    __syncthreads();
    if (G.write_back) {
        for (int i = tid; i < nrep * N; i += blockDim.x) {
            const int r = i / N;
            const int o = i - r * N;
            G.out[(size_t)(first + r) * N + o] = sb[r * NP + o];
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
// Initial population (Sec. 2 step 1; Sec. 5 Eq. 6) for quads [i0, i1) of the
// flattened (slot, site / 4) index.
// ===========================================================================
__device__ __forceinline__ void init_quad(uint8_t *spins, int32_t *anc, int q, int L, long long i, uint32_t k0,
                                          uint32_t k1, uint32_t stream_hi, int ground)
{
    const int N = L * L;
    const int NH = N / 2;
    const int L2 = L / 2;
    const int slot = (int)(i / (N / 4));
    const int quad = (int)(i - (long long)slot * (N / 4));
    uint8_t *rep = spins + (size_t)slot * N;
    uint8_t v[4];
    if (ground) {
        const uint4 w = philox10(make_uint4((uint32_t)slot >> 2, DOM_GROUND, 0u, stream_hi), k0, k1);
        const uint8_t alpha = (uint8_t)__umulhi(pick_word(w, slot & 3), (uint32_t)q);
        v[0] = v[1] = v[2] = v[3] = alpha;
    } else {
        const uint4 w = philox10(make_uint4((uint32_t)quad, DOM_INIT, 0u, (uint32_t)slot | stream_hi), k0, k1);
        v[0] = (uint8_t)__umulhi(w.x, (uint32_t)q);
        v[1] = (uint8_t)__umulhi(w.y, (uint32_t)q);
        v[2] = (uint8_t)__umulhi(w.z, (uint32_t)q);
        v[3] = (uint8_t)__umulhi(w.w, (uint32_t)q);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int site = 4 * quad + j;  // canonical y*L + x
        const int y = site / L, x = site - y * L;
        const int c = (x + y) & 1;
        rep[c * NH + y * L2 + (x >> 1)] = v[j];
    }
    if (quad == 0 && anc) anc[slot] = slot;
}

// ===========================================================================
// Resampling bodies (Sec. 2 step 2, Eq. 2)
// ===========================================================================

// One block: reference bin, weight table, S and ln Q of the pending resample.
__device__ __forceinline__ void weights_body(const int32_t *hist, int nbins, double dbeta, DevState *st, double *wtab,
                                             double *s_d, long long *s_l)
{
    if (st->err) return;
    const int tid = threadIdx.x;
    // reference bin: lowest occupied for dbeta >= 0, highest for dbeta < 0
    long long best = dbeta >= 0.0 ? (long long)INT_MAX : -1;
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

    // only occupied bins: an empty bin on the far side of E_ref could hold an
    // overflowing factor, and 0 * inf would poison the sum
    double part = 0.0;
    for (int k = tid; k < nbins; k += blockDim.x) {
        const int h = hist[k];
        if (h == 0) continue;
        const double w = exp(__dmul_rn(-dbeta, (double)(k - kref)));
        wtab[k] = w;
        part = __dadd_rn(part, __dmul_rn((double)h, w));
    }
    const double S = block_sum_fixed(part, s_d);
    if (tid == 0) {
        const int E_ref = kref - (nbins - 1);
        st->S = S;
        st->E_ref = E_ref;
        st->lnQ = __dadd_rn(__dmul_rn(-dbeta, (double)E_ref), log(S / (double)st->pop));
    }
}

// A Poisson draw with mean rho for replica j (Sec. 2, Eq. 1): inversion of
// the cumulative distribution with the mean split into pieces of at most 64;
// the k-th uniform (U_k + 1/2) / 2^32 is word k & 3 of counter
// (j, RESAMPLE | (1 + k / 4), step, stream).
__device__ __forceinline__ int poisson_draw(double rho, int j, int step, uint32_t stream_hi, uint32_t k0, uint32_t k1)
{
    int r = 0;
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
        while (u > F && n < 1000) {
            n += 1;
            p = __ddiv_rn(__dmul_rn(p, mu), (double)n);
            F = __dadd_rn(F, p);
        }
        r += n;
    }
    return r;
}

// One block of 1024 old replicas (chunk): copy numbers and their block scan.
__device__ __forceinline__ void counts_body(int chunk, const int32_t *E, int twoN, int R_target, int mode, int step,
                                            uint32_t stream_hi, uint32_t k0, uint32_t k1, const double *wtab,
                                            int32_t *counts, int32_t *local_off, int32_t *blocksum, DevState *st,
                                            int *s_i)
{
    if (st->err) return;
    const int R_prev = st->pop;
    if (chunk * (int)blockDim.x >= R_prev) return;
    const int j = chunk * blockDim.x + threadIdx.x;
    int r = 0;
    if (j < R_prev) {
        const double w = wtab[E[j] + twoN];
        const double rho = __ddiv_rn(__dmul_rn((double)R_target, w), st->S);
        const double n = floor(rho);
        const double frac = __dsub_rn(rho, n);
        if (mode == 2) {
            r = poisson_draw(rho, j, step, stream_hi, k0, k1);
        } else if (mode == 3) {
            r = 1;
        } else {
            int up;
            if (mode == 1) {
                up = frac >= 0.5;
            } else {
                const uint4 u = philox10(make_uint4((uint32_t)j >> 2, DOM_RESAMPLE, (uint32_t)step, stream_hi), k0, k1);
                up = (double)pick_word(u, j & 3) < __dmul_rn(frac, 4294967296.0);
            }
            r = (int)n + up;
        }
        counts[j] = r;
    }
    int total;
    const int before = block_exclusive_scan(r, s_i, &total);
    if (j < R_prev) local_off[j] = before;
    if (threadIdx.x == 0) blocksum[chunk] = total;
}

// One block (chunk of nchunks): block offsets, new size (capacity check),
// parent map; the chunks also clear the histogram for the next sweep.
__device__ __forceinline__ void scatter_body(int chunk, int nchunks, const int32_t *counts, const int32_t *local_off,
                                             const int32_t *blocksum, int32_t *parent, int R_cap, int32_t *hist_zero,
                                             int nbins, DevState *st, long long *s_l)
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
    if (tot > R_cap || tot <= 0) {
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
__device__ __forceinline__ void finalize_body(DevState *st, unsigned long long *acc, int32_t *fam, int R0, DevObs *obs,
                                              double beta, int q, int N, int gathered, int resampled, double *s_d,
                                              long long *s_l)
{
    if (st->err) return;
    const int R = gathered ? st->pop_next : st->pop;
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
            st->pop = R;
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
        o.sumE = sE;
        o.sumE2 = sE2;
        o.sumMt = sM;
        *obs = o;
    }
}

}  // namespace dev
}  // namespace pa
