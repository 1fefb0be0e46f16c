// pa_sweep.cu -- the Metropolis sweep kernel of population annealing
// (Barash, Weigel, Shchur & Janke, arXiv:1704.01888, Sec. 2 step 3 and Sec. 3),
// fused with the replica gather of the preceding resampling step (Sec. 2 step 2)
// and with the per-replica measurements of step 4 (Eq. 3 energy, Eq. 5
// largest-state occupation) and the energy histogram.
//
// One block keeps `rpb` whole lattices resident in shared memory and runs all
// theta sweeps on them, so HBM sees each lattice once in and once out per
// temperature step.  Blocks are persistent: they stride over groups of rpb
// replicas until the device-side population size is covered.
//
// Inner loop (lattices with L % 8 == 0): one thread updates four consecutive
// same-colour sites held in one 32-bit word.  Their neighbours are the
// aligned words of the other colour in the rows above and below and in the
// same row, plus that row word shifted by one byte.  Neighbour agreement is
// counted four bytes at a time (SWAR).  Each site takes one 32-bit Philox
// word u: the high and low halves of u (q-1) are its proposal offset and its
// acceptance uniform.  Lattices with other even L use a per-site kernel with
// the same random-number assignment, so both give identical results.
#include "pa_internal.cuh"

namespace pa {

namespace {

// Bit 7 of each byte is set where the bytes of a and b differ (all bytes < 128).
__device__ __forceinline__ uint32_t differ_bits(uint32_t a, uint32_t b)
{
    return ((a ^ b) + 0x7F7F7F7Fu) & 0x80808080u;
}

// Per byte: how many of the four neighbour words differ from a (0..4).
__device__ __forceinline__ uint32_t count_differ(uint32_t a, uint32_t n0, uint32_t n1, uint32_t n2,
                                                 uint32_t n3)
{
    return (differ_bits(a, n0) >> 7) + (differ_bits(a, n1) >> 7) + (differ_bits(a, n2) >> 7) +
           (differ_bits(a, n3) >> 7);
}

struct Neighbours {
    uint32_t up, down, same, shifted;
};

// Neighbour words of word t in row y of a colour whose row offset is p =
// (y + colour) & 1.  `oth` is the other colour's sublattice of the replica.
__device__ __forceinline__ Neighbours load_neighbours(const uint32_t *oth, int L, int L8, int y, int t,
                                                      int p)
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

__device__ __forceinline__ void accumulate_totals(unsigned long long *acc, long long sE, long long sE2,
                                                  long long sM)
{
    atomicAdd(acc + 0, (unsigned long long)sE);
    atomicAdd(acc + 1, (unsigned long long)sE2);
    atomicAdd(acc + 2, (unsigned long long)sM);
}

// Copies of the per-replica bookkeeping shared by both kernels: energies,
// occupations, histogram and ancestors of one finished replica.
__device__ __forceinline__ void record_replica(const SweepArgs &a, int slot, int E, int Mt, int N,
                                               long long &sE, long long &sE2, long long &sM)
{
    a.E[slot] = E;
    a.Mt[slot] = Mt;
    atomicAdd(a.hist + (E + 2 * N), 1);
    sE += E;
    sE2 += (long long)E * (long long)E;
    sM += Mt;
}

// ---------------------------------------------------------------------------
// Row-segment kernel: L % 8 == 0.  LT > 0 fixes L at compile time; S is the
// number of 32-bit words (4 same-colour sites each) one thread updates per
// step of its loop: S consecutive words of one row of one colour, read and
// written with one vector access per neighbour row.
// ---------------------------------------------------------------------------
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

using KernelFnPtr = void (*)(const SweepArgs);

template <int LT, int S>
__global__ void __launch_bounds__(1024) k_sweep_rows(const SweepArgs a)
{
    extern __shared__ uint4 smem4[];
    __shared__ uint32_t s_thr[9];
    uint32_t *sw = reinterpret_cast<uint32_t *>(smem4);

    const int L = LT > 0 ? LT : a.L;
    const int N = L * L;
    const int L8 = L / 8;    // words per row of one colour
    const int WPC = N / 8;   // words per colour per replica
    const int WPR = N / 4;   // words per replica
    const int UPR = N / 16;  // uint4 per replica
    const int SPR = L8 / S;  // segments per row
    const int UPC = L * SPR; // segments per colour per replica
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;

    if (tid < 9) s_thr[tid] = a.thr[tid];
    DevState *st = a.st;
    if (st->err) return;
    const int parity = st->parity;
    const int R = a.gather ? st->pop_next : st->pop;
    const uint8_t *in = a.buf[parity];
    uint8_t *out = a.gather ? a.buf[parity ^ 1] : a.buf[parity];
    const int32_t *anc_in = a.anc[parity];
    int32_t *anc_out = a.gather ? a.anc[parity ^ 1] : a.anc[parity];
    const uint32_t qm1 = (uint32_t)(a.q - 1);
    const uint32_t qb = (uint32_t)a.q;
    const bool write_back = a.gather || a.theta > 0;
    const char *thr_bytes = reinterpret_cast<const char *>(s_thr);

    long long sE = 0, sE2 = 0, sM = 0;
    for (int g = blockIdx.x; g * a.rpb < R; g += gridDim.x) {
        const int first = g * a.rpb;
        const int nrep = min(a.rpb, R - first);

        // gather: replica first + r comes from its parent's lattice
        for (int i = tid; i < nrep * UPR; i += blockDim.x) {
            const int r = i / UPR;
            const int o = i - r * UPR;
            const int slot = first + r;
            const int src = a.gather ? a.parent[slot] : slot;
            smem4[r * UPR + o] = reinterpret_cast<const uint4 *>(in + (size_t)src * N)[o];
        }
        __syncthreads();

        for (int k = 0; k < a.theta; ++k) {
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
                    const uint32_t slot = (uint32_t)(first + r);
                    Vec<S> NW;
#pragma unroll
                    for (int j = 0; j < S; ++j) {
                        const uint32_t lo = p ? H.v[j] : (j == 0 ? edge : H.v[j > 0 ? j - 1 : 0]);
                        const uint32_t hi = p ? (j == S - 1 ? edge : H.v[j < S - 1 ? j + 1 : 0]) : H.v[j];
                        const uint32_t shifted = __funnelshift_r(lo, hi, sh);
                        const uint32_t Wj = W.v[j];
                        // one word per site: (high, low) of u (q-1) = (proposal offset, acceptance uniform)
                        const uint4 ru = philox10_rk(make_uint4(quad0 + j, ctr1, (uint32_t)a.step, slot), a.rk0,
                                                     a.rk1);
                        const uint32_t m = __umulhi(ru.x, qm1) | (__umulhi(ru.y, qm1) << 8) |
                                           (__umulhi(ru.z, qm1) << 16) | (__umulhi(ru.w, qm1) << 24);
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
                        sel += (ru.x * qm1 < T0) ? 0x4u : 0u;
                        sel += (ru.y * qm1 < T1) ? 0x40u : 0u;
                        sel += (ru.z * qm1 < T2) ? 0x400u : 0u;
                        sel += (ru.w * qm1 < T3) ? 0x4000u : 0u;
                        NW.v[j] = __byte_perm(Wj, P, sel);
                    }
                    NW.store(own + row + t0);
                }
                __syncthreads();
            }
        }

        // measurements: one warp per replica
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
            for (int s = 0; s < a.q; ++s) {
                const uint32_t S4 = (uint32_t)s * 0x01010101u;
                int cnt = 0;
                for (int w = lane; w < WPR; w += 32) cnt += 4 - __popc(differ_bits(rep[w], S4));
                cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
                best = max(best, cnt);
            }
            if (lane == 0) record_replica(a, first + r, -agree, best, N, sE, sE2, sM);
        }
        if (a.fam) {
            for (int r = tid; r < nrep; r += blockDim.x) {
                const int slot = first + r;
                const int f = anc_in[a.gather ? a.parent[slot] : slot];
                if (a.gather) anc_out[slot] = f;
                atomicAdd(a.fam + f, 1);
            }
        }
        __syncthreads();
        if (write_back) {
            for (int i = tid; i < nrep * UPR; i += blockDim.x) {
                const int r = i / UPR;
                const int o = i - r * UPR;
                reinterpret_cast<uint4 *>(out + (size_t)(first + r) * N)[o] = smem4[r * UPR + o];
            }
        }
        __syncthreads();
    }
    if (lane == 0 && (sE | sE2 | sM)) accumulate_totals(a.acc, sE, sE2, sM);
}

// ---------------------------------------------------------------------------
// Site kernel: any even L (used where L % 8 != 0).  One thread per site.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_sweep_sites(const SweepArgs a)
{
    extern __shared__ uint4 smem4[];
    __shared__ uint32_t s_thr[9];
    uint8_t *sb = reinterpret_cast<uint8_t *>(smem4);

    const int L = a.L;
    const int L2 = L / 2;
    const int N = L * L;
    const int NH = N / 2;
    const int NP = (N + 15) & ~15;  // padded bytes per replica in shared memory
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;

    if (tid < 9) s_thr[tid] = a.thr[tid];
    DevState *st = a.st;
    if (st->err) return;
    const int parity = st->parity;
    const int R = a.gather ? st->pop_next : st->pop;
    const uint8_t *in = a.buf[parity];
    uint8_t *out = a.gather ? a.buf[parity ^ 1] : a.buf[parity];
    const int32_t *anc_in = a.anc[parity];
    int32_t *anc_out = a.gather ? a.anc[parity ^ 1] : a.anc[parity];
    const uint32_t qm1 = (uint32_t)(a.q - 1);
    const bool write_back = a.gather || a.theta > 0;

    long long sE = 0, sE2 = 0, sM = 0;
    for (int g = blockIdx.x; g * a.rpb < R; g += gridDim.x) {
        const int first = g * a.rpb;
        const int nrep = min(a.rpb, R - first);
        for (int i = tid; i < nrep * N; i += blockDim.x) {
            const int r = i / N;
            const int o = i - r * N;
            const int slot = first + r;
            const int src = a.gather ? a.parent[slot] : slot;
            sb[r * NP + o] = in[(size_t)src * N + o];
        }
        __syncthreads();
        for (int k = 0; k < a.theta; ++k) {
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
                    const int n0 = oth[yu * L2 + m], n1 = oth[yd * L2 + m], n2 = oth[y * L2 + m],
                              n3 = oth[y * L2 + mo];
                    const int s = own[h];
                    const uint4 rw = philox10_rk(make_uint4((uint32_t)h >> 2, ctr1, (uint32_t)a.step,
                                                            (uint32_t)(first + r)),
                                                 a.rk0, a.rk1);
                    const uint32_t u = pick_word(rw, h & 3);
                    int prop = s + 1 + (int)__umulhi(u, qm1);
                    if (prop >= a.q) prop -= a.q;
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
            for (int s = 0; s < a.q; ++s) {
                int cnt = 0;
                for (int i = lane; i < N; i += 32) cnt += rep[i] == s;
                cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
                best = max(best, cnt);
            }
            if (lane == 0) record_replica(a, first + r, -agree, best, N, sE, sE2, sM);
        }
        if (a.fam) {
            for (int r = tid; r < nrep; r += blockDim.x) {
                const int slot = first + r;
                const int f = anc_in[a.gather ? a.parent[slot] : slot];
                if (a.gather) anc_out[slot] = f;
                atomicAdd(a.fam + f, 1);
            }
        }
        __syncthreads();
        if (write_back) {
            for (int i = tid; i < nrep * N; i += blockDim.x) {
                const int r = i / N;
                const int o = i - r * N;
                out[(size_t)(first + r) * N + o] = sb[r * NP + o];
            }
        }
        __syncthreads();
    }
    if (lane == 0 && (sE | sE2 | sM)) accumulate_totals(a.acc, sE, sE2, sM);
}

// Allows each kernel the device's full opt-in shared memory, so that the
// per-launch request alone decides occupancy.
cudaError_t prepare(KernelFnPtr kernel)
{
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - 1024);
    return e;
}

KernelFnPtr pick_kernel(int L)
{
    if (L % 8 != 0) return k_sweep_sites;
    switch (L) {
    case 16: return k_sweep_rows<16, 2>;
    case 32: return k_sweep_rows<32, 4>;
    case 48: return k_sweep_rows<48, 2>;
    case 64: return k_sweep_rows<64, 4>;
    case 128: return k_sweep_rows<128, 4>;
    case 256: return k_sweep_rows<256, 4>;
    default:
        if ((L / 8) % 4 == 0) return k_sweep_rows<0, 4>;
        if ((L / 8) % 2 == 0) return k_sweep_rows<0, 2>;
        return k_sweep_rows<0, 1>;
    }
}

}  // namespace

size_t sweep_smem_bytes(int L, int rpb)
{
    const size_t N = (size_t)L * L;
    return (size_t)rpb * ((N + 15) & ~(size_t)15);
}

int sweep_max_blocks_per_sm(int L, int rpb, int threads)
{
    KernelFnPtr k = pick_kernel(L);
    const size_t smem = sweep_smem_bytes(L, rpb);
    if (prepare(k) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem) != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_sweep(const SweepArgs &a, int threads, int grid, cudaStream_t s)
{
    KernelFnPtr k = pick_kernel(a.L);
    const size_t smem = sweep_smem_bytes(a.L, a.rpb);
    k<<<grid, threads, smem, s>>>(a);
    bump_launch_count(1);
    return cudaGetLastError();
}

}  // namespace pa
