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
#include "pa_kernels.cuh"

namespace pa {

namespace {

using KernelFnPtr = void (*)(const SweepArgs);

__device__ __forceinline__ dev::Group make_group(const SweepArgs &a, int parity, int first, int nrep)
{
    dev::Group G;
    G.in = a.buf[parity];
    G.out = a.gather ? a.buf[parity ^ 1] : a.buf[parity];
    G.parent = a.parent;
    G.anc_in = a.anc[parity];
    G.anc_out = a.gather ? a.anc[parity ^ 1] : a.anc[parity];
    G.fam = a.fam;
    G.E = a.E;
    G.Mt = a.Mt;
    G.hist = a.hist;
    G.first = first;
    G.nrep = nrep;
    G.q = a.q;
    G.theta = a.theta;
    G.step = a.step;
    G.stream_hi = a.stream_hi;
    G.gather = a.gather != 0;
    G.write_back = a.gather || a.theta > 0;
    return G;
}

// Row-segment kernel (L % 8 == 0): persistent blocks stride over groups of
// rpb replicas of the current population.
template <int LT, int S>
__global__ void __launch_bounds__(1024) k_sweep_rows(const SweepArgs a)
{
    extern __shared__ uint4 smem4[];
    __shared__ uint32_t s_thr[9];
    if (threadIdx.x < 9) s_thr[threadIdx.x] = a.thr[threadIdx.x];
    DevState *st = a.st;
    if (st->err) return;
    const int parity = st->parity;
    const int R = a.gather ? st->pop_next : st->pop;
    long long sE = 0, sE2 = 0, sM = 0;
    for (int g = blockIdx.x; g * a.rpb < R; g += gridDim.x) {
        const int first = g * a.rpb;
        const dev::Group G = make_group(a, parity, first, min(a.rpb, R - first));
        dev::sweep_group_rows<LT, S>(G, a.L, smem4, s_thr, a.rk0, a.rk1, sE, sE2, sM);
    }
    if ((threadIdx.x & 31) == 0 && (sE | sE2 | sM)) dev::accumulate_totals(a.acc, sE, sE2, sM);
}

// Site kernel: any even L (used where L % 8 != 0).
__global__ void __launch_bounds__(1024) k_sweep_sites(const SweepArgs a)
{
    extern __shared__ uint4 smem4[];
    __shared__ uint32_t s_thr[9];
    if (threadIdx.x < 9) s_thr[threadIdx.x] = a.thr[threadIdx.x];
    DevState *st = a.st;
    if (st->err) return;
    const int parity = st->parity;
    const int R = a.gather ? st->pop_next : st->pop;
    long long sE = 0, sE2 = 0, sM = 0;
    for (int g = blockIdx.x; g * a.rpb < R; g += gridDim.x) {
        const int first = g * a.rpb;
        const dev::Group G = make_group(a, parity, first, min(a.rpb, R - first));
        dev::sweep_group_sites(G, a.L, smem4, s_thr, a.rk0, a.rk1, sE, sE2, sM);
    }
    if ((threadIdx.x & 31) == 0 && (sE | sE2 | sM)) dev::accumulate_totals(a.acc, sE, sE2, sM);
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
