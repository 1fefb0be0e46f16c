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
// Spins are multi-spin coded: the states of 32 same-colour sites of a row sit
// in B bit planes (B = ceil(log2 q)), and each thread updates such a site
// word with 32-bit logic: the proposal by ripple-carry additions over the
// planes, the energy change by bitwise equality tests and a carry-save count,
// the acceptance by a most-significant-bit-first comparison of random bits
// with the thresholds (the body is dev::sweep_group_bits).  One kernel is
// compiled per B and row geometry.
#include "pa_sweep_body.cuh"

namespace pa {

namespace {

using KernelFnPtr = void (*)(const SweepArgs);

// Group of the local slots [first, first + nrep).  A population spread over
// several GPUs numbers its replicas by global slot (slot0 + local slot): the
// group carries global slot numbers, for the random keys, and array bases
// moved down by slot0, so that indexing by global slot lands on the local
// entries (slot0 = 0 on one GPU).
__device__ __forceinline__ dev::Group make_group(const SweepArgs &a, int parity, int first, int nrep)
{
    const size_t s0 = a.slot0;
    const size_t RW = (size_t)replica_words(a.q, a.L);
    // arrays indexed by slot move down by slot0; a gather's sources are indexed
    // by the parent map's values, which are local
    const size_t s_in = a.gather ? 0 : s0;
    dev::Group G;
    G.in = a.buf[parity] - s_in * RW;
    G.out = (a.gather ? a.buf[parity ^ 1] : a.buf[parity]) - s0 * RW;
    G.parent = a.parent ? a.parent - s0 : nullptr;
    G.anc_in = a.anc[parity] ? a.anc[parity] - s_in : nullptr;
    G.anc_out = a.gather ? a.anc[parity ^ 1] : a.anc[parity];
    if (G.anc_out) G.anc_out -= s0;
    G.fam = a.fam;
    G.E = a.E - s0;
    G.Mt = a.Mt - s0;
    G.hist = a.hist;
    G.first = (int)a.slot0 + first;
    G.nrep = nrep;
    G.q = a.q;
    G.theta = a.theta;
    G.step = a.step;
    G.stream_hi = a.stream_hi;
    G.gather = a.gather != 0;
    G.write_back = a.gather || a.theta > 0;
#if PA_CHECKED
    G.src_limit = a.st->pop;  // the old population (received runs on a shard) until k_finalize
    G.err = &a.st->err;
#endif
    return G;
}

// Persistent blocks over groups of at most rpb replicas of the current
// population (R_i is known only on the device).  With a.work the blocks take
// groups one at a time from a counter, which ends every block within one
// group of the others (for launches of a few groups per block: 1915 against
// 1845 attempts/ns at q = 10, L = 64, R = 1e5); else each block takes an equal
// share, counted in quanta of blockDim / (site words per colour) replicas, the
// number that fills one pass of the block's threads over the site words, so
// that no block and no pass is left part-empty.
// B: bits per state; MODE: 0 for L = 64, 1 for L a multiple of 64, 3 for
// L = 8, 16, 32 (rows packed several to a word), 4 for L = 48, 80, 96, ...
// (banded 8-column segments), 2 otherwise (rows padded to whole words).
template <int B, int MODE, int Q>
__global__ void __launch_bounds__(1024) k_sweep(const SweepArgs a)
{
    extern __shared__ uint4 smem4[];
    __shared__ uint4 s_tab[dev::kThresholdEntries];
    constexpr int QCAP = B <= 4 ? 384 : dev::kQueueCap;
    __shared__ uint32_t s_queue[dev::queue_words(B, QCAP)];
    dev::build_threshold_table(s_tab, a.thr);
    DevState *st = a.st;
    if (st->err) return;
    const int parity = st->parity;
    const int R = a.gather ? st->pop_next : st->pop;
    __shared__ int s_group;
    const bool dynamic = a.work != nullptr;
    const int words = colour_words(a.L);
    const int quantum = max(1, min(a.rpb, (int)blockDim.x / words));
    const long long nq = (R + quantum - 1) / quantum;
    const int end = dynamic ? R : min(R, (int)(nq * (blockIdx.x + 1) / gridDim.x) * quantum);
    int first = dynamic ? 0 : (int)(nq * blockIdx.x / gridDim.x) * quantum;
    long long sE = 0, sE2 = 0, sM = 0;
    for (;; first += a.rpb) {
        if (dynamic) {
            if (threadIdx.x == 0) s_group = atomicAdd(a.work, 1);
            __syncthreads();
            first = s_group * a.rpb;
            __syncthreads();
        }
        if (first >= end) break;
        const dev::Group G = make_group(a, parity, first, min(a.rpb, end - first));
        dev::sweep_group_bits<B, MODE, Q, MODE == 0 || MODE == 1, QCAP, MODE != 0>(
            G, a.L, reinterpret_cast<uint32_t *>(smem4), s_tab, s_queue, a.rk0, a.rk1, sE, sE2, sM);
    }
    if ((threadIdx.x & 31) == 0 && (sE | sE2 | sM)) dev::accumulate_totals(a.acc, sE, sE2, sM);
}

// Allows each kernel the device's full opt-in shared memory (less its static
// shared memory), so that the per-launch request alone decides occupancy.
cudaError_t prepare(KernelFnPtr kernel)
{
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    return e;
}

// Kernels for the common q with q fixed at compile time (the reduction mod q
// then uses constant masks), and one kernel per bit count for any other q.
template <int MODE>
KernelFnPtr pick_q(int q)
{
    switch (q) {
    case 2: return k_sweep<state_bits(2), MODE, 2>;
    case 3: return k_sweep<state_bits(3), MODE, 3>;
    case 4: return k_sweep<state_bits(4), MODE, 4>;
    case 5: return k_sweep<state_bits(5), MODE, 5>;
    case 6: return k_sweep<state_bits(6), MODE, 6>;
    case 8: return k_sweep<state_bits(8), MODE, 8>;
    case 10: return k_sweep<state_bits(10), MODE, 10>;
    case 20: return k_sweep<state_bits(20), MODE, 20>;
    }
    switch (state_bits(q)) {
    case 1: return k_sweep<1, MODE, 0>;
    case 2: return k_sweep<2, MODE, 0>;
    case 3: return k_sweep<3, MODE, 0>;
    case 4: return k_sweep<4, MODE, 0>;
    case 5: return k_sweep<5, MODE, 0>;
    case 6: return k_sweep<6, MODE, 0>;
    default: return k_sweep<7, MODE, 0>;
    }
}

KernelFnPtr pick_kernel(int q, int L)
{
    if (L == 64) return pick_q<0>(q);
    if (L % 64 == 0) return pick_q<1>(q);
    if (rows_packed(L)) return pick_q<3>(q);
    if (rows_banded(L)) return pick_q<4>(q);
    return pick_q<2>(q);
}

}  // namespace

size_t sweep_smem_bytes(int q, int L, int rpb) { return (size_t)rpb * replica_bytes(q, L); }

int sweep_max_blocks_per_sm(int q, int L, int rpb, int threads)
{
    KernelFnPtr k = pick_kernel(q, L);
    const size_t smem = sweep_smem_bytes(q, L, rpb);
    if (prepare(k) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem) != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_sweep(const SweepArgs &a, int threads, int grid, cudaStream_t s)
{
    KernelFnPtr k = pick_kernel(a.q, a.L);
    const size_t smem = sweep_smem_bytes(a.q, a.L, a.rpb);
    if (a.work) {
        const cudaError_t e = cudaMemsetAsync(a.work, 0, sizeof(int32_t), s);
        if (e != cudaSuccess) return e;
    }
    k<<<grid, threads, smem, s>>>(a);
    bump_launch_count(1);
    return cudaGetLastError();
}

}  // namespace pa
