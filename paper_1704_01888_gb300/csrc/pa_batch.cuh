// pa_batch.cuh -- device structures of the batched engine (pa_batch.cu) and
// its persistent sweep kernel.  The sweep kernel comes in two parts, each
// holding the bodies of one range of bits per state: part 0 the runs with
// q <= 16 (at most four bit planes), part 1 the runs with larger q.  They are
// compiled in separate translation units (part 1 in pa_batch_hi.cu), so that
// each part gets its own register allocation -- one function over every body
// spilled for the sake of the seven-plane bodies -- and the two build in
// parallel.  A temperature step launches the parts its runs need, one after
// the other; results do not depend on the split.
#pragma once
#include "pa_kernels.cuh"

namespace pa {

constexpr int kB = 1024;
constexpr int kMaxRuns = 1024;

struct RunDev {
    uint32_t *buf[2];
    int32_t *anc[2];
    int32_t *parent, *E, *Mt, *hist, *fam, *counts, *local_off, *blocksum;
    unsigned long long *acc;
    DevState *st;
    DevObs *obs;  // K + 1 records
    int32_t q, L, N, nbins, R0, R_cap, mode, rpb, chunk0, nchunks, K, ground;
    uint32_t stream_hi;
    long long item0;  // first site word of this run in the flattened init index
};

struct StepDev {  // one per (step, run)
    Thresholds thr;
    double beta, dbeta;
    const double *wtab;  // weight table of dbeta (pa::weight_table), 2N + 1 entries
    int32_t theta, active;
};

struct BatchArgs {
    const RunDev *runs;
    const StepDev *steps;  // (K_max + 1) x M
    const int32_t *step_counter;
    int32_t *work;         // per part and step: next replica group to hand out (zeroed at start)
    int32_t work_stride;   // counters per part (K_max + 1)
    const int32_t *order;  // runs by decreasing estimated cost of one group
    int32_t M, total_chunks;
    long long total_items;
    uint32_t k0, k1;
    uint32_t rk0[10], rk1[10];
    int32_t gather;  // 0 for the measurement at step 0
};

// The part of the batched sweep that takes a run's replica groups.
__host__ __device__ constexpr int batch_part(int q) { return state_bits(q) > 4 ? 1 : 0; }

using BatchSweepFn = void (*)(const BatchArgs);
BatchSweepFn batch_sweep_kernel_hi();  // part 1, pa_batch_hi.cu

namespace {

// The sweep body for a run's q -- fixed at compile time for q = 5, 6, 8, 10
// (part 0) and q = 20 (part 1), so that the reduction mod q uses constant
// masks -- else its bits per state, and its row geometry.
template <int MODE, int PART>
__device__ __forceinline__ void batch_body(int qv, int B, const dev::Group &G, int L, uint32_t *sw,
                                           const uint4 *s_tab, uint32_t *q, const BatchArgs &b, long long &sE,
                                           long long &sE2, long long &sM)
{
    if constexpr (PART == 0) {
        switch (qv) {
        case 5: dev::sweep_group_bits<3, MODE, 5>(G, L, sw, s_tab, q, b.rk0, b.rk1, sE, sE2, sM); return;
        case 6: dev::sweep_group_bits<3, MODE, 6>(G, L, sw, s_tab, q, b.rk0, b.rk1, sE, sE2, sM); return;
        case 8: dev::sweep_group_bits<3, MODE, 8>(G, L, sw, s_tab, q, b.rk0, b.rk1, sE, sE2, sM); return;
        case 10: dev::sweep_group_bits<4, MODE, 10>(G, L, sw, s_tab, q, b.rk0, b.rk1, sE, sE2, sM); return;
        default: break;
        }
        switch (B) {
        case 1: dev::sweep_group_bits<1, MODE>(G, L, sw, s_tab, q, b.rk0, b.rk1, sE, sE2, sM); break;
        case 2: dev::sweep_group_bits<2, MODE>(G, L, sw, s_tab, q, b.rk0, b.rk1, sE, sE2, sM); break;
        case 3: dev::sweep_group_bits<3, MODE>(G, L, sw, s_tab, q, b.rk0, b.rk1, sE, sE2, sM); break;
        default: dev::sweep_group_bits<4, MODE>(G, L, sw, s_tab, q, b.rk0, b.rk1, sE, sE2, sM); break;
        }
    } else {
        if (qv == 20) {
            dev::sweep_group_bits<5, MODE, 20>(G, L, sw, s_tab, q, b.rk0, b.rk1, sE, sE2, sM);
            return;
        }
        switch (B) {
        case 5: dev::sweep_group_bits<5, MODE>(G, L, sw, s_tab, q, b.rk0, b.rk1, sE, sE2, sM); break;
        case 6: dev::sweep_group_bits<6, MODE>(G, L, sw, s_tab, q, b.rk0, b.rk1, sE, sE2, sM); break;
        default: dev::sweep_group_bits<7, MODE>(G, L, sw, s_tab, q, b.rk0, b.rk1, sE, sE2, sM); break;
        }
    }
}

// One persistent launch over the replica groups of every active run of this
// part.  Blocks take groups from the part's shared counter, the groups of the
// costliest runs first, so that the heterogeneous groups of different runs
// balance over the SMs.
template <int PART>
__global__ void __launch_bounds__(1024) k_batch_sweep(const BatchArgs b)
{
    extern __shared__ uint4 smem4[];
    __shared__ uint4 s_tab[dev::kThresholdEntries];
    __shared__ int s_prefix[kMaxRuns + 1];
    __shared__ int s_group;
    __shared__ uint32_t s_queue[dev::queue_words(PART == 0 ? 4 : 7)];
    const int i = *b.step_counter;
    int *work = b.work + PART * b.work_stride + i;
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int k = 0; k < b.M; ++k) {
            s_prefix[k] = acc;
            const int m = b.order[k];
            const RunDev &r = b.runs[m];
            const StepDev &sp = b.steps[(size_t)i * b.M + m];
            if (batch_part(r.q) == PART && sp.active && !r.st->err) {
                const int R = b.gather ? r.st->pop_next : r.st->pop;
                acc += (R + r.rpb - 1) / r.rpb;
            }
        }
        s_prefix[b.M] = acc;
    }
    __syncthreads();
    const int total = s_prefix[b.M];
    for (;;) {
        if (threadIdx.x == 0) s_group = atomicAdd(work, 1);
        __syncthreads();
        const int g = s_group;
        __syncthreads();
        if (g >= total) break;
        // the last run whose prefix is <= g: runs without groups here (other
        // part, inactive) share their successor's prefix and are passed over
        int lo = 0, hi = b.M - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (s_prefix[mid] <= g) lo = mid; else hi = mid - 1;
        }
        const int m = b.order[lo];
        const RunDev &r = b.runs[m];
        const StepDev &sp = b.steps[(size_t)i * b.M + m];
        const int parity = r.st->parity;
        const int R = b.gather ? r.st->pop_next : r.st->pop;
        const int first = (g - s_prefix[lo]) * r.rpb;
        dev::Group G;
        G.in = r.buf[parity];
        G.out = b.gather ? r.buf[parity ^ 1] : r.buf[parity];
        G.parent = r.parent;
        G.anc_in = r.anc[parity];
        G.anc_out = b.gather ? r.anc[parity ^ 1] : r.anc[parity];
        G.fam = r.fam;
        G.E = r.E;
        G.Mt = r.Mt;
        G.hist = r.hist;
        G.first = first;
        G.nrep = min(r.rpb, R - first);
        G.q = r.q;
        G.theta = sp.theta;
        G.step = i;
        G.stream_hi = r.stream_hi;
        G.gather = b.gather != 0;
        G.write_back = b.gather || sp.theta > 0;
#if PA_CHECKED
        G.src_limit = r.st->pop;
        G.err = &r.st->err;
#endif
        dev::build_threshold_table(s_tab, sp.thr);
        long long sE = 0, sE2 = 0, sM = 0;
        uint32_t *sw = reinterpret_cast<uint32_t *>(smem4);
        const int B = state_bits(r.q);
        if (r.L == 64)
            batch_body<0, PART>(r.q, B, G, 64, sw, s_tab, s_queue, b, sE, sE2, sM);
        else if (r.L % 64 == 0)
            batch_body<1, PART>(r.q, B, G, r.L, sw, s_tab, s_queue, b, sE, sE2, sM);
        else if (rows_packed(r.L))
            batch_body<3, PART>(r.q, B, G, r.L, sw, s_tab, s_queue, b, sE, sE2, sM);
        else if (rows_banded(r.L))
            batch_body<4, PART>(r.q, B, G, r.L, sw, s_tab, s_queue, b, sE, sE2, sM);
        else
            batch_body<2, PART>(r.q, B, G, r.L, sw, s_tab, s_queue, b, sE, sE2, sM);
        if ((threadIdx.x & 31) == 0 && (sE | sE2 | sM)) dev::accumulate_totals(r.acc, sE, sE2, sM);
    }
}

}  // namespace

}  // namespace pa
