// pa_resample.cu -- initial populations, the resampling step and the
// per-step estimators of population annealing (Barash, Weigel, Shchur & Janke,
// arXiv:1704.01888).
//
//   k_init      Sec. 2 step 1 (uniform spins at beta_0 = 0) or Sec. 5 Eq. 6
//               (a uniformly chosen ground state per replica), written in the
//               multi-spin-coded layout.
//   k_weights   Sec. 2 step 2: reference energy, the histogram-weighted sum
//               S of the Boltzmann factors w = exp(-dbeta (E - E_ref)) (taken
//               from a table the host computes with the C library's exp;
//               summed exactly and rounded once) and
//               ln Q_i = -dbeta E_ref + ln(S/R_{i-1}).
//   k_counts    copy numbers r_j from rho_j = R w(E_j) / S and their
//               block-local exclusive scan (warp shuffles).
//   k_scatter   block offsets, the new population size R_i (checked against
//               the capacity) and the parent map parent[off_j + c] = j.
//   k_resample_small  the three stages above in one block, for capacities
//               of at most 4096 replicas.
//   k_finalize  Sec. 2 step 4 / Sec. 3 Eq. 4: population averages from exact
//               integer sums, the fluctuation-formula specific heat, the
//               magnetisation of Eq. 5, ln Z of Eq. 2 and the family entropy.
// All floating-point steps that feed a decision (S, rho, the rounding test)
// use explicitly rounded operations so that no multiply-add is contracted.
#include "pa_kernels.cuh"

namespace pa {

namespace {

constexpr int kBlock = 1024;

__global__ void k_init(uint32_t *spins, int32_t *anc, int q, int L, int R, uint32_t k0, uint32_t k1,
                       uint32_t stream_hi, int ground, uint32_t slot0)
{
    const long long total = (long long)R * (2 * colour_words(L));
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x)
        dev::init_item(spins, anc, q, L, i, k0, k1, stream_hi, ground, slot0);
}

__global__ void __launch_bounds__(kBlock) k_weights(const int32_t *hist, int nbins, double dbeta, const double *wtab,
                                                    DevState *st, int R_prev_all)
{
    __shared__ unsigned long long s_acc[dev::kSumLimbs];
    __shared__ long long s_l[32];
    dev::weights_body(hist, nbins, dbeta, wtab, st, s_acc, s_l, R_prev_all);
}

__global__ void __launch_bounds__(kBlock) k_counts(const int32_t *E, int twoN, int R_target, int mode, int step,
                                                   uint32_t stream_hi, uint32_t k0, uint32_t k1, const double *wtab,
                                                   int32_t *counts, int32_t *local_off, int32_t *blocksum,
                                                   DevState *st, int j0)
{
    __shared__ int s_i[32];
    dev::counts_body(blockIdx.x, E, twoN, R_target, mode, step, stream_hi, k0, k1, wtab, counts, local_off, blocksum,
                     st, s_i, j0);
}

__global__ void __launch_bounds__(kBlock) k_scatter(const int32_t *counts, const int32_t *local_off,
                                                    const int32_t *blocksum, int32_t *parent, int R_cap,
                                                    int32_t *hist_zero, int nbins, DevState *st, int min_total)
{
    __shared__ long long s_l[32];
    dev::scatter_body(blockIdx.x, gridDim.x, counts, local_off, blocksum, parent, R_cap, hist_zero, nbins, st, s_l,
                      min_total);
}

// Small populations (R_cap <= kSmallResample replicas): the three resampling
// stages in one block, one after the other, with the bodies of k_weights,
// k_counts and k_scatter run chunk by chunk.  Same arithmetic and the same
// results; two launches fewer per step where launch latency dominates.
constexpr int kSmallResample = 4 * kBlock;

__global__ void __launch_bounds__(kBlock) k_resample_small(const int32_t *hist, int nbins, const int32_t *E,
                                                           double dbeta, int R_target, int R_cap, int mode, int step,
                                                           uint32_t stream_hi, uint32_t k0, uint32_t k1,
                                                           const double *wtab, int32_t *counts, int32_t *local_off,
                                                           int32_t *blocksum, int32_t *parent, int32_t *hist_zero,
                                                           DevState *st, int j0, int R_prev_all)
{
    __shared__ unsigned long long s_acc[dev::kSumLimbs];
    __shared__ long long s_l[32];
    __shared__ int s_i[32];
    dev::weights_body(hist, nbins, dbeta, wtab, st, s_acc, s_l, R_prev_all);
    __syncthreads();
    const int nb = (R_cap + kBlock - 1) / kBlock;
    for (int chunk = 0; chunk < nb; ++chunk) {
        dev::counts_body(chunk, E, nbins - 1, R_target, mode, step, stream_hi, k0, k1, wtab, counts, local_off,
                         blocksum, st, s_i, j0);
        __syncthreads();
    }
    const int nb2 = nb > (nbins + kBlock - 1) / kBlock ? nb : (nbins + kBlock - 1) / kBlock;
    for (int chunk = 0; chunk < nb2; ++chunk) {
        dev::scatter_body(chunk, nb2, counts, local_off, blocksum, parent, R_cap, hist_zero, nbins, st, s_l,
                          R_prev_all > 0 ? 0 : 1);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kBlock) k_finalize(DevState *st, unsigned long long *acc, int32_t *fam, int R0,
                                                     DevObs *obs, double beta, int q, int N, int gathered,
                                                     int resampled, int R_all)
{
    __shared__ double s_d[32];
    __shared__ long long s_l[32];
    dev::finalize_body(st, acc, fam, R0, obs, beta, q, N, gathered, resampled, s_d, s_l, R_all);
}

// ---- One GPU's share of a population spread over several ----------------
// The children of the pending resample (c = 0..T-1 in new-slot order, parent
// map `parent`) go to destination rank d for c in [A_d, A_{d+1}).  Each rank
// sends, per destination, the runs of its children: a run is a maximal
// stretch of one destination's children with one parent, sent as that parent
// replica once with its child count, so a rank never sends more than its own
// replicas plus one per destination.

// Run heads: child c starts a run if it is a destination's first child or its
// parent differs from child c-1's.  Block-local exclusive scan of the heads
// (local_off[c] = -1 for children that are not heads).
__global__ void __launch_bounds__(kBlock) k_shard_heads(const int32_t *parent, int T, const int32_t *A, int G,
                                                        int32_t *local_off, int32_t *blocksum)
{
    __shared__ int s_i[32];
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    int head = 0;
    if (c < T) {
        int lo = 0, hi = G;  // the largest d with A_d <= c
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (A[mid] <= c) lo = mid; else hi = mid - 1;
        }
        head = (c == 0 || A[lo] == c || parent[c] != parent[c - 1]) ? 1 : 0;
    }
    int total;
    const int before = dev::block_exclusive_scan(head, s_i, &total);
    if (c < T) local_off[c] = head ? before : -1;
    if (threadIdx.x == 0) blocksum[blockIdx.x] = total;
}

// Entry index of each run: headpos[e] = its first child.
__global__ void __launch_bounds__(kBlock) k_shard_runs(int T, const int32_t *local_off, const int32_t *blocksum,
                                                       int32_t *headpos)
{
    __shared__ long long s_l[32];
    long long off = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += blockDim.x) off += blocksum[b];
    off = dev::block_sum_ll(off, s_l);
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < T && local_off[c] >= 0) headpos[off + local_off[c]] = c;
}

// ent_before[d] = runs before destination d's first child (d = 0..G; the
// last is the number of runs).
__global__ void k_shard_run_bounds(int T, const int32_t *A, int G, const int32_t *local_off, const int32_t *blocksum,
                                   long long *ent_before)
{
    for (int d = threadIdx.x; d <= G; d += blockDim.x) {
        const int pos = A[d];
        long long e = 0;
        const int nb = pos < T ? pos / kBlock : (T + kBlock - 1) / kBlock;
        for (int b = 0; b < nb; ++b) e += blocksum[b];
        if (pos < T) e += local_off[pos];  // a destination's first child is a head
        ent_before[d] = e;
    }
}

// Run e: its parent replica, family id and number of children.
__global__ void k_shard_pack(const uint32_t *spins, const int32_t *anc, const int32_t *parent, const int32_t *headpos,
                             int E, int T, int RW, uint32_t *send, int32_t *send_anc, int32_t *send_cnt)
{
    const int U = RW / 4;
    const long long total = (long long)E * U;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(i / U), o = (int)(i - (long long)e * U);
        const int c = headpos[e];
        const int p = parent[c];
        reinterpret_cast<uint4 *>(send + (size_t)e * RW)[o] = reinterpret_cast<const uint4 *>(spins + (size_t)p * RW)[o];
        if (o == 0) {
            send_cnt[e] = (e + 1 < E ? headpos[e + 1] : T) - c;
            if (send_anc) send_anc[e] = anc[p];
        }
    }
}

// The received runs become the parents of this rank's new population: the
// buffer they arrived in becomes the current one (the next sweep gathers
// from it) and the run counts are scanned into a parent map by k_scatter.
__global__ void k_shard_accept(DevState *st, int n_runs)
{
    if (threadIdx.x == 0 && blockIdx.x == 0 && !st->err) {
        st->pop = n_runs;
        st->parity ^= 1;
    }
}

__global__ void __launch_bounds__(kBlock) k_shard_run_scan(const int32_t *cnt, int n, int32_t *local_off,
                                                           int32_t *blocksum)
{
    __shared__ int s_i[32];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = j < n ? cnt[j] : 0;
    int total;
    const int before = dev::block_exclusive_scan(r, s_i, &total);
    if (j < n) local_off[j] = before;
    if (threadIdx.x == 0) blocksum[blockIdx.x] = total;
}

// The new local size must be the plan's: anything else means an exchange
// that did not deliver what the plan placed here.
__global__ void k_shard_check(DevState *st, int expected)
{
    if (threadIdx.x == 0 && blockIdx.x == 0 && !st->err && st->pop_next != expected) st->err = 1;  // PA_ERR_INVALID
}

__global__ void k_to_canonical(const uint32_t *spins, uint8_t *out, int q, int L, long long count)
{
    const long long total = count * L * L;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = dev::canonical_state(spins, q, L, i);
}

__global__ void k_from_canonical(uint32_t *spins, const uint8_t *canon, int q, int L, long long count)
{
    const long long total = count * (2 * colour_words(L));
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x)
        dev::from_canonical_item(spins, canon, q, L, i);
}

int grid_for(long long work, int threads)
{
    long long g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 65535LL * 16) g = 65535LL * 16;
    return (int)g;
}

}  // namespace

cudaError_t launch_init(uint32_t *spins, int32_t *anc, int q, int L, int R, uint32_t k0, uint32_t k1,
                        uint32_t stream_hi, int ground, cudaStream_t s, uint32_t slot0)
{
    const long long work = (long long)R * (2 * colour_words(L));
    k_init<<<grid_for(work, 256), 256, 0, s>>>(spins, anc, q, L, R, k0, k1, stream_hi, ground, slot0);
    bump_launch_count(1);
    return cudaGetLastError();
}

cudaError_t launch_resample(const int32_t *hist, int nbins, const int32_t *E, double dbeta, int R_target,
                            int R_cap, int mode, int step, uint32_t stream_hi, uint32_t k0, uint32_t k1,
                            const double *wtab, int32_t *counts, int32_t *local_off, int32_t *blocksum,
                            int32_t *parent, int32_t *hist_zero, DevState *st, cudaStream_t s, int j0,
                            int R_prev_all)
{
    if (R_cap <= kSmallResample) {
        k_resample_small<<<1, kBlock, 0, s>>>(hist, nbins, E, dbeta, R_target, R_cap, mode, step, stream_hi, k0, k1,
                                              wtab, counts, local_off, blocksum, parent, hist_zero, st, j0,
                                              R_prev_all);
        bump_launch_count(1);
        return cudaGetLastError();
    }
    const int nb = (R_cap + kBlock - 1) / kBlock;
    k_weights<<<1, kBlock, 0, s>>>(hist, nbins, dbeta, wtab, st, R_prev_all);
    k_counts<<<nb, kBlock, 0, s>>>(E, nbins - 1, R_target, mode, step, stream_hi, k0, k1, wtab, counts, local_off,
                                   blocksum, st, j0);
    const int nb2 = nb > (nbins + kBlock - 1) / kBlock ? nb : (nbins + kBlock - 1) / kBlock;
    k_scatter<<<nb2, kBlock, 0, s>>>(counts, local_off, blocksum, parent, R_cap, hist_zero, nbins, st,
                                     R_prev_all > 0 ? 0 : 1);
    bump_launch_count(3);
    return cudaGetLastError();
}

cudaError_t launch_finalize(DevState *st, unsigned long long *acc, int32_t *fam, int R0, DevObs *obs,
                            double beta, int q, int N, int gathered, int resampled, cudaStream_t s, int R_all)
{
    k_finalize<<<1, kBlock, 0, s>>>(st, acc, fam, R0, obs, beta, q, N, gathered, resampled, R_all);
    bump_launch_count(1);
    return cudaGetLastError();
}

cudaError_t launch_to_canonical(const uint32_t *spins, uint8_t *out, int q, int L, int64_t count, cudaStream_t s)
{
    k_to_canonical<<<grid_for(count * L * L, 256), 256, 0, s>>>(spins, out, q, L, count);
    bump_launch_count(1);
    return cudaGetLastError();
}

cudaError_t launch_from_canonical(uint32_t *spins, const uint8_t *canon, int q, int L, int64_t count,
                                  cudaStream_t s)
{
    k_from_canonical<<<grid_for(count * 2 * colour_words(L), 256), 256, 0, s>>>(spins, canon, q, L, count);
    bump_launch_count(1);
    return cudaGetLastError();
}

cudaError_t launch_shard_runs(const int32_t *parent, int T, const int32_t *A, int G, int32_t *local_off,
                             int32_t *blocksum, int32_t *headpos, long long *ent_before, cudaStream_t s)
{
    const int nb = (T + kBlock - 1) / kBlock;
    if (nb > 0) {
        k_shard_heads<<<nb, kBlock, 0, s>>>(parent, T, A, G, local_off, blocksum);
        k_shard_runs<<<nb, kBlock, 0, s>>>(T, local_off, blocksum, headpos);
        bump_launch_count(2);
    }
    k_shard_run_bounds<<<1, 256, 0, s>>>(T, A, G, local_off, blocksum, ent_before);
    bump_launch_count(1);
    return cudaGetLastError();
}

cudaError_t launch_shard_pack(const uint32_t *spins, const int32_t *anc, const int32_t *parent,
                             const int32_t *headpos, int E, int T, int RW, uint32_t *send, int32_t *send_anc,
                             int32_t *send_cnt, cudaStream_t s)
{
    if (E <= 0) return cudaSuccess;
    k_shard_pack<<<grid_for((long long)E * (RW / 4), 256), 256, 0, s>>>(spins, anc, parent, headpos, E, T, RW, send,
                                                                        send_anc, send_cnt);
    bump_launch_count(1);
    return cudaGetLastError();
}

cudaError_t launch_shard_accept(DevState *st, const int32_t *recv_cnt, int n_runs, int n_expected, int R_cap,
                               int32_t *local_off, int32_t *blocksum, int32_t *parent, int32_t *hist_zero,
                               int nbins, cudaStream_t s)
{
    k_shard_accept<<<1, 32, 0, s>>>(st, n_runs);
    const int nb = (n_runs + kBlock - 1) / kBlock;
    if (nb > 0) k_shard_run_scan<<<nb, kBlock, 0, s>>>(recv_cnt, n_runs, local_off, blocksum);
    k_scatter<<<nb > 0 ? nb : 1, kBlock, 0, s>>>(recv_cnt, local_off, blocksum, parent, R_cap, hist_zero, nbins, st,
                                                 0);
    k_shard_check<<<1, 32, 0, s>>>(st, n_expected);
    bump_launch_count(nb > 0 ? 4 : 3);
    return cudaGetLastError();
}

}  // namespace pa
