// pa_internal.cuh -- device helpers and host<->device structures shared by the
// translation units of the GB300 population-annealing library.
//
// Device layout of one replica (multi-spin coding).  A state 0..q-1 takes
// B = ceil(log2 q) bits.  The sites of colour c = (x + y) & 1, with column index
// m = x >> 1, are packed 32 to a "site word", stored as BP 32-bit planes (BP = B
// rounded up to 1, 2 or 4 for B <= 4, else B; plane p holds bit p of the states):
//   word index (c * IPC + w) * BP + p,   IPC = site words per colour.
// When L/2 divides 32 (L = 8, 16, 32, 64) the colour's sites in row-major order
// h = y L/2 + m fill the words in turn (w = h >> 5, bit h & 31; IPC = L^2/64).
// When L is a multiple of 16 but not of 64 and L > 32 (L = 48, 80, 96, ...)
// the rows form four bands of L/4 rows and each row L/16 segments of 8
// columns: word w = k L/16 + j holds segment j of rows k + a L/4, a = 0..3,
// the site of band a and column m = 8j + t at bit 8a + t (IPC = L^2/64).
// Otherwise each row starts a new word: w = y WPR + (m >> 5), bit m & 31,
// WPR = ceil(L / 64), IPC = L WPR, and columns >= L/2 of a row's last word are
// always zero.  Planes >= B are always zero.  One replica takes RW = 2 IPC BP
// words, rounded up to a multiple of 4; replica s starts at word s * RW.  The four neighbours of
// a site word are words of the other colour (rows above and below, the same
// row, and that row shifted by one column), so one 32-bit logic instruction
// serves 32 sites.  The canonical [y][x] byte layout exists only at the API
// boundary (pa_get_spins).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

// Checked builds (-DPA_CHECKED=1; build.build(checked=True) makes
// libpa_gb300_checked.so): the kernels test the indices they take from device
// data -- a gather's parent slot, a replica's energy bin -- before using them;
// a failed test sets the run's error flag to PA_ERR_INVALID (1) and skips the
// access, so the host call reports it and no access leaves its array.  Off by
// default: the tests cost instructions on the hot path.
#ifndef PA_CHECKED
#define PA_CHECKED 0
#endif

namespace pa {

// Top two bits of the second Philox counter word separate the uses of the
// generator (initial spins, sweeps, copy numbers, ground states).
constexpr uint32_t DOM_SWEEP = 0x00000000u;
constexpr uint32_t DOM_INIT = 0x40000000u;
constexpr uint32_t DOM_RESAMPLE = 0x80000000u;
constexpr uint32_t DOM_GROUND = 0xC0000000u;

// Sweeps per temperature step: 2k + colour must fit below the domain tag of
// the counter word in which it is shifted left by 8.
constexpr int kMaxTheta = 1 << 21;

// Largest replica (bytes of its bit planes) a sweep block keeps in shared
// memory, leaving room for the threshold table and reductions within 227 KB.
constexpr int kMaxLatticeBytes = 200 * 1024;

// Bits per state, planes stored per site word, words per row of one colour,
// words per replica (see the layout above).
__host__ __device__ constexpr int state_bits(int q) { return q <= 2 ? 1 : q <= 4 ? 2 : q <= 8 ? 3 : q <= 16 ? 4 : q <= 32 ? 5 : q <= 64 ? 6 : 7; }
__host__ __device__ constexpr int plane_stride(int B) { return B <= 1 ? 1 : B <= 2 ? 2 : B <= 4 ? 4 : B; }
__host__ __device__ constexpr int row_words(int L) { return (L + 63) / 64; }
// Rows packed several to a word: L/2 divides 32 (L = 8, 16, 32; at L = 64 both
// layouts coincide).
__host__ __device__ constexpr bool rows_packed(int L) { return L >= 8 && 64 % L == 0; }
// Rows in four bands of 8-column segments: L = 48, 80, 96, 112, 144, ...
__host__ __device__ constexpr bool rows_banded(int L) { return L > 32 && L % 16 == 0 && L % 64 != 0; }
__host__ __device__ constexpr int colour_words(int L)
{
    return (rows_packed(L) || rows_banded(L)) ? L * L / 64 : L * row_words(L);
}
// Words of one replica, padded to whole 16-byte vectors (the gather moves uint4).
__host__ __device__ constexpr int replica_words_of(int B, int L) { return (2 * colour_words(L) * plane_stride(B) + 3) & ~3; }
__host__ __device__ constexpr int replica_words(int q, int L) { return replica_words_of(state_bits(q), L); }
inline size_t replica_bytes(int q, int L) { return (size_t)replica_words(q, L) * 4; }

// Acceptance thresholds T[d] = floor(exp(-beta d) 2^32), d = 1..4, as the low 32
// bits plus a flag for T[d] = 2^32 (beta = 0), computed on the host with libm.
struct Thresholds {
    uint32_t T[4];
    uint32_t full;  // bit d-1 set where T[d] = 2^32
};

// Device-resident run state.  Kernels read and update it so that a whole
// schedule can be enqueued (or captured in a graph) with no host round trip.
struct DevState {
    int32_t pop;       // current population size R_i
    int32_t pop_next;  // size after the pending resample
    int32_t err;       // 0, or a pa_status code set by a kernel
    int32_t parity;    // spin / ancestor buffer holding the current population
    int32_t E_ref;     // reference energy of the pending resample
    int32_t ties;      // copy numbers of the pending resample flagged as near ties
    double S;          // sum of shifted Boltzmann factors of the pending resample
    double lnQ;        // ln Q of the pending resample
    double lnZ;        // running ln Z (Eq. 2)
};

// Per-step estimators; field order matches pa_obs in include/pa.h.
struct DevObs {
    double beta, lnQ, lnZ, meanE, meanE2, C, meanM, S_f;
    int64_t R, n_families, sumE, sumE2, sumMt, n_near_ties;
};

struct SweepArgs {
    uint32_t *buf[2];          // spin double buffer (layout above)
    int32_t *anc[2];           // ancestor double buffer (null: no families)
    const int32_t *parent;     // parent map of the pending resample (null: in place)
    int32_t *E;                // per-replica energies
    int32_t *Mt;               // per-replica occupation of the most common state
    int32_t *hist;             // energy histogram, bin E + 2N
    unsigned long long *acc;   // [3] running sums of E, E^2, Mt (two's complement)
    int32_t *fam;              // family counts (null: no families)
    DevState *st;
    Thresholds thr;            // acceptance thresholds
    uint32_t k0, k1;           // Philox key (seed low / high word)
    uint32_t rk0[10], rk1[10]; // Philox round keys k + r * (Weyl constant), r = 0..9
    int32_t q, L, theta, step;
    int32_t rpb;               // replicas per block iteration
    int32_t gather;            // 1: read parents from buf[parity], write buf[parity^1]
    uint32_t stream_hi;        // stream number << 24 (top byte of the slot counter word)
    uint32_t slot0;            // global slot of local slot 0 (0 unless the population spans GPUs)
    int32_t *work;             // next replica group to hand out (zeroed before each launch), or
                               // null: each block takes an equal share
};

// Launchers (pa_sweep.cu)
cudaError_t launch_sweep(const SweepArgs &a, int threads, int grid, cudaStream_t s);
size_t sweep_smem_bytes(int q, int L, int rpb);
int sweep_max_blocks_per_sm(int q, int L, int rpb, int threads);

// Launchers (pa_resample.cu)
// slot0: global slot of local slot 0 (random keys and family ids follow it).
cudaError_t launch_init(uint32_t *spins, int32_t *anc, int q, int L, int R, uint32_t k0, uint32_t k1,
                        uint32_t stream_hi, int ground, cudaStream_t s, uint32_t slot0 = 0u);
// wtab: the weight table of dbeta (weight_table below), 2N + 1 entries.
// j0 / R_prev_all: global index of local replica 0 and the size of the whole
// population when it spans several GPUs (0, 0 otherwise).
cudaError_t launch_resample(const int32_t *hist, int nbins, const int32_t *E, double dbeta, int R_target,
                            int R_cap, int mode, int step, uint32_t stream_hi, uint32_t k0, uint32_t k1,
                            const double *wtab, int32_t *counts, int32_t *local_off, int32_t *blocksum,
                            int32_t *parent, int32_t *hist_zero, DevState *st, cudaStream_t s, int j0 = 0,
                            int R_prev_all = 0);
// R_all: size of the whole population when the sums cover several GPUs (0 otherwise).
cudaError_t launch_finalize(DevState *st, unsigned long long *acc, int32_t *fam, int R0, DevObs *obs,
                            double beta, int q, int N, int gathered, int resampled, cudaStream_t s, int R_all = 0);
// A population spread over several GPUs.  The T children of the pending
// resample (parent map, new-slot order) go to destination d for c in
// [A[d], A[d+1]); runs of one destination's children with one parent become
// entries (headpos[e] = the run's first child, ent_before[d] = entries before
// destination d); the pack copies each run's parent replica, family id and
// child count into the send buffers.  Accepting the received runs makes their
// buffer current and scans their counts into the parent map of the next
// (gathering) sweep; the new size must equal n_expected.
cudaError_t launch_shard_runs(const int32_t *parent, int T, const int32_t *A, int G, int32_t *local_off,
                             int32_t *blocksum, int32_t *headpos, long long *ent_before, cudaStream_t s);
cudaError_t launch_shard_pack(const uint32_t *spins, const int32_t *anc, const int32_t *parent,
                             const int32_t *headpos, int E, int T, int RW, uint32_t *send, int32_t *send_anc,
                             int32_t *send_cnt, cudaStream_t s);
cudaError_t launch_shard_accept(DevState *st, const int32_t *recv_cnt, int n_runs, int n_expected, int R_cap,
                               int32_t *local_off, int32_t *blocksum, int32_t *parent, int32_t *hist_zero,
                               int nbins, cudaStream_t s);
cudaError_t launch_to_canonical(const uint32_t *spins, uint8_t *out, int q, int L, int64_t count,
                                cudaStream_t s);
// The inverse: count replicas [count][L][L] (one byte per spin) into the layout above.
cudaError_t launch_from_canonical(uint32_t *spins, const uint8_t *canon, int q, int L, int64_t count,
                                  cudaStream_t s);

// Host: the thresholds of inverse temperature beta.
Thresholds acceptance_thresholds(double beta);

// Host: the Boltzmann factors of a resampling step dbeta by energy distance
// t = |E - E_ref| from the reference energy, t = 0..n-1:
// out[t] = exp(-dbeta d) with d = t (dbeta >= 0, E_ref the lowest energy) or
// d = -t (dbeta < 0, E_ref the highest), using the C library's exp, so the
// factors do not depend on the device.
void weight_table(double dbeta, int n, double *out);

// Launchers (pa_reweight.cu)
cudaError_t launch_newton(const int32_t *hist, int nbins, const DevState *st, double target, double cap, int iters,
                          double *out, cudaStream_t s);

int64_t bump_launch_count(int64_t n);

// Records the message returned by pa_last_cuda_error() on this thread.
void record_cuda_error(const char *msg);

}  // namespace pa

namespace pa {

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 32x32 -> 64 bit products whose high halves are xored with the other counter
// words and the round key; the key advances by the Weyl constants each round.
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// The same generator with its ten round keys supplied by the caller (kernel
// parameters), so no key arithmetic runs per call.
__device__ __forceinline__ uint4 philox10_rk(uint4 c, const uint32_t *rk0, const uint32_t *rk1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk0[round], (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ rk1[round], (uint32_t)p0);
    }
    return c;
}

__device__ __forceinline__ uint32_t pick_word(const uint4 &w, int i)
{
    return i == 0 ? w.x : i == 1 ? w.y : i == 2 ? w.z : w.w;
}

}  // namespace pa
