// pa_capi.cu -- host runtime and C ABI (include/pa.h) of the GB300
// population-annealing library (Barash, Weigel, Shchur & Janke,
// arXiv:1704.01888, Sec. 2 steps 1-5).
//
// A pa_ctx owns the device buffers of one PA run and enqueues its kernels on
// one stream.  The run state that kernels need (population size, buffer
// parity, pending normaliser, ln Z, error flag) lives in device memory, so a
// whole temperature schedule can be enqueued or captured as one CUDA graph
// without host round trips.  The host computes only the per-beta acceptance
// thresholds (four 32-bit integers, passed as kernel arguments), using the C
// library's exp so that they are reproducible bit for bit on the host.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/pa.h"
#include "pa_internal.cuh"
#include "pa_trace.h"

namespace pa {

static std::atomic<long long> g_launches{0};

int64_t bump_launch_count(int64_t n) { return g_launches.fetch_add(n) + n; }

static thread_local std::string t_cuda_error;

void record_cuda_error(const char *msg) { t_cuda_error = msg; }

Thresholds acceptance_thresholds(double beta)
{
    Thresholds th{};
    for (int d = 1; d <= 4; ++d) {
        const uint64_t T = (uint64_t)(std::exp(-beta * (double)d) * 4294967296.0);
        if (T >= 4294967296ull) {
            th.full |= 1u << (d - 1);
            th.T[d - 1] = 0u;
        } else {
            th.T[d - 1] = (uint32_t)T;
        }
    }
    return th;
}

void weight_table(double dbeta, int n, double *out)
{
    for (int t = 0; t < n; ++t) {
        const double d = dbeta >= 0.0 ? (double)t : -(double)t;
        out[t] = std::exp(-dbeta * d);
    }
}

}  // namespace pa

namespace {

using pa::t_cuda_error;

pa_status cuda_fail(cudaError_t e)
{
    t_cuda_error = cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PA_ERR_NOMEM : PA_ERR_CUDA;
}

#define PA_CK(expr)                                   \
    do {                                              \
        cudaError_t pa_e_ = (expr);                   \
        if (pa_e_ != cudaSuccess) return cuda_fail(pa_e_); \
    } while (0)

}  // namespace

struct pa_ctx {
    pa_config cfg{};
    int N = 0, nbins = 0, R_cap = 0;
    cudaStream_t stream = nullptr;
    uint32_t k0 = 0, k1 = 0;
    int sms = 0;

    uint32_t *spins[2] = {nullptr, nullptr};  // multi-spin-coded populations
    int32_t *anc[2] = {nullptr, nullptr};
    int32_t *E = nullptr, *Mt = nullptr, *hist = nullptr, *fam = nullptr;
    int32_t *counts = nullptr, *local_off = nullptr, *blocksum = nullptr, *parent = nullptr;
    // Weight tables of the resampling steps (pa::weight_table), one per
    // distinct dbeta, in a device arena of kWTableSlots tables reused least
    // recently used first; a constant schedule has a handful of distinct
    // steps, so each table is computed once.  A new table is computed on the
    // host into one of kWStage pinned staging slots and uploaded on the
    // context's stream, which orders the upload after every earlier reader of
    // the arena slot it overwrites.
    double *wt_arena = nullptr;                 // device, kWTableSlots x nbins
    double *wt_stage = nullptr;                 // pinned host, kWStage x nbins
    std::vector<cudaEvent_t> wt_stage_done;     // upload from each staging slot done
    std::vector<uint64_t> wt_key;               // dbeta bits held by each arena slot
    std::vector<long long> wt_stamp;            // last use (0: empty)
    long long wt_clock = 0;
    int wt_next_stage = 0;
    double *wt_run = nullptr;                   // tables of a long pa_run schedule
    std::vector<std::pair<uint64_t, const double *>> wt_run_at;
    bool resampled = false;  // parent holds the map of a resample
    unsigned long long *acc = nullptr;
    pa::DevState *st = nullptr;
    pa::DevObs *obs = nullptr;
    int obs_cap = 0;
    long long n_obs = 0;  // estimator records written so far
    uint8_t *stage = nullptr;
    size_t stage_bytes = 0;
    uint8_t *host_stage = nullptr;  // pinned: device state, one record, the histogram
    double *aux = nullptr;  // small device outputs (Newton step)
    int32_t *work = nullptr;  // the sweep kernel's group counter

    int step = 0;          // last completed temperature step
    int pending_step = 0;  // step of an enqueued resample awaiting its sweep
    double beta = 0.0;     // inverse temperature of the current population
    bool failed = false;

    int rpb = 1, threads = 32, grid = 1;

    // A population spread over several GPUs (pa_shard_init): this context
    // holds the global slots [slot0, slot0 + R_i(local)) of one population of
    // R_all replicas; the caller sums the histogram, the integer sums and the
    // family counts over the ranks and exchanges the children between steps.
    bool shard = false;
    int rank = 0, world = 1;
    int R_fill = 0;           // replicas the launch shape is sized for (R, or R / world)
    int slot0 = 0, R_all = 0; // current population
    int slot0_next = 0, n_next = 0, R_all_next = 0, n_pack = 0;
    int host_parity = 0;      // buffer holding the current population (the device's parity)
    int shard_stage = 0;      // kShard* below
    bool shard_resampled = false;
    uint32_t *send = nullptr;   // runs sent to other ranks: parent replicas,
    int32_t *send_anc = nullptr; // their family ids
    int32_t *send_cnt = nullptr; // and child counts
    int32_t *recv_cnt = nullptr; // child counts of the runs received
    int32_t *headpos = nullptr;  // first child of each run
    int32_t *bounds = nullptr;   // [world + 1] destination bounds in child order
    long long *ent_before = nullptr; // [world + 1] runs before each destination
    int n_runs = 0;
    cudaStream_t capture_stream = nullptr;  // private stream for graph capture

    // event timing (pa_profile)
    bool profiling = false;
    std::vector<cudaEvent_t> ev[2];  // start/stop pairs per category
    int64_t ev_used[2] = {0, 0};
};

namespace {

template <typename T>
pa_status dev_alloc(T **p, size_t count)
{
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e);
    }
    return PA_OK;
}

void release_events(pa_ctx *c)
{
    for (int k = 0; k < 2; ++k) {
        for (cudaEvent_t e : c->ev[k]) cudaEventDestroy(e);
        c->ev[k].clear();
        c->ev_used[k] = 0;
    }
}

// Records the start (first = true) or stop event of category k.
pa_status profile_mark(pa_ctx *c, int k, bool first)
{
    if (!c->profiling) return PA_OK;
    const size_t idx = (size_t)(first ? 2 * c->ev_used[k] : 2 * c->ev_used[k] + 1);
    while (c->ev[k].size() <= idx) {
        cudaEvent_t e;
        PA_CK(cudaEventCreate(&e));
        c->ev[k].push_back(e);
    }
    PA_CK(cudaEventRecord(c->ev[k][idx], c->stream));
    if (!first) c->ev_used[k] += 1;
    return PA_OK;
}

constexpr int kWTableSlots = 32;
constexpr int kWStage = 4;

// Device arena and pinned staging of the weight tables (at context creation).
pa_status alloc_wtables(pa_ctx *c)
{
    const size_t n = (size_t)c->nbins;
    pa_status s = dev_alloc(&c->wt_arena, n * kWTableSlots);
    if (s) return s;
    cudaError_t e = cudaHostAlloc((void **)&c->wt_stage, sizeof(double) * n * kWStage, cudaHostAllocDefault);
    if (e != cudaSuccess) {
        c->wt_stage = nullptr;
        return cuda_fail(e);
    }
    c->wt_stage_done.assign(kWStage, nullptr);
    for (cudaEvent_t &ev : c->wt_stage_done)
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e);
    c->wt_key.assign(kWTableSlots, 0);
    c->wt_stamp.assign(kWTableSlots, 0);
    return PA_OK;
}

void release_wtables(pa_ctx *c)
{
    for (cudaEvent_t ev : c->wt_stage_done)
        if (ev) cudaEventDestroy(ev);
    c->wt_stage_done.clear();
    if (c->wt_arena) cudaFree(c->wt_arena);
    if (c->wt_stage) cudaFreeHost(c->wt_stage);
    if (c->wt_run) cudaFree(c->wt_run);
    c->wt_arena = c->wt_run = nullptr;
    c->wt_stage = nullptr;
}

// Frees the tables of a long pa_run schedule (after its work has finished).
void release_run_tables(pa_ctx *c)
{
    if (c->wt_run) cudaFree(c->wt_run);
    c->wt_run = nullptr;
    c->wt_run_at.clear();
}

// The device weight table of dbeta: a schedule's own tables during a long
// pa_run, else the arena slot holding it, else a new table in the least
// recently used slot.
pa_status get_wtable(pa_ctx *c, double dbeta, const double **out)
{
    uint64_t key;
    std::memcpy(&key, &dbeta, sizeof(key));
    for (const auto &kv : c->wt_run_at) {
        if (kv.first == key) {
            *out = kv.second;
            return PA_OK;
        }
    }
    const size_t n = (size_t)c->nbins;
    int slot = 0;
    for (int i = 0; i < kWTableSlots; ++i) {
        if (c->wt_stamp[i] && c->wt_key[i] == key) {
            c->wt_stamp[i] = ++c->wt_clock;
            *out = c->wt_arena + n * i;
            return PA_OK;
        }
        if (c->wt_stamp[i] < c->wt_stamp[slot]) slot = i;
    }
    const int k = c->wt_next_stage;
    c->wt_next_stage = (k + 1) % kWStage;
    double *host = c->wt_stage + n * k;
    PA_CK(cudaEventSynchronize(c->wt_stage_done[k]));  // its previous upload has left
    pa::weight_table(dbeta, c->nbins, host);
    double *dev = c->wt_arena + n * slot;
    PA_CK(cudaMemcpyAsync(dev, host, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    PA_CK(cudaEventRecord(c->wt_stage_done[k], c->stream));
    c->wt_key[slot] = key;
    c->wt_stamp[slot] = ++c->wt_clock;
    *out = dev;
    return PA_OK;
}

// Steps of a shard's temperature step, in order.
enum { kShardMeasured = 1, kShardReady = 2, kShardCounted = 3, kShardPacked = 4, kShardAccepted = 5 };

void release(pa_ctx *c)
{
    release_events(c);
    release_wtables(c);
    void *shard_bufs[] = {c->send, c->send_anc, c->send_cnt, c->recv_cnt, c->headpos, c->bounds, c->ent_before};
    for (void *p : shard_bufs)
        if (p) cudaFree(p);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    void *ptrs[] = {c->spins[0], c->spins[1], c->anc[0], c->anc[1], c->E, c->Mt, c->hist, c->fam,
                    c->counts, c->local_off, c->blocksum, c->parent, c->acc, c->st, c->obs,
                    c->stage, c->aux, c->work};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->host_stage) cudaFreeHost(c->host_stage);
}

// Offsets in the pinned host staging area of pa_observables.
constexpr size_t kStageObs = 256;
constexpr size_t kStageHist = 512;
static_assert(sizeof(pa::DevState) <= kStageObs && sizeof(pa_obs) <= kStageHist - kStageObs, "staging layout");

pa_status choose_launch(pa_ctx *c, int rpb_req, int threads_req)
{
    const int L = c->cfg.L;
    const size_t RB = pa::replica_bytes(c->cfg.q, L);
    // work items per replica and half sweep: the site words of one colour
    const long long units = pa::colour_words(L);
    int rpb = rpb_req;
    int threads = threads_req;
    if (rpb <= 0 && threads <= 0 && (units == 1024 || units == 256) && pa::state_bits(c->cfg.q) <= 5 &&
        c->R_fill / (4 * c->sms) >= 4) {
        // 1024 or 256 site words per colour (L = 256, 128): blocks of 1024
        // threads, each keeping one site word index through all passes, with
        // as many lattices as fit in whole passes (L = 256, q = 20: five, 1439
        // against 1339 attempts/ns with two lattices and 512 threads; q = 6:
        // 1855 against 1731; q = 10 even.  L = 128: q = 20 1411 against 1243,
        // q = 8 1952 against 1919, q = 5 1857 against 1829, q = 10 even.  With
        // six or seven planes the 1024-thread blocks are slower)
        const int per_pass = (int)(1024 / units);
        rpb = (int)((size_t)pa::kMaxLatticeBytes / RB) / per_pass * per_pass;
        threads = 1024;
    }
    if (rpb <= 0) {
        // 96 KB of lattices per block: two blocks of 512 threads per SM
        int rpb_mem = (int)(98304 / RB);
        if (rpb_mem < 1) rpb_mem = 1;
        int rpb_fill = c->R_fill / (4 * c->sms);
        if (rpb_fill < 1) rpb_fill = 1;
        rpb = rpb_mem < rpb_fill ? rpb_mem : rpb_fill;
        // a group spanning several passes of 512 threads over its site words
        // fills each pass: q = 10, L = 64 takes 48 replicas (6 words per
        // thread), not 44 (5.5)
        const long long per_pass = 512 / units;
        if (per_pass >= 1 && rpb > per_pass) rpb = (int)(rpb / per_pass * per_pass);
        // at least one warp of work items per block
        const int rpb_warp = (int)((32 + units - 1) / units);
        if (rpb < rpb_warp) rpb = rpb_warp < rpb_mem ? rpb_warp : rpb_mem;
    }
    if ((size_t)rpb * RB > (size_t)pa::kMaxLatticeBytes) return rpb == 1 ? PA_ERR_TOO_LARGE : PA_ERR_INVALID;
    if (threads <= 0) {
        // one thread per site word, at most 512; a block that holds a single
        // large replica takes about four words per thread instead (measured
        // best at q = 20, L = 256: fewer words per thread leave the barriers
        // and the queue pass of each half sweep poorly amortised)
        const long long work = (long long)rpb * units;
        const long long per_thread = rpb == 1 ? 4 : 1;
        threads = (int)(((work + per_thread - 1) / per_thread + 31) / 32 * 32);
        if (threads > 512) threads = 512;
        if (threads < 32) threads = 32;
    }
    if (threads % 32 != 0 || threads > 1024) return PA_ERR_INVALID;
    const int per_sm = pa::sweep_max_blocks_per_sm(c->cfg.q, L, rpb, threads);
    if (per_sm <= 0) return PA_ERR_INVALID;
    const long long groups = ((long long)c->R_cap + rpb - 1) / rpb;
    long long grid = (long long)per_sm * c->sms;
    if (grid > groups) grid = groups;
    c->rpb = rpb;
    c->threads = threads;
    c->grid = (int)grid;
    return PA_OK;
}

pa::SweepArgs sweep_args(pa_ctx *c, double beta, int theta, int step, int gather)
{
    pa::SweepArgs a{};
    a.buf[0] = c->spins[0];
    a.buf[1] = c->spins[1];
    a.anc[0] = c->anc[0];
    a.anc[1] = c->anc[1];
    a.parent = c->parent;
    a.E = c->E;
    a.Mt = c->Mt;
    a.hist = c->hist;
    a.acc = c->acc;
    a.fam = c->cfg.track_families ? c->fam : nullptr;
    a.st = c->st;
    a.thr = pa::acceptance_thresholds(beta);
    a.k0 = c->k0;
    a.k1 = c->k1;
    for (int r = 0; r < 10; ++r) {
        a.rk0[r] = c->k0 + 0x9E3779B9u * (uint32_t)r;
        a.rk1[r] = c->k1 + 0xBB67AE85u * (uint32_t)r;
    }
    a.q = c->cfg.q;
    a.L = c->cfg.L;
    a.theta = theta;
    a.step = step;
    a.rpb = c->rpb;
    a.gather = gather;
    a.stream_hi = (uint32_t)c->cfg.stream << 24;
    a.slot0 = (uint32_t)c->slot0;
    // few groups per block: hand them out from a counter, so that the blocks
    // end together; with many, equal shares (their ends even out)
    const long long R_est = c->R_fill > 0 ? c->R_fill : c->cfg.R;
    a.work = R_est < 16LL * c->rpb * c->grid ? c->work : nullptr;
    return a;
}

pa::DevObs *next_obs_slot(pa_ctx *c)
{
    pa::DevObs *slot = c->obs + (c->n_obs % c->obs_cap);
    c->n_obs += 1;
    return slot;
}

// Enqueues theta sweeps (with the pending gather, if any) and the estimators.
pa_status enqueue_sweep(pa_ctx *c, double beta, int theta, int step)
{
    const int gather = c->pending_step != 0;
    pa::SweepArgs a = sweep_args(c, beta, theta, step, gather);
    pa_status s = profile_mark(c, 0, true);
    if (s) return s;
    PA_CK(pa::launch_sweep(a, c->threads, c->grid, c->stream));
    if ((s = profile_mark(c, 0, false))) return s;
    if (!c->shard)
        PA_CK(pa::launch_finalize(c->st, c->acc, a.fam, c->cfg.R, next_obs_slot(c), beta, c->cfg.q, c->N,
                                  gather, gather, c->stream));
    c->pending_step = 0;
    c->step = step;
    c->beta = beta;
    return PA_OK;
}

pa_status enqueue_resample(pa_ctx *c, double dbeta, int step)
{
    const double *wtab = nullptr;
    pa_status s = get_wtable(c, dbeta, &wtab);
    if (s) return s;
    if ((s = profile_mark(c, 1, true))) return s;
    PA_CK(pa::launch_resample(c->hist, c->nbins, c->E, dbeta, c->cfg.R, c->R_cap, c->cfg.resample_mode, step,
                              (uint32_t)c->cfg.stream << 24, c->k0, c->k1, wtab, c->counts, c->local_off,
                              c->blocksum, c->parent, c->hist, c->st, c->stream));
    if ((s = profile_mark(c, 1, false))) return s;
    c->pending_step = step;
    c->resampled = true;
    return PA_OK;
}

// Reads the device state after synchronising; maps a kernel-raised error.
pa_status sync_state(pa_ctx *c, pa::DevState *out)
{
    pa::DevState h;
    PA_CK(cudaMemcpyAsync(&h, c->st, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    PA_CK(cudaStreamSynchronize(c->stream));
    if (out) *out = h;
    if (h.err != 0) {
        c->failed = true;
        return (pa_status)h.err;
    }
    return PA_OK;
}

}  // namespace

extern "C" {

const char *pa_status_str(pa_status s)
{
    switch (s) {
    case PA_OK: return "ok";
    case PA_ERR_INVALID: return "invalid argument";
    case PA_ERR_CAPACITY: return "population exceeds capacity";
    case PA_ERR_CUDA: return "CUDA error";
    case PA_ERR_TIMEOUT: return "device wait timed out";
    case PA_ERR_STATE: return "call out of order or context failed";
    case PA_ERR_NOMEM: return "out of memory";
    case PA_ERR_TOO_LARGE: return "size exceeds shared memory (lattice) or fixed working memory (no-allocation call)";
    }
    return "unknown status";
}

const char *pa_last_cuda_error(void) { return t_cuda_error.c_str(); }

int64_t pa_kernel_launch_count(void) { return pa::g_launches.load(); }

}  // extern "C"

namespace {

// Validates a configuration, allocates a context and its device buffers and
// picks the sweep launch shape; no kernel runs.
pa_status ctx_create(const pa_config &g, void *cuda_stream, pa_ctx **out, int rank = 0, int world = 1)
{
    *out = nullptr;
    if (world < 1 || world > 1024 || rank < 0 || rank >= world) return PA_ERR_INVALID;
    if (g.q < 2 || g.q > 128 || g.L < 2 || g.L > 1024 || (g.L & 1) || g.R < 1 || g.stream < 0 || g.stream > 255)
        return PA_ERR_INVALID;
    if (g.resample_mode < PA_RESAMPLE_NEAREST_INT || g.resample_mode > PA_RESAMPLE_OFF) return PA_ERR_INVALID;
    if (g.init_mode != PA_INIT_RANDOM && g.init_mode != PA_INIT_GROUND) return PA_ERR_INVALID;
    if (!(g.beta0 >= 0.0) || !std::isfinite(g.beta0)) return PA_ERR_INVALID;
    if (pa::replica_bytes(g.q, g.L) > (size_t)pa::kMaxLatticeBytes) return PA_ERR_TOO_LARGE;
    long long R_cap = g.R_cap > 0 ? g.R_cap : (long long)g.R + g.R / 4 + 1024;
    if (R_cap < g.R || R_cap >= (1LL << 24)) return PA_ERR_INVALID;

    pa_ctx *c = new (std::nothrow) pa_ctx();
    if (!c) return PA_ERR_NOMEM;
    c->cfg = g;
    c->cfg.R_cap = (int32_t)R_cap;
    c->N = g.L * g.L;
    c->nbins = 2 * c->N + 1;
    c->rank = rank;
    c->world = world;
    c->shard = world > 1;
    // a shard holds about R_cap / world replicas; the children it sends in one
    // step can exceed its share by the spread of the copy numbers, hence the
    // margin
    c->R_cap = world > 1 ? (int)((R_cap + world - 1) / world + R_cap / (8 * world) + 1024) : (int)R_cap;
    c->R_fill = world > 1 ? (g.R + world - 1) / world : g.R;
    c->stream = (cudaStream_t)cuda_stream;
    c->k0 = (uint32_t)(g.seed & 0xFFFFFFFFu);
    c->k1 = (uint32_t)(g.seed >> 32);
    c->beta = g.beta0;

    pa_status s = PA_OK;
    auto fail = [&](pa_status e) {
        release(c);
        delete c;
        return e;
    };
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(cuda_fail(e));

    const size_t spin_bytes = (size_t)c->R_cap * pa::replica_bytes(g.q, g.L);
    // a shard's children (parent map, run scan) can number up to the whole
    // population's capacity, its own replicas only up to its share
    const int R_child = (int)R_cap;
    const int nb = (R_child + 1023) / 1024;
    if ((s = dev_alloc(&c->spins[0], spin_bytes)) || (s = dev_alloc(&c->spins[1], spin_bytes)) ||
        (s = dev_alloc(&c->E, c->R_cap)) || (s = dev_alloc(&c->Mt, c->R_cap)) ||
        (s = dev_alloc(&c->hist, c->nbins)) || (s = dev_alloc(&c->counts, c->R_cap)) ||
        (s = dev_alloc(&c->local_off, R_child)) || (s = dev_alloc(&c->blocksum, nb)) ||
        (s = dev_alloc(&c->parent, R_child)) || (s = dev_alloc(&c->acc, 4)) || (s = dev_alloc(&c->st, 1)) || (s = dev_alloc(&c->aux, 4)) ||
        (s = dev_alloc(&c->work, 1)))
        return fail(s);
    if (g.track_families) {
        if ((s = dev_alloc(&c->anc[0], c->R_cap)) || (s = dev_alloc(&c->anc[1], c->R_cap)) ||
            (s = dev_alloc(&c->fam, g.R)))
            return fail(s);
    }
    if (c->shard) {
        const size_t runs = (size_t)c->R_cap + world;  // own replicas, plus one split run per destination
        if ((s = dev_alloc(&c->send, runs * pa::replica_words(g.q, g.L))) ||
            (g.track_families && (s = dev_alloc(&c->send_anc, runs))) || (s = dev_alloc(&c->send_cnt, runs)) ||
            (s = dev_alloc(&c->recv_cnt, runs)) || (s = dev_alloc(&c->headpos, runs)) ||
            (s = dev_alloc(&c->bounds, (size_t)world + 1)) || (s = dev_alloc(&c->ent_before, (size_t)world + 1)))
            return fail(s);
    }
    c->obs_cap = 1024;
    if ((s = dev_alloc(&c->obs, c->obs_cap))) return fail(s);
    // staging for the canonical layout of pa_get_spins (at least one replica)
    const size_t canon_bytes = (size_t)c->R_cap * c->N;
    c->stage_bytes = canon_bytes < (64u << 20) ? canon_bytes : (64u << 20);
    if ((s = dev_alloc(&c->stage, c->stage_bytes))) return fail(s);
    e = cudaHostAlloc((void **)&c->host_stage, kStageHist + sizeof(int32_t) * c->nbins, cudaHostAllocDefault);
    if (e != cudaSuccess) {
        c->host_stage = nullptr;
        return fail(cuda_fail(e));
    }
    if ((s = alloc_wtables(c))) return fail(s);
    if ((s = choose_launch(c, 0, 0))) return fail(s);
    *out = c;
    return PA_OK;
}

// Checkpoint file: a fixed header, the population's arrays, and an FNV-1a
// checksum of everything before it.
constexpr char kMagic[8] = {'P', 'A', 'G', 'B', '3', '0', '0', '\x01'};
// 4: spins in the canonical [replica][y][x] byte layout, independent of the
// device layout (versions 2 and 3 stored the device layout)
constexpr uint32_t kVersion = 4;

struct CkptHeader {
    char magic[8];
    uint32_t version, header_bytes;
    pa_config cfg;
    int32_t step, pop;
    double beta, lnZ;
    pa_obs last;
    uint64_t payload_bytes;
};

uint64_t fnv1a(const unsigned char *p, size_t n, uint64_t h)
{
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

}  // namespace

extern "C" {

pa_status pa_init(const pa_config *cfg, void *cuda_stream, pa_ctx **out)
{
    pa::TraceRange trace("pa_init");
    if (!out) return PA_ERR_INVALID;
    *out = nullptr;
    if (!cfg) return PA_ERR_INVALID;
    const pa_config &g = *cfg;
    pa_ctx *c = nullptr;
    pa_status s = ctx_create(g, cuda_stream, &c);
    if (s) return s;
    auto fail = [&](pa_status e) {
        release(c);
        delete c;
        return e;
    };
    pa::DevState h{};
    h.pop = g.R;
    if (g.init_mode == PA_INIT_GROUND)
        h.lnZ = std::log((double)g.q) - g.beta0 * (double)(-2 * c->N);
    else
        h.lnZ = (double)c->N * std::log((double)g.q);
    cudaError_t e = cudaMemcpyAsync(c->st, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->hist, 0, sizeof(int32_t) * c->nbins, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->acc, 0, sizeof(unsigned long long) * 4, c->stream);
    if (e == cudaSuccess && c->fam) e = cudaMemsetAsync(c->fam, 0, sizeof(int32_t) * g.R, c->stream);
    if (e == cudaSuccess)
        e = pa::launch_init(c->spins[0], c->anc[0], g.q, g.L, g.R, c->k0, c->k1, (uint32_t)g.stream << 24,
                            g.init_mode == PA_INIT_GROUND, c->stream);
    if (e != cudaSuccess) return fail(cuda_fail(e));
    if ((s = enqueue_sweep(c, g.beta0, 0, 0))) return fail(s);
    if ((s = sync_state(c, nullptr))) return fail(s);
    *out = c;
    return PA_OK;
}

pa_status pa_save(pa_ctx *c, const char *path)
{
    pa::TraceRange trace("pa_save");
    if (!c || !path) return PA_ERR_INVALID;
    if (c->shard) return PA_ERR_STATE;
    if (c->failed || c->pending_step != 0) return PA_ERR_STATE;
    pa::DevState st;
    pa_status s = sync_state(c, &st);
    if (s) return s;
    const size_t pop = (size_t)st.pop, N = (size_t)c->N;
    const size_t RW = (size_t)pa::replica_words(c->cfg.q, c->cfg.L);
    const bool fam = c->cfg.track_families != 0;
    std::vector<unsigned char> payload(pop * N + 4 * (2 * pop + (size_t)c->nbins + (fam ? pop : 0)));
    unsigned char *p = payload.data();
    // spins in the canonical layout, through the staging buffer
    const size_t per = c->stage_bytes / N;
    for (size_t done = 0; done < pop; done += per) {
        const size_t n = pop - done < per ? pop - done : per;
        PA_CK(pa::launch_to_canonical(c->spins[st.parity] + done * RW, c->stage, c->cfg.q, c->cfg.L, (int64_t)n,
                                      c->stream));
        PA_CK(cudaMemcpyAsync(p + done * N, c->stage, n * N, cudaMemcpyDeviceToHost, c->stream));
        PA_CK(cudaStreamSynchronize(c->stream));
    }
    p += pop * N;
    PA_CK(cudaMemcpy(p, c->E, 4 * pop, cudaMemcpyDeviceToHost));
    p += 4 * pop;
    PA_CK(cudaMemcpy(p, c->Mt, 4 * pop, cudaMemcpyDeviceToHost));
    p += 4 * pop;
    PA_CK(cudaMemcpy(p, c->hist, 4 * (size_t)c->nbins, cudaMemcpyDeviceToHost));
    p += 4 * (size_t)c->nbins;
    if (fam) PA_CK(cudaMemcpy(p, c->anc[st.parity], 4 * pop, cudaMemcpyDeviceToHost));
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kMagic, 8);
    h.version = kVersion;
    h.header_bytes = sizeof(CkptHeader);
    h.cfg = c->cfg;
    h.step = c->step;
    h.pop = st.pop;
    h.beta = c->beta;
    h.lnZ = st.lnZ;
    PA_CK(cudaMemcpy(&h.last, c->obs + ((c->n_obs - 1) % c->obs_cap), sizeof(pa_obs), cudaMemcpyDeviceToHost));
    h.payload_bytes = payload.size();
    uint64_t sum = fnv1a(reinterpret_cast<const unsigned char *>(&h), sizeof(h), 1469598103934665603ull);
    sum = fnv1a(payload.data(), payload.size(), sum);
    FILE *f = std::fopen(path, "wb");
    if (!f) return PA_ERR_INVALID;
    const bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1 &&
                    std::fwrite(payload.data(), 1, payload.size(), f) == payload.size() &&
                    std::fwrite(&sum, sizeof(sum), 1, f) == 1;
    const bool closed = std::fclose(f) == 0;
    return ok && closed ? PA_OK : PA_ERR_INVALID;
}

pa_status pa_load(const char *path, void *cuda_stream, pa_ctx **out)
{
    pa::TraceRange trace("pa_load");
    if (!out) return PA_ERR_INVALID;
    *out = nullptr;
    if (!path) return PA_ERR_INVALID;
    FILE *f = std::fopen(path, "rb");
    if (!f) return PA_ERR_INVALID;
    CkptHeader h;
    std::vector<unsigned char> payload;
    uint64_t sum = 0;
    bool ok = std::fread(&h, sizeof(h), 1, f) == 1 && std::memcmp(h.magic, kMagic, 8) == 0 &&
              h.version == kVersion && h.header_bytes == sizeof(CkptHeader) && h.payload_bytes < (1ull << 40);
    if (ok) {
        payload.resize(h.payload_bytes);
        ok = std::fread(payload.data(), 1, payload.size(), f) == payload.size() &&
             std::fread(&sum, sizeof(sum), 1, f) == 1;
    }
    std::fclose(f);
    if (!ok) return PA_ERR_INVALID;
    uint64_t check = fnv1a(reinterpret_cast<const unsigned char *>(&h), sizeof(h), 1469598103934665603ull);
    check = fnv1a(payload.data(), payload.size(), check);
    if (check != sum) return PA_ERR_INVALID;
    if (h.cfg.q < 2 || h.cfg.q > 128 || h.cfg.L < 2 || h.cfg.L > 1024) return PA_ERR_INVALID;
    const size_t N = (size_t)h.cfg.L * h.cfg.L, pop = (size_t)h.pop;
    const size_t RW = (size_t)pa::replica_words(h.cfg.q, h.cfg.L);
    const bool fam = h.cfg.track_families != 0;
    const size_t nbins = 2 * N + 1;
    if (h.pop < 1 || h.pop > h.cfg.R_cap || h.step < 0 ||
        payload.size() != pop * N + 4 * (2 * pop + nbins + (fam ? pop : 0)))
        return PA_ERR_INVALID;
    for (size_t k = 0; k < pop * N; ++k)
        if (payload[k] >= (unsigned)h.cfg.q) return PA_ERR_INVALID;  // a state outside 0..q-1
    pa_ctx *c = nullptr;
    pa_status s = ctx_create(h.cfg, cuda_stream, &c);
    if (s) return s;
    auto fail = [&](pa_status e) {
        release(c);
        delete c;
        return e;
    };
    const unsigned char *p = payload.data();
    cudaError_t e = cudaSuccess;
    const size_t per = c->stage_bytes / N;
    for (size_t done = 0; done < pop && e == cudaSuccess; done += per) {
        const size_t n = pop - done < per ? pop - done : per;
        e = cudaMemcpy(c->stage, p + done * N, n * N, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = pa::launch_from_canonical(c->spins[0] + done * RW, c->stage, h.cfg.q, h.cfg.L, (int64_t)n, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    p += pop * N;
    if (e == cudaSuccess) e = cudaMemcpy(c->E, p, 4 * pop, cudaMemcpyHostToDevice);
    p += 4 * pop;
    if (e == cudaSuccess) e = cudaMemcpy(c->Mt, p, 4 * pop, cudaMemcpyHostToDevice);
    p += 4 * pop;
    if (e == cudaSuccess) e = cudaMemcpy(c->hist, p, 4 * nbins, cudaMemcpyHostToDevice);
    p += 4 * nbins;
    if (e == cudaSuccess && fam) e = cudaMemcpy(c->anc[0], p, 4 * pop, cudaMemcpyHostToDevice);
    pa::DevState st{};
    st.pop = h.pop;
    st.lnZ = h.lnZ;
    if (e == cudaSuccess) e = cudaMemcpy(c->st, &st, sizeof(st), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(c->acc, 0, sizeof(unsigned long long) * 4);
    if (e == cudaSuccess && c->fam) e = cudaMemset(c->fam, 0, sizeof(int32_t) * h.cfg.R);
    if (e == cudaSuccess) e = cudaMemcpy(c->obs, &h.last, sizeof(pa_obs), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(cuda_fail(e));
    c->n_obs = 1;
    c->step = h.step;
    c->beta = h.beta;
    *out = c;
    return PA_OK;
}

void pa_destroy(pa_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    release(c);
    delete c;
}

pa_status pa_set_launch(pa_ctx *c, int32_t replicas_per_block, int32_t threads_per_block)
{
    if (!c) return PA_ERR_INVALID;
    if (replicas_per_block < 0 || threads_per_block < 0) return PA_ERR_INVALID;
    return choose_launch(c, replicas_per_block, threads_per_block);
}

pa_status pa_get_launch(pa_ctx *c, int32_t *rpb, int32_t *threads, int32_t *blocks)
{
    if (!c) return PA_ERR_INVALID;
    if (rpb) *rpb = c->rpb;
    if (threads) *threads = c->threads;
    if (blocks) *blocks = c->grid;
    return PA_OK;
}

pa_status pa_resample(pa_ctx *c, double dbeta, int32_t step, double *lnQ_out, int32_t *R_out)
{
    pa::TraceRange trace("pa_resample");
    if (!c) return PA_ERR_INVALID;
    if (c->shard) return PA_ERR_STATE;
    if (c->failed || c->pending_step != 0 || step <= c->step) return PA_ERR_STATE;
    if (!std::isfinite(dbeta) || !(c->beta + dbeta >= 0.0)) return PA_ERR_INVALID;
    const bool had_parents = c->resampled;
    pa_status s = enqueue_resample(c, dbeta, step);
    if (s) return s;
    if (lnQ_out || R_out) {
        pa::DevState h;
        s = sync_state(c, &h);
        if (s == PA_ERR_CAPACITY) {
            // undo: clear the flag, the population is still the previous step's
            pa::DevState fix = h;
            fix.err = 0;
            PA_CK(cudaMemcpyAsync(c->st, &fix, sizeof(fix), cudaMemcpyHostToDevice, c->stream));
            PA_CK(cudaStreamSynchronize(c->stream));
            c->failed = false;
            c->pending_step = 0;
            c->resampled = had_parents;  // the scatter stopped before writing parents
            return PA_ERR_CAPACITY;
        }
        if (s) return s;
        if (lnQ_out) *lnQ_out = h.lnQ;
        if (R_out) *R_out = h.pop_next;
    }
    return PA_OK;
}

pa_status pa_sweep(pa_ctx *c, double beta, int32_t theta, int32_t step)
{
    pa::TraceRange trace("pa_sweep");
    if (!c) return PA_ERR_INVALID;
    if (theta < 0 || theta > pa::kMaxTheta || !(beta >= 0.0) || !std::isfinite(beta)) return PA_ERR_INVALID;
    if (c->failed) return PA_ERR_STATE;
    if (c->shard) {
        // after pa_shard_accept (the step's own number), or extra sweeps of a
        // completed step
        if (c->shard_stage == kShardAccepted ? step != c->pending_step
                                             : (c->shard_stage != kShardReady || step != c->step))
            return PA_ERR_STATE;
        // after pa_shard_accept the sweep gathers the new replicas from the
        // received runs
        pa_status s = enqueue_sweep(c, beta, theta, step);
        if (s) return s;
        c->shard_stage = kShardMeasured;
        return PA_OK;
    }
    if (c->pending_step != 0 ? step != c->pending_step : step != c->step) return PA_ERR_STATE;
    return enqueue_sweep(c, beta, theta, step);
}

pa_status pa_energy(pa_ctx *c, int32_t *E_out, int32_t on_device)
{
    if (!c || !E_out) return PA_ERR_INVALID;
    pa::DevState h;
    pa_status s = sync_state(c, &h);
    if (s) return s;
    PA_CK(cudaMemcpyAsync(E_out, c->E, sizeof(int32_t) * h.pop,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (!on_device) PA_CK(cudaStreamSynchronize(c->stream));
    return PA_OK;
}

pa_status pa_occupations(pa_ctx *c, int32_t *Mt_out, int32_t on_device)
{
    if (!c || !Mt_out) return PA_ERR_INVALID;
    pa::DevState h;
    pa_status s = sync_state(c, &h);
    if (s) return s;
    PA_CK(cudaMemcpyAsync(Mt_out, c->Mt, sizeof(int32_t) * h.pop,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (!on_device) PA_CK(cudaStreamSynchronize(c->stream));
    return PA_OK;
}

pa_status pa_observables_history(pa_ctx *c, int32_t count, pa_obs *out)
{
    if (!c || !out || count < 1) return PA_ERR_INVALID;
    if (count > c->n_obs || count > c->obs_cap) return PA_ERR_INVALID;
    pa_status s = sync_state(c, nullptr);
    if (s) return s;
    for (int32_t i = 0; i < count;) {
        const long long rec = c->n_obs - count + i;
        const int at = (int)(rec % c->obs_cap);
        int run = c->obs_cap - at;
        if (run > count - i) run = count - i;
        PA_CK(cudaMemcpyAsync(out + i, c->obs + at, sizeof(pa_obs) * run, cudaMemcpyDeviceToHost, c->stream));
        i += run;
    }
    PA_CK(cudaStreamSynchronize(c->stream));
    return PA_OK;
}

pa_status pa_population_size(pa_ctx *c, int32_t *R_out)
{
    if (!c || !R_out) return PA_ERR_INVALID;
    pa::DevState h;
    pa_status s = sync_state(c, &h);
    if (s) return s;
    *R_out = h.pop;
    return PA_OK;
}

pa_status pa_observables(pa_ctx *c, pa_obs *out, int32_t *hist_out, int32_t hist_len)
{
    pa::TraceRange trace("pa_observables");
    if (!c || !out) return PA_ERR_INVALID;
    if (hist_out && hist_len < c->nbins) return PA_ERR_INVALID;
    // one round trip: the device state, the latest record and the histogram
    // into pinned staging, a single synchronisation, then the error check
    pa::DevState *h = reinterpret_cast<pa::DevState *>(c->host_stage);
    pa_obs *rec = reinterpret_cast<pa_obs *>(c->host_stage + kStageObs);
    int32_t *hist = reinterpret_cast<int32_t *>(c->host_stage + kStageHist);
    const pa::DevObs *slot = c->obs + ((c->n_obs - 1) % c->obs_cap);
    static_assert(sizeof(pa::DevObs) == sizeof(pa_obs), "pa_obs layout");
    PA_CK(cudaMemcpyAsync(h, c->st, sizeof(pa::DevState), cudaMemcpyDeviceToHost, c->stream));
    PA_CK(cudaMemcpyAsync(rec, slot, sizeof(pa_obs), cudaMemcpyDeviceToHost, c->stream));
    if (hist_out)
        PA_CK(cudaMemcpyAsync(hist, c->hist, sizeof(int32_t) * c->nbins, cudaMemcpyDeviceToHost, c->stream));
    PA_CK(cudaStreamSynchronize(c->stream));
    if (h->err != 0) {
        c->failed = true;
        return (pa_status)h->err;
    }
    *out = *rec;
    if (hist_out) std::memcpy(hist_out, hist, sizeof(int32_t) * c->nbins);
    return PA_OK;
}

pa_status pa_get_spins(pa_ctx *c, int64_t slot_begin, int64_t count, uint8_t *host)
{
    if (!c || !host || slot_begin < 0 || count < 0) return PA_ERR_INVALID;
    pa::DevState h;
    pa_status s = sync_state(c, &h);
    if (s) return s;
    if (slot_begin + count > h.pop) return PA_ERR_INVALID;
    const int64_t per = (int64_t)(c->stage_bytes / c->N);
    for (int64_t done = 0; done < count; done += per) {
        const int64_t n = count - done < per ? count - done : per;
        const size_t RW = (size_t)pa::replica_words(c->cfg.q, c->cfg.L);
        PA_CK(pa::launch_to_canonical(c->spins[h.parity] + (size_t)(slot_begin + done) * RW, c->stage, c->cfg.q,
                                      c->cfg.L, n, c->stream));
        PA_CK(cudaMemcpyAsync(host + (size_t)done * c->N, c->stage, (size_t)n * c->N, cudaMemcpyDeviceToHost,
                              c->stream));
        PA_CK(cudaStreamSynchronize(c->stream));
    }
    return PA_OK;
}

pa_status pa_get_ancestors(pa_ctx *c, int32_t *host)
{
    if (!c || !host) return PA_ERR_INVALID;
    if (!c->cfg.track_families) return PA_ERR_STATE;
    pa::DevState h;
    pa_status s = sync_state(c, &h);
    if (s) return s;
    PA_CK(cudaMemcpyAsync(host, c->anc[h.parity], sizeof(int32_t) * h.pop, cudaMemcpyDeviceToHost, c->stream));
    PA_CK(cudaStreamSynchronize(c->stream));
    return PA_OK;
}

pa_status pa_get_parents(pa_ctx *c, int32_t *out, int32_t on_device)
{
    if (!c || !out) return PA_ERR_INVALID;
    if (!c->resampled) return PA_ERR_STATE;
    pa::DevState h;
    pa_status s = sync_state(c, &h);
    if (s) return s;
    const int n = c->pending_step != 0 ? h.pop_next : h.pop;
    PA_CK(cudaMemcpyAsync(out, c->parent, sizeof(int32_t) * (size_t)n,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (!on_device) PA_CK(cudaStreamSynchronize(c->stream));
    return PA_OK;
}

pa_status pa_shard_plan(const int64_t *totals, int32_t world, int32_t rank, int64_t *R_new, int64_t *lo, int64_t *hi,
                        int64_t *send_counts, int64_t *recv_counts)
{
    if (!totals || world < 1 || world > 1024 || rank < 0 || rank >= world) return PA_ERR_INVALID;
    int64_t R = 0;
    for (int g = 0; g < world; ++g) {
        if (totals[g] < 0) return PA_ERR_INVALID;
        R += totals[g];
    }
    if (R < 1 || R >= (int64_t)1 << 24) return PA_ERR_CAPACITY;
    auto bound = [&](int64_t d) { return d * R / world; };
    auto overlap = [](int64_t a0, int64_t a1, int64_t b0, int64_t b1) {
        const int64_t x = std::max(a0, b0), y = std::min(a1, b1);
        return y > x ? y - x : (int64_t)0;
    };
    // rank g's children are the new slots [O_g, O_g + T_g), O_g = sum_{h<g} T_h
    int64_t O = 0, my0 = 0;
    for (int g = 0; g < rank; ++g) O += totals[g];
    my0 = O;
    const int64_t b0 = bound(rank), b1 = bound(rank + 1);
    int64_t Og = 0;
    for (int g = 0; g < world; ++g) {
        if (send_counts) send_counts[g] = overlap(my0, my0 + totals[rank], bound(g), bound(g + 1));
        if (recv_counts) recv_counts[g] = overlap(Og, Og + totals[g], b0, b1);
        Og += totals[g];
    }
    if (R_new) *R_new = R;
    if (lo) *lo = b0;
    if (hi) *hi = b1;
    return PA_OK;
}

pa_status pa_shard_init(const pa_config *cfg, int32_t rank, int32_t world, void *cuda_stream, pa_ctx **out)
{
    pa::TraceRange trace("pa_shard_init");
    if (!out) return PA_ERR_INVALID;
    *out = nullptr;
    if (!cfg || world < 2) return PA_ERR_INVALID;
    const pa_config &g = *cfg;
    pa_ctx *c = nullptr;
    pa_status s = ctx_create(g, cuda_stream, &c, rank, world);
    if (s) return s;
    auto fail = [&](pa_status e) {
        release(c);
        delete c;
        return e;
    };
    const int lo = (int)((int64_t)rank * g.R / world), hi = (int)((int64_t)(rank + 1) * g.R / world);
    c->slot0 = lo;
    c->R_all = g.R;
    pa::DevState h{};
    h.pop = hi - lo;
    if (g.init_mode == PA_INIT_GROUND)
        h.lnZ = std::log((double)g.q) - g.beta0 * (double)(-2 * c->N);
    else
        h.lnZ = (double)c->N * std::log((double)g.q);
    cudaError_t e = cudaMemcpyAsync(c->st, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->hist, 0, sizeof(int32_t) * c->nbins, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->acc, 0, sizeof(unsigned long long) * 4, c->stream);
    if (e == cudaSuccess && c->fam) e = cudaMemsetAsync(c->fam, 0, sizeof(int32_t) * g.R, c->stream);
    if (e == cudaSuccess && hi > lo)
        e = pa::launch_init(c->spins[0], c->anc[0], g.q, g.L, hi - lo, c->k0, c->k1, (uint32_t)g.stream << 24,
                            g.init_mode == PA_INIT_GROUND, c->stream, (uint32_t)lo);
    if (e != cudaSuccess) return fail(cuda_fail(e));
    if ((s = enqueue_sweep(c, g.beta0, 0, 0))) return fail(s);
    if ((s = sync_state(c, nullptr))) return fail(s);
    c->shard_stage = kShardMeasured;
    c->shard_resampled = false;
    *out = c;
    return PA_OK;
}

pa_status pa_shard_get_buffers(pa_ctx *c, pa_shard_buffers *out)
{
    if (!c || !out) return PA_ERR_INVALID;
    if (!c->shard) return PA_ERR_STATE;
    const int nxt = c->host_parity ^ 1;
    out->hist = c->hist;
    out->sums = reinterpret_cast<int64_t *>(c->acc);
    out->fam = c->fam;
    out->send = c->send;
    out->send_anc = c->send_anc;
    out->send_cnt = c->send_cnt;
    out->recv = c->spins[nxt];
    out->recv_anc = c->anc[nxt];
    out->recv_cnt = c->recv_cnt;
    out->replica_words = pa::replica_words(c->cfg.q, c->cfg.L);
    out->capacity = c->R_cap;
    out->n_bins = c->nbins;
    return PA_OK;
}

pa_status pa_shard_finalize(pa_ctx *c, double beta)
{
    pa::TraceRange trace("pa_shard_finalize");
    if (!c || !std::isfinite(beta)) return PA_ERR_INVALID;
    if (!c->shard || c->failed || c->shard_stage != kShardMeasured) return PA_ERR_STATE;
    const int gathered = c->shard_resampled ? 1 : 0;
    PA_CK(pa::launch_finalize(c->st, c->acc, c->fam, c->cfg.R, next_obs_slot(c), beta, c->cfg.q, c->N, gathered,
                              gathered, c->stream, c->R_all));
    c->host_parity ^= gathered;  // the gathering sweep wrote the other buffer
    c->shard_resampled = false;
    c->shard_stage = kShardReady;
    return PA_OK;
}

pa_status pa_shard_counts(pa_ctx *c, double dbeta, int32_t step, int64_t *local_total)
{
    pa::TraceRange trace("pa_shard_counts");
    if (!c || !local_total) return PA_ERR_INVALID;
    if (!c->shard || c->failed || c->shard_stage != kShardReady || step <= c->step) return PA_ERR_STATE;
    if (!std::isfinite(dbeta) || !(c->beta + dbeta >= 0.0)) return PA_ERR_INVALID;
    const double *wtab = nullptr;
    pa_status s = get_wtable(c, dbeta, &wtab);
    if (s) return s;
    PA_CK(pa::launch_resample(c->hist, c->nbins, c->E, dbeta, c->cfg.R, c->cfg.R_cap, c->cfg.resample_mode, step,
                              (uint32_t)c->cfg.stream << 24, c->k0, c->k1, wtab, c->counts, c->local_off,
                              c->blocksum, c->parent, c->hist, c->st, c->stream, c->slot0, c->R_all));
    pa::DevState h;
    s = sync_state(c, &h);
    if (s == PA_ERR_CAPACITY) {
        // this rank's children exceed its buffers: the population stays at step i-1
        pa::DevState fix = h;
        fix.err = 0;
        PA_CK(cudaMemcpyAsync(c->st, &fix, sizeof(fix), cudaMemcpyHostToDevice, c->stream));
        PA_CK(cudaStreamSynchronize(c->stream));
        c->failed = false;
        return PA_ERR_CAPACITY;
    }
    if (s) return s;
    // this rank's near ties join the sums that the caller adds over the ranks
    const int64_t ties = h.ties;
    PA_CK(cudaMemcpyAsync(c->acc + 3, &ties, sizeof(ties), cudaMemcpyHostToDevice, c->stream));
    c->n_pack = h.pop_next;
    c->pending_step = step;
    c->resampled = true;
    c->shard_stage = kShardCounted;
    *local_total = h.pop_next;
    return PA_OK;
}

pa_status pa_shard_pack(pa_ctx *c, const int64_t *totals, int64_t *send_counts)
{
    pa::TraceRange trace("pa_shard_pack");
    if (!c || !totals || !send_counts) return PA_ERR_INVALID;
    if (!c->shard || c->failed || c->shard_stage != kShardCounted) return PA_ERR_STATE;
    if (totals[c->rank] != c->n_pack) return PA_ERR_INVALID;
    int64_t R_new = 0, lo = 0, hi = 0;
    pa_status s = pa_shard_plan(totals, c->world, c->rank, &R_new, &lo, &hi, nullptr, nullptr);
    if (s) return s;
    if (hi - lo > c->R_cap || R_new > c->cfg.R_cap) return PA_ERR_CAPACITY;
    // destination bounds in this rank's child order: its children are the new
    // slots [O, O + T), rank d holds [floor(d R_new / world), ...)
    int64_t O = 0;
    for (int g = 0; g < c->rank; ++g) O += totals[g];
    const int T = c->n_pack, G = c->world;
    std::vector<int32_t> A((size_t)G + 1);
    for (int d = 0; d <= G; ++d) {
        const int64_t b = (int64_t)d * R_new / G - O;
        A[d] = (int32_t)(b < 0 ? 0 : b > T ? T : b);
    }
    PA_CK(cudaMemcpyAsync(c->bounds, A.data(), sizeof(int32_t) * A.size(), cudaMemcpyHostToDevice, c->stream));
    PA_CK(pa::launch_shard_runs(c->parent, T, c->bounds, G, c->local_off, c->blocksum, c->headpos, c->ent_before,
                                c->stream));
    std::vector<long long> ent((size_t)G + 1);
    PA_CK(cudaMemcpyAsync(ent.data(), c->ent_before, sizeof(long long) * ent.size(), cudaMemcpyDeviceToHost,
                          c->stream));
    PA_CK(cudaStreamSynchronize(c->stream));
    const long long E = ent[G];
    if (E > (long long)c->R_cap + G) return PA_ERR_CAPACITY;
    PA_CK(pa::launch_shard_pack(c->spins[c->host_parity], c->cfg.track_families ? c->anc[c->host_parity] : nullptr,
                                c->parent, c->headpos, (int)E, T, pa::replica_words(c->cfg.q, c->cfg.L), c->send,
                                c->send_anc, c->send_cnt, c->stream));
    for (int d = 0; d < G; ++d) send_counts[d] = ent[d + 1] - ent[d];
    c->slot0_next = (int)lo;
    c->n_next = (int)(hi - lo);
    c->R_all_next = (int)R_new;
    c->shard_stage = kShardPacked;
    return PA_OK;
}

pa_status pa_shard_accept(pa_ctx *c, const int64_t *recv_counts)
{
    pa::TraceRange trace("pa_shard_accept");
    if (!c || !recv_counts) return PA_ERR_INVALID;
    if (!c->shard || c->failed || c->shard_stage != kShardPacked) return PA_ERR_STATE;
    int64_t n = 0;
    for (int g = 0; g < c->world; ++g) {
        if (recv_counts[g] < 0) return PA_ERR_INVALID;
        n += recv_counts[g];
    }
    if (n > c->n_next) return PA_ERR_INVALID;  // every received run has at least one child here
    PA_CK(pa::launch_shard_accept(c->st, c->recv_cnt, (int)n, c->n_next, c->R_cap, c->local_off, c->blocksum,
                                  c->parent, c->hist, c->nbins, c->stream));
    c->host_parity ^= 1;  // the received runs are the current buffer until the sweep gathers from them
    c->slot0 = c->slot0_next;
    c->R_all = c->R_all_next;
    c->n_runs = (int)n;
    c->shard_resampled = true;
    c->shard_stage = kShardAccepted;
    return PA_OK;
}

pa_status pa_shard_range(pa_ctx *c, int64_t *slot0, int64_t *count, int64_t *R_all)
{
    if (!c) return PA_ERR_INVALID;
    if (!c->shard) return PA_ERR_STATE;
    pa::DevState h;
    pa_status s = sync_state(c, &h);
    if (s) return s;
    if (slot0) *slot0 = c->slot0;
    if (count) *count = h.pop;
    if (R_all) *R_all = c->R_all;
    return PA_OK;
}

pa_status pa_run(pa_ctx *c, const double *betas, int32_t K, int32_t theta, pa_obs *obs_out,
                 const int32_t *hist_steps, int32_t n_hist, int32_t *hist_out, int32_t use_graph)
{
    pa::TraceRange trace("pa_run");
    if (!c || !betas || K < 1 || theta < 0 || theta > pa::kMaxTheta || n_hist < 0 || (n_hist > 0 && (!hist_steps || !hist_out)))
        return PA_ERR_INVALID;
    if (c->shard) return PA_ERR_STATE;
    if (c->failed || c->pending_step != 0) return PA_ERR_STATE;
    for (int i = 0; i <= K; ++i)
        if (!std::isfinite(betas[i]) || !(betas[i] >= 0.0)) return PA_ERR_INVALID;
    for (int h = 0; h < n_hist; ++h)
        if (hist_steps[h] < 1 || hist_steps[h] > K) return PA_ERR_INVALID;

    // estimator slots for K steps, contiguous
    if (c->obs_cap < K + 1) {
        PA_CK(cudaStreamSynchronize(c->stream));
        pa::DevObs *bigger = nullptr;
        pa_status s = dev_alloc(&bigger, (size_t)K + 1);
        if (s) return s;
        PA_CK(cudaMemcpy(bigger, c->obs + ((c->n_obs - 1) % c->obs_cap), sizeof(pa::DevObs), cudaMemcpyDeviceToDevice));
        cudaFree(c->obs);
        c->obs = bigger;
        c->obs_cap = K + 1;
        c->n_obs = 1;
    }
    int32_t *hstore = nullptr;
    if (n_hist > 0) {
        pa_status s = dev_alloc(&hstore, (size_t)n_hist * c->nbins);
        if (s) return s;
    }
    const long long first_obs = c->n_obs;
    const int step0 = c->step;
    // every weight table of the schedule is on the device before any capture
    // begins and stays until the run has finished: in the arena when the
    // schedule has at most kWTableSlots distinct steps (loaded in turn, none
    // evicts another), else in tables of the run's own
    {
        std::vector<uint64_t> keys;
        for (int i = 1; i <= K; ++i) {
            const double d = betas[i] - betas[i - 1];
            uint64_t key;
            std::memcpy(&key, &d, sizeof(key));
            if (std::find(keys.begin(), keys.end(), key) == keys.end()) keys.push_back(key);
        }
        pa_status s = PA_OK;
        if (keys.size() <= (size_t)kWTableSlots) {
            for (uint64_t key : keys) {
                double d;
                std::memcpy(&d, &key, sizeof(d));
                const double *w = nullptr;
                if ((s = get_wtable(c, d, &w))) break;
            }
        } else {
            const size_t n = (size_t)c->nbins;
            std::vector<double> host(n * keys.size());
            if (!(s = dev_alloc(&c->wt_run, host.size()))) {
                for (size_t k = 0; k < keys.size(); ++k) {
                    double d;
                    std::memcpy(&d, &keys[k], sizeof(d));
                    pa::weight_table(d, c->nbins, host.data() + n * k);
                    c->wt_run_at.emplace_back(keys[k], c->wt_run + n * k);
                }
                cudaError_t e = cudaMemcpyAsync(c->wt_run, host.data(), sizeof(double) * host.size(),
                                                cudaMemcpyHostToDevice, c->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
                if (e != cudaSuccess) s = cuda_fail(e);
            }
        }
        if (s) {
            release_run_tables(c);
            if (hstore) cudaFree(hstore);
            return s;
        }
    }

    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    pa_status s = PA_OK;
    // The graph is captured on a private stream (the legacy default stream
    // cannot be captured) and launched on the context's stream.
    const bool was_profiling = c->profiling;
    cudaStream_t user_stream = c->stream;
    if (use_graph) {
        c->profiling = false;
        cudaError_t e = cudaSuccess;
        if (!c->capture_stream) e = cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            c->profiling = was_profiling;
            release_run_tables(c);
            if (hstore) cudaFree(hstore);
            return cuda_fail(e);
        }
        c->stream = c->capture_stream;
    }
    for (int i = 1; i <= K && s == PA_OK; ++i) {
        s = enqueue_resample(c, betas[i] - betas[i - 1], step0 + i);
        if (s == PA_OK) s = enqueue_sweep(c, betas[i], theta, step0 + i);
        for (int h = 0; h < n_hist && s == PA_OK; ++h) {
            if (hist_steps[h] == i) {
                cudaError_t e = cudaMemcpyAsync(hstore + (size_t)h * c->nbins, c->hist, sizeof(int32_t) * c->nbins,
                                                cudaMemcpyDeviceToDevice, c->stream);
                if (e != cudaSuccess) s = cuda_fail(e);
            }
        }
    }
    if (use_graph) {
        cudaError_t e = cudaStreamEndCapture(c->capture_stream, &graph);
        c->stream = user_stream;
        if (e == cudaSuccess && s == PA_OK) e = cudaGraphInstantiate(&exec, graph, 0);
        if (e == cudaSuccess && s == PA_OK) e = cudaGraphLaunch(exec, c->stream);
        if (e != cudaSuccess && s == PA_OK) s = cuda_fail(e);
    }
    c->profiling = was_profiling;
    if (s == PA_OK) s = sync_state(c, nullptr);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamSynchronize(c->stream);
    release_run_tables(c);
    if (s == PA_OK && obs_out) {
        for (int i = 0; i < K; ++i) {
            const pa::DevObs *slot = c->obs + ((first_obs + i) % c->obs_cap);
            cudaError_t e = cudaMemcpy(obs_out + i, slot, sizeof(pa_obs), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) {
                s = cuda_fail(e);
                break;
            }
        }
    }
    if (s == PA_OK && n_hist > 0) {
        cudaError_t e = cudaMemcpy(hist_out, hstore, sizeof(int32_t) * (size_t)n_hist * c->nbins,
                                   cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) s = cuda_fail(e);
    }
    if (hstore) cudaFree(hstore);
    return s;
}

pa_status pa_next_dbeta(pa_ctx *c, double target, double dbeta_cap, int32_t iters, double *dbeta_out)
{
    pa::TraceRange trace("pa_next_dbeta");
    if (!c || !dbeta_out || !(target > 0.0 && target < 1.0) || !(dbeta_cap > 0.0) || !std::isfinite(dbeta_cap) ||
        iters < 0 || iters > 200)
        return PA_ERR_INVALID;
    if (c->shard) return PA_ERR_STATE;
    if (c->failed || c->pending_step != 0) return PA_ERR_STATE;
    PA_CK(pa::launch_newton(c->hist, c->nbins, c->st, target, dbeta_cap, iters, c->aux, c->stream));
    double h[2];
    PA_CK(cudaMemcpyAsync(h, c->aux, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    pa_status s = sync_state(c, nullptr);
    if (s) return s;
    *dbeta_out = h[0];
    return PA_OK;
}

pa_status pa_run_adaptive(pa_ctx *c, double beta_end, double target, double dbeta_max, int32_t iters, int32_t theta,
                          int32_t max_steps, pa_obs *obs_out, double *betas_out, int32_t *K_out)
{
    pa::TraceRange trace("pa_run_adaptive");
    if (!c || !K_out || theta < 0 || theta > pa::kMaxTheta || max_steps < 1 || !(beta_end >= 0.0) || !std::isfinite(beta_end) ||
        !(dbeta_max > 0.0))
        return PA_ERR_INVALID;
    if (c->failed || c->pending_step != 0) return PA_ERR_STATE;
    if (c->obs_cap < max_steps + 1) {
        PA_CK(cudaStreamSynchronize(c->stream));
        pa::DevObs *bigger = nullptr;
        pa_status s = dev_alloc(&bigger, (size_t)max_steps + 1);
        if (s) return s;
        PA_CK(cudaMemcpy(bigger, c->obs + ((c->n_obs - 1) % c->obs_cap), sizeof(pa::DevObs), cudaMemcpyDeviceToDevice));
        cudaFree(c->obs);
        c->obs = bigger;
        c->obs_cap = max_steps + 1;
        c->n_obs = 1;
    }
    const long long first_obs = c->n_obs;
    double beta = c->beta;
    int K = 0;
    while (beta < beta_end && K < max_steps) {
        const double room = beta_end - beta;
        const double cap = dbeta_max < room ? dbeta_max : room;
        double dbeta = 0.0;
        pa_status s = pa_next_dbeta(c, target, cap, iters, &dbeta);
        if (s) return s;
        const double nb = (dbeta == room) ? beta_end : beta + dbeta;
        const int step = c->step + 1;
        if ((s = enqueue_resample(c, dbeta, step)) || (s = enqueue_sweep(c, nb, theta, step))) return s;
        K += 1;
        if (betas_out) betas_out[K - 1] = nb;
        beta = nb;
    }
    pa_status s = sync_state(c, nullptr);
    if (s) return s;
    if (obs_out) {
        for (int i = 0; i < K; ++i) {
            const pa::DevObs *slot = c->obs + ((first_obs + i) % c->obs_cap);
            PA_CK(cudaMemcpy(obs_out + i, slot, sizeof(pa_obs), cudaMemcpyDeviceToHost));
        }
    }
    *K_out = K;
    return PA_OK;
}

pa_status pa_profile(pa_ctx *c, int32_t enable)
{
    if (!c) return PA_ERR_INVALID;
    PA_CK(cudaStreamSynchronize(c->stream));
    c->ev_used[0] = c->ev_used[1] = 0;
    c->profiling = enable != 0;
    return PA_OK;
}

pa_status pa_profile_read(pa_ctx *c, double *ms_out2, int64_t *launches_out2)
{
    if (!c) return PA_ERR_INVALID;
    PA_CK(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < 2; ++k) {
        double total = 0.0;
        for (int64_t i = 0; i < c->ev_used[k]; ++i) {
            float ms = 0.f;
            PA_CK(cudaEventElapsedTime(&ms, c->ev[k][2 * i], c->ev[k][2 * i + 1]));
            total += ms;
        }
        if (ms_out2) ms_out2[k] = total;
        if (launches_out2) launches_out2[k] = c->ev_used[k];
    }
    return PA_OK;
}

}  // extern "C"
